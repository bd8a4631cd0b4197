"""FP64 CPU oracle of the L1 IRLS + PCG phase-unwrapping method (test infrastructure only).

This is the plain, slow, obviously-correct statement of what the CUDA path computes.  It follows
the paper's steps in the paper's order and notation, with dense NumPy algebra and no blocking or
fusion.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` use it.

Notation (Sec. 2):  X is the N x M wrapped phase; U the N x M unwrapped estimate; Gv, Cv, Vv,
Wv live on the (N-1) x M vertical edges and Gh, Ch, Vh, Wh on the N x (M-1) horizontal edges;
S is the (N-1) x N forward difference (S U)_{ij} = U_{i+1,j} - U_{ij}; T is the M x (M-1)
difference with (U T)_{ij} = U_{i,j+1} - U_{ij}.

Readings where the paper is silent or inconsistent (each is repeated in the design notes):
  * wrap: "mod 2 pi" of a difference is taken as the representative in [-pi, pi), evaluated
    in float32 as t - 2pi * floor((t + pi) / 2pi) with t = fl32(X1 - X0) and 2pi, pi the float32
    constants (the wrap decides an integer, so both sides decide it in the same precision);
  * the linear system is the symmetric one of Prop. (linear system) / eq. (vectorised A, b),
    not the unscaled U row printed inside Alg. 1;
  * CG is warm-started from the current IRLS iterate (Alg. 2 leaves the start open);
  * CG stops when ||r||_2 / ||b||_2 <= cg_tol (full three-block residual) or after cg_max
    matrix-vector products;
  * coherence -> edge weights: Cv_ij = (coh_ij + coh_{i+1,j}) / 2, Ch_ij = (coh_ij + coh_{i,j+1}) / 2;
  * the singular preconditioner uses the pseudo-inverse (zero-frequency DCT coefficient -> 0,
    Appendix B) and U is shifted to zero mean after every solve (Prop. 'minimising (alt1)');
  * eps of the library's signature is the smoothing delta of F_delta (Sec. 3.1); tau defaults to
    the paper's 1e-2 (Sec. 4.4).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "TWO_PI_F32", "PI_F32", "wrap_f32", "wrapped_gradients", "edge_weights",
    "S_op", "St_op", "T_op", "Tt_op", "rhs_b", "apply_A", "reweight", "diag_d", "dD_dV", "dD_dC",
    "dct_basis", "precond_apply", "pcg", "l1_objective", "F_value", "F_delta_value",
    "H_delta_value", "gradient_candidate", "smoothness_L", "irls_unwrap", "paper_cg_cap", "k_map",
    "round_congruent", "schur_weights", "schur_matvec", "schur_rhs", "schur_recover_v",
    "pcg_schur",
    "best_shift_error", "dense_operators", "Problem", "irls_adjoint",
    "tile_starts", "tile_cores", "overlap_offset", "stitch_tiles", "irls_unwrap_tiled",
]

TWO_PI_F32 = np.float32(2.0 * np.pi)
PI_F32 = np.float32(np.pi)


# --------------------------------------------------------------------------------------------
# Sec. 2: wrapped phase gradients and weights
# --------------------------------------------------------------------------------------------
def wrap_f32(t):
    """Wrapped value of a float32 phase difference, in [-pi, pi) (Sec. 2, 'mod 2 pi').

    Evaluated in float32, one correctly rounded operation at a time:
    k = floor((t + pi) / 2pi), result = t - (2pi * k)."""
    t = np.asarray(t, dtype=np.float32)
    k = np.floor((t + PI_F32) / TWO_PI_F32).astype(np.float32)
    prod = (TWO_PI_F32 * k).astype(np.float32)
    return (t - prod).astype(np.float32)


def wrapped_gradients(X):
    """Gv = wrap(X_{i+1,j} - X_{ij}) ((N-1) x M) and Gh = wrap(X_{i,j+1} - X_{ij}) (N x (M-1)),
    Sec. 2.  The float32 input difference is formed in float32, then held in float64."""
    X = np.asarray(X, dtype=np.float32)
    dv = (X[1:, :] - X[:-1, :]).astype(np.float32)
    dh = (X[:, 1:] - X[:, :-1]).astype(np.float32)
    return wrap_f32(dv).astype(np.float64), wrap_f32(dh).astype(np.float64)


def edge_weights(coherence, N, M):
    """Edge weights (Cv, Ch) of problem (main), Sec. 2.  Uniform weights (all ones) when no
    coherence is given (Sec. 4.4, 'uniform'); otherwise the mean of the two end-pixel
    coherences of each edge."""
    if coherence is None:
        return np.ones((N - 1, M)), np.ones((N, M - 1))
    c = np.asarray(coherence, dtype=np.float64)
    return 0.5 * (c[1:, :] + c[:-1, :]), 0.5 * (c[:, 1:] + c[:, :-1])


# --------------------------------------------------------------------------------------------
# Sec. 2: difference operators S, T and their transposes (definitions of S_N and T_M)
# --------------------------------------------------------------------------------------------
def S_op(U):
    """(S U)_{ij} = U_{i+1,j} - U_{ij}, S in R^{(N-1) x N}."""
    return U[1:, :] - U[:-1, :]


def St_op(Y, N):
    """S^T Y for Y of shape (N-1) x M: (S^T Y)_i = Y_{i-1} [i >= 1] - Y_i [i <= N-2]."""
    out = np.zeros((N, Y.shape[1]))
    out[1:, :] += Y
    out[:-1, :] -= Y
    return out


def T_op(U):
    """(U T)_{ij} = U_{i,j+1} - U_{ij}, T in R^{M x (M-1)}."""
    return U[:, 1:] - U[:, :-1]


def Tt_op(Y, M):
    """Y T^T for Y of shape N x (M-1): (Y T^T)_{:,j} = Y_{:,j-1} [j >= 1] - Y_{:,j} [j <= M-2]."""
    out = np.zeros((Y.shape[0], M))
    out[:, 1:] += Y
    out[:, :-1] -= Y
    return out


# --------------------------------------------------------------------------------------------
# Sec. 3.1 / 3.2: reweighting, linear system, right-hand side
# --------------------------------------------------------------------------------------------
def reweight(Vv, Vh, Cv, Ch, delta):
    """Closed-form weight update W = sqrt(C^2 V^2 + delta^2) (Sec. 3.1, Alg. 1)."""
    return np.sqrt(Cv * Cv * Vv * Vv + delta * delta), np.sqrt(Ch * Ch * Vh * Vh + delta * delta)


def diag_d(Cv, Ch, Wv, Wh):
    """Diagonal blocks Dv = C^2 / W, Dh = C^2 / W of the vectorised matrix A (Sec. 3.2)."""
    return Cv * Cv / Wv, Ch * Ch / Wh


def dD_dV(C, V, W):
    """Derivative of D = C^2 / W with W = sqrt(C^2 V^2 + delta^2) (Sec. 3.1) in V, per edge:
    dD/dV = -C^2 / W^2 * dW/dV = -C^4 V / W^3."""
    return -(C ** 4) * V / W ** 3


def dD_dC(C, V, W):
    """Derivative of D = C^2 / W in C, per edge: 2 C / W - C^2 / W^2 * dW/dC
    = 2 C / W - C^3 V^2 / W^3."""
    return 2.0 * C / W - C ** 3 * V ** 2 / W ** 3


def rhs_b(Gv, Gh, tau):
    """b = (B1, B2, B3) with B1 = (S^T Gv + Gh T^T) / tau, B2 = -Gv / tau, B3 = -Gh / tau
    (Sec. 3.2, definition of B1, B2, B3)."""
    N, M = Gh.shape[0], Gv.shape[1]
    return ((St_op(Gv, N) + Tt_op(Gh, M)) / tau, -Gv / tau, -Gh / tau)


def apply_A(x, dv, dh, tau):
    """Left-hand side of the linear system (Prop. 'linear system', Sec. 3.1):

        q_U  = (S^T S U + U T T^T - S^T Vv - Vh T^T) / tau
        q_Vv = Dv o Vv + (Vv - S U) / tau
        q_Vh = Dh o Vh + (Vh - U T) / tau
    """
    U, Vv, Vh = x
    N, M = U.shape
    SU, UT = S_op(U), T_op(U)
    qU = (St_op(SU, N) + Tt_op(UT, M) - St_op(Vv, N) - Tt_op(Vh, M)) / tau
    qVv = dv * Vv + (Vv - SU) / tau
    qVh = dh * Vh + (Vh - UT) / tau
    return (qU, qVv, qVh)


# --------------------------------------------------------------------------------------------
# Sec. 3.3: block-diagonal preconditioner, Sylvester block by eigendecomposition
# --------------------------------------------------------------------------------------------
def dct_basis(N):
    """Eigendecomposition S^T S = P diag(lam) P^T of the 1-D Neumann Laplacian (Sec. 3.3).

    Closed form (orthonormal DCT-II vectors): P[i, k] = c_k cos(pi k (i + 1/2) / N),
    c_0 = sqrt(1/N), c_k = sqrt(2/N); lam_k = 2 - 2 cos(pi k / N)."""
    i = np.arange(N, dtype=np.float64)[:, None]
    k = np.arange(N, dtype=np.float64)[None, :]
    c = np.full((1, N), math.sqrt(2.0 / N))
    c[0, 0] = math.sqrt(1.0 / N)
    P = c * np.cos(np.pi * k * (i + 0.5) / N)
    lam = 2.0 - 2.0 * np.cos(np.pi * np.arange(N, dtype=np.float64) / N)
    return P, lam


def precond_apply(r, dv, dh, tau, basis_N, basis_M):
    """z = D^+ r for the block-diagonal preconditioner D (Sec. 3.3).

    U block: solve S^T S Z + Z T T^T = tau R by Z = P_S [(P_S^T tau R P_T) / (lam_i + mu_j)] P_T^T,
    with the zero-frequency coefficient set to 0 (the pseudo-inverse choice of Appendix B).
    V blocks: z = r / (D + 1/tau)."""
    rU, rVv, rVh = r
    PN, lamN = basis_N
    PM, lamM = basis_M
    Y = PN.T @ (tau * rU) @ PM
    den = lamN[:, None] + lamM[None, :]
    Zp = np.zeros_like(Y)
    nz = den > 0
    nz[0, 0] = False
    Zp[nz] = Y[nz] / den[nz]
    zU = PN @ Zp @ PM.T
    return (zU, rVv / (dv + 1.0 / tau), rVh / (dh + 1.0 / tau))


# --------------------------------------------------------------------------------------------
# Alg. 2: preconditioned conjugate gradient
# --------------------------------------------------------------------------------------------
def _dot(a, b):
    return float(sum(np.vdot(x, y) for x, y in zip(a, b)))


def _axpy(alpha, x, y):
    return tuple(yi + alpha * xi for xi, yi in zip(x, y))


def _stored(v, storage):
    if storage is None:
        return v
    return tuple(np.asarray(a, dtype=storage).astype(np.float64) for a in v)


def pcg(x0, b, dv, dh, tau, basis_N, basis_M, tol, cg_max, beta_rule="fr", storage=None,
        precond_rounding=None):
    """Preconditioned CG (Alg. 2) on A x = b from the warm start x0.

    Stops when ||r|| / ||b|| <= tol or after cg_max products with A.  ``beta_rule`` 'fr' is the
    Fletcher-Reeves ratio printed in Alg. 2; 'pr' is the Polak-Ribiere (flexible) ratio
    r_{l+1}^T (z_{l+1} - z_l) / rho_l, which equals it in exact arithmetic.  ``storage`` (None or
    a numpy dtype such as float32) rounds the vectors x, r, z, p to that type after every update:
    another valid floating-point execution of the same algorithm, used to measure how far such
    executions spread; the arithmetic itself stays float64.  ``precond_rounding`` (None or
    (rel, seed)) multiplies each preconditioner output by 1 + rel * N(0, 1) elementwise (seeded):
    a model of the preconditioner evaluated at finite precision, for the same purpose.
    Returns (x, iterations, final relative residual, status); status -5 flags a breakdown."""
    if precond_rounding is not None:
        rel_pc, seed_pc = precond_rounding
        rng_pc = np.random.default_rng(seed_pc)

    def precond(rr):
        z = precond_apply(rr, dv, dh, tau, basis_N, basis_M)
        if precond_rounding is None:
            return z
        return tuple(zi * (1.0 + rel_pc * rng_pc.standard_normal(zi.shape)) for zi in z)

    x = _stored(tuple(np.array(a, dtype=np.float64) for a in x0), storage)
    bnorm = math.sqrt(_dot(b, b))
    r = tuple(bi - qi for bi, qi in zip(b, apply_A(x, dv, dh, tau)))
    rel = math.sqrt(_dot(r, r)) / bnorm if bnorm > 0 else 0.0
    if bnorm == 0.0 or rel <= tol or cg_max <= 0:
        return x, 0, rel, 0
    r = _stored(r, storage)
    z = _stored(precond(r), storage)
    p = z
    rho = _dot(r, z)
    it = 0
    while True:
        q = apply_A(p, dv, dh, tau)
        pq = _dot(p, q)
        if not (pq > 0.0 and rho > 0.0):
            return x, it, rel, -5
        alpha = rho / pq
        x = _stored(_axpy(alpha, p, x), storage)
        r = _stored(_axpy(-alpha, q, r), storage)
        it += 1
        rel = math.sqrt(_dot(r, r)) / bnorm
        if rel <= tol or it >= cg_max:
            return x, it, rel, 0
        z_new = _stored(precond(r), storage)
        rho_new = _dot(r, z_new)
        if beta_rule == "pr":
            beta = (rho_new - _dot(r, z)) / rho
        else:
            beta = rho_new / rho
        rho = rho_new
        z = z_new
        p = _stored(tuple(zi + beta * pi for zi, pi in zip(z_new, p)), storage)


# --------------------------------------------------------------------------------------------
# U-only (Schur complement) form of the same linear system
# --------------------------------------------------------------------------------------------
# The V rows of the system of Sec. 3.1 give (D + 1/tau) V = (D U - G) / tau edge by edge, i.e.
# V = (D U - G) / (1 + tau D).  Substituted into the U row:  S^T Om_v (S U - Gv) +
# (U T - Gh) Om_h T^T = 0  with  Om = D / (1 + tau D)  per edge.
def schur_weights(dv, dh, tau):
    """Om = D / (1 + tau D) on the vertical and horizontal edges."""
    return dv / (1.0 + tau * dv), dh / (1.0 + tau * dh)


def schur_matvec(U, Ov, Oh):
    """L_Om U = S^T (Om_v o S U) + (Om_h o U T) T^T."""
    N, M = U.shape
    return St_op(Ov * S_op(U), N) + Tt_op(Oh * T_op(U), M)


def schur_rhs(Gv, Gh, Ov, Oh, N, M):
    """f = S^T (Om_v o Gv) + (Om_h o Gh) T^T."""
    return St_op(Ov * Gv, N) + Tt_op(Oh * Gh, M)


def schur_recover_v(U, Gv, Gh, dv, dh, tau):
    """V = (D U - G) / (1 + tau D), the V rows solved for the given U."""
    return (S_op(U) - Gv) / (1.0 + tau * dv), (T_op(U) - Gh) / (1.0 + tau * dh)


def pcg_schur(U0, f, Ov, Oh, tau, basis_N, basis_M, tol, cg_max, beta_rule="fr", storage=None):
    """Alg. 2 on L_Om U = f from the warm start U0, preconditioned by the Laplacian block of
    Sec. 3.3 (z = P_S [(P_S^T tau r P_T) / (lam_i + mu_j)] P_T^T, zero frequency dropped; Om <=
    1/tau, so (1/tau) times the Laplacian is its upper bound).  Stops when ||r|| / ||f|| <= tol
    or after cg_max products with L_Om.  storage as in pcg.
    Returns (U, iterations, relative residual, status)."""
    N, M = f.shape
    zeros_v, zeros_h = np.zeros((N - 1, M)), np.zeros((N, M - 1))

    def prec(r):
        return precond_apply((r, zeros_v, zeros_h), zeros_v, zeros_h, tau, basis_N, basis_M)[0]

    def keep(a):
        return a if storage is None else np.asarray(a, dtype=storage).astype(np.float64)

    U = keep(np.array(U0, dtype=np.float64))
    fnorm = float(np.linalg.norm(f))
    r = f - schur_matvec(U, Ov, Oh)
    rel = float(np.linalg.norm(r)) / fnorm if fnorm > 0 else 0.0
    if fnorm == 0.0 or rel <= tol or cg_max <= 0:
        return U, 0, rel, 0
    r = keep(r)
    z = keep(prec(r))
    p = z
    rho = float(np.vdot(r, z))
    it = 0
    while True:
        q = schur_matvec(p, Ov, Oh)
        pq = float(np.vdot(p, q))
        if not (pq > 0.0 and rho > 0.0):
            return U, it, rel, -5
        alpha = rho / pq
        U = keep(U + alpha * p)
        r = keep(r - alpha * q)
        it += 1
        rel = float(np.linalg.norm(r)) / fnorm
        if rel <= tol or it >= cg_max:
            return U, it, rel, 0
        z_new = keep(prec(r))
        rho_new = float(np.vdot(r, z_new))
        beta = (rho_new - float(np.vdot(r, z))) / rho if beta_rule == "pr" else rho_new / rho
        rho, z = rho_new, z_new
        p = keep(z_new + beta * p)


# --------------------------------------------------------------------------------------------
# Objectives: problem (main), F (soft constraints), F_delta, H_delta (problem alt1)
# --------------------------------------------------------------------------------------------
def l1_objective(U, Gv, Gh, Cv, Ch):
    """sum Cv |U_{i+1,j} - U_{ij} - Gv| + sum Ch |U_{i,j+1} - U_{ij} - Gh| (problem (main), Sec. 2)."""
    return float(np.sum(Cv * np.abs(S_op(U) - Gv)) + np.sum(Ch * np.abs(T_op(U) - Gh)))


def _penalty(U, Vv, Vh, Gv, Gh, tau):
    return (float(np.sum((S_op(U) - Gv - Vv) ** 2)) + float(np.sum((T_op(U) - Gh - Vh) ** 2))) / (2 * tau)


def F_value(U, Vv, Vh, Gv, Gh, Cv, Ch, tau):
    """F of problem (soft constraints), Sec. 3.1."""
    return float(np.sum(Cv * np.abs(Vv)) + np.sum(Ch * np.abs(Vh))) + _penalty(U, Vv, Vh, Gv, Gh, tau)


def F_delta_value(U, Vv, Vh, Gv, Gh, Cv, Ch, tau, delta):
    """F_delta, Sec. 3.1 (the delta-smoothed F)."""
    s = float(np.sum(np.sqrt(Cv * Cv * Vv * Vv + delta * delta))
              + np.sum(np.sqrt(Ch * Ch * Vh * Vh + delta * delta)))
    return s + _penalty(U, Vv, Vh, Gv, Gh, tau)


def H_delta_value(U, Vv, Vh, Wv, Wh, Gv, Gh, Cv, Ch, tau, delta):
    """Objective of problem (alt1), Sec. 3.1: 1/2 sum [(C^2 V^2 + delta^2) / W + W] + penalties."""
    s = 0.5 * float(np.sum((Cv * Cv * Vv * Vv + delta * delta) / Wv + Wv)
                    + np.sum((Ch * Ch * Vh * Vh + delta * delta) / Wh + Wh))
    return s + _penalty(U, Vv, Vh, Gv, Gh, tau)


def smoothness_L(Cv, Ch, tau, delta):
    """L = 12 / tau + C_max^2 / delta (Theorem on the sublinear rate, Sec. 3.1)."""
    cmax = max(float(np.max(Cv, initial=0.0)), float(np.max(Ch, initial=0.0)))
    return 12.0 / tau + cmax * cmax / delta


def gradient_candidate(U, Vv, Vh, Wv, Wh, Gv, Gh, Cv, Ch, tau, delta):
    """One gradient step of length 1/L on (U, Vv, Vh) at fixed W: the candidate of the
    sufficient-decrease condition (Theorem on the sublinear rate, Sec. 3.1)."""
    N, M = U.shape
    L = smoothness_L(Cv, Ch, tau, delta)
    Ev = S_op(U) - Gv - Vv
    Eh = T_op(U) - Gh - Vh
    Ut = U - (St_op(Ev, N) + Tt_op(Eh, M)) / (tau * L)
    Vvt = Vv - (Cv * Cv / Wv * Vv + (Vv - S_op(U) + Gv) / tau) / L
    Vht = Vh - (Ch * Ch / Wh * Vh + (Vh - T_op(U) + Gh) / tau) / L
    return Ut, Vvt, Vht


# --------------------------------------------------------------------------------------------
# Alg. 1: IRLS
# --------------------------------------------------------------------------------------------
class Problem:
    """Inputs of Alg. 1 for one image: G, C, b and the two DCT bases."""

    def __init__(self, X, coherence=None, Cv=None, Ch=None, tau=1e-2):
        X = np.asarray(X, dtype=np.float32)
        self.N, self.M = X.shape
        self.tau = float(tau)
        self.Gv, self.Gh = wrapped_gradients(X)
        if Cv is None or Ch is None:
            Cv, Ch = edge_weights(coherence, self.N, self.M)
        self.Cv = np.asarray(Cv, dtype=np.float64)
        self.Ch = np.asarray(Ch, dtype=np.float64)
        self.b = rhs_b(self.Gv, self.Gh, self.tau)
        self.basis_N = dct_basis(self.N)
        self.basis_M = self.basis_N if self.M == self.N else dct_basis(self.M)


def paper_cg_cap(delta_rel, m_prev, raised_prev, eps_tol, alpha):
    """One step of the CG-budget rule of Sec. 4.3, taken at IRLS iteration k >= 1 once the
    weights W^k are known.  delta_rel = Delta_{k-1,k}, the relative drop of H_delta at x^k when
    the weights go from W^{k-1} to W^k; m_prev = m_CG(k-1); raised_prev tells whether
    m_CG(k-1) != m_CG(k-2).  Returns (m_CG(k), raised) or (None, raised_prev) for "stop and
    return U^k":
      Delta > eps_tol                    -> keep the budget;
      Delta <= eps_tol, raised last time -> stop;
      Delta <= eps_tol, not raised       -> budget times alpha.
    Readings: m_CG(-1) = m_CG(0) (nothing was raised before k = 1), and the scaled budget is
    rounded down to an integer number of iterations."""
    if delta_rel > eps_tol:
        return m_prev, False
    if raised_prev:
        return None, raised_prev
    return int(np.floor(alpha * m_prev)), True


def irls_unwrap(X, coherence=None, *, Cv=None, Ch=None, tau=1e-2, delta=1e-3, outer_iters=10,
                cg_tol=1e-5, cg_max=1000, beta_rule="fr", x0=None, record=False, storage=None,
                cg_schedule="fixed", m0=5, eps_tol=1e-3, alpha=1.7, precond_rounding=None,
                system="full", cg_caps=None):
    """Alg. 1 with Alg. 2 as the inner solver.

    cg_schedule "fixed": outer_iters IRLS iterations, every inner solve capped at cg_max.
    cg_schedule "paper": the CG budget m_CG(k) and the IRLS stop of Sec. 4.3 (paper_cg_cap,
    m_CG(0) = m0), at most outer_iters iterations, each solve capped at min(m_CG(k), cg_max).

    Returns a dict with U (zero mean), Vv, Vh, and per-outer statistics: cg_iters, rel_res,
    l1_obj (problem (main) at U^{k+1}), h_delta (H_delta(x^{k+1}, W^k)), h_before
    (H_delta(x^k, W^k)), h_after_rw (H_delta(x^{k+1}, W^{k+1})), f_delta, cg_cap (the cap of
    each solve), delta_rel (Delta_{k-1,k} for k >= 1, "paper" only), schedule_stop and h_stop
    (H_delta(x^k, W^k) at the iteration where the rule stopped the run), status.
    With ``record`` the per-outer weights W^k and iterates are kept too (used by the adjoint).
    ``storage`` and ``precond_rounding`` are passed to pcg (other valid floating-point
    executions; the latter's seed advances with the outer iteration).  ``cg_caps`` (a list)
    caps solve k at cg_caps[k] (with cg_tol = 0: exactly that many iterations), to replay another
    execution's stopping decisions.
    system "full": Alg. 2 on the (U, Vv, Vh) system of Sec. 3.1 with the block-diagonal
    preconditioner (the paper's method).  system "schur": Alg. 2 on the U-only system obtained
    by eliminating V (pcg_schur), then V = (D U - G) / (1 + tau D); the same outer loop, stopping
    rule on the U-only residual (with precond_rounding unsupported)."""
    if system not in ("full", "schur"):
        raise ValueError("system is 'full' or 'schur'")
    if cg_schedule not in ("fixed", "paper"):
        raise ValueError("cg_schedule is 'fixed' or 'paper'")
    pb = Problem(X, coherence, Cv, Ch, tau)
    N, M = pb.N, pb.M
    if x0 is None:
        U = np.zeros((N, M))
        Vv = S_op(U) - pb.Gv          # V^0 = S U^0 - Gv
        Vh = T_op(U) - pb.Gh
    else:
        U, Vv, Vh = (np.array(a, dtype=np.float64) for a in x0)
    st = {k: [] for k in ("cg_iters", "rel_res", "l1_obj", "h_delta", "h_before", "h_after_rw",
                          "f_delta", "cg_cap", "delta_rel")}
    rec = {"W": [], "x": []}
    status = 0
    m_cg, raised, stop, h_stop = m0, False, False, None
    for k in range(outer_iters):
        Wv, Wh = reweight(Vv, Vh, pb.Cv, pb.Ch, delta)
        dv, dh = diag_d(pb.Cv, pb.Ch, Wv, Wh)
        h_before = H_delta_value(U, Vv, Vh, Wv, Wh, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta)
        cap = cg_max if cg_caps is None else cg_caps[k]
        if cg_schedule == "paper":
            if k >= 1:
                # Delta_{k-1,k} = (H(x^k, W^{k-1}) - H(x^k, W^k)) / H(x^k, W^{k-1})
                d = (st["h_delta"][-1] - h_before) / st["h_delta"][-1]
                st["delta_rel"].append(d)
                m_next, raised = paper_cg_cap(d, m_cg, raised, eps_tol, alpha)
                if m_next is None:
                    stop = True
                    h_stop = h_before
                    break
                m_cg = m_next
            cap = min(m_cg, cg_max)
        if record:
            rec["W"].append((Wv, Wh))
            rec["x"].append((U.copy(), Vv.copy(), Vh.copy()))
        st["h_before"].append(h_before)
        st["cg_cap"].append(cap)
        if system == "schur":
            Ov, Oh = schur_weights(dv, dh, tau)
            f = schur_rhs(pb.Gv, pb.Gh, Ov, Oh, N, M)
            U, it, rel, s = pcg_schur(U, f, Ov, Oh, tau, pb.basis_N, pb.basis_M, cg_tol, cap,
                                      beta_rule, storage)
            Vv, Vh = schur_recover_v(U, pb.Gv, pb.Gh, dv, dh, tau)
        else:
            pr = None if precond_rounding is None else (precond_rounding[0],
                                                        precond_rounding[1] + 7919 * k)
            (U, Vv, Vh), it, rel, s = pcg((U, Vv, Vh), pb.b, dv, dh, tau, pb.basis_N, pb.basis_M,
                                          cg_tol, cap, beta_rule, storage, pr)
        if s < 0:
            status = s
        elif it >= cap and cap >= cg_max and rel > cg_tol and status == 0:
            # the hard cap ended a solve short of cg_tol (a planned budget of Sec. 4.3 does not)
            status = 1
        U = U - U.mean()
        st["cg_iters"].append(it)
        st["rel_res"].append(rel)
        st["h_delta"].append(H_delta_value(U, Vv, Vh, Wv, Wh, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta))
        Wv2, Wh2 = reweight(Vv, Vh, pb.Cv, pb.Ch, delta)
        st["h_after_rw"].append(H_delta_value(U, Vv, Vh, Wv2, Wh2, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta))
        st["l1_obj"].append(l1_objective(U, pb.Gv, pb.Gh, pb.Cv, pb.Ch))
        st["f_delta"].append(F_delta_value(U, Vv, Vh, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta))
        if s < 0:
            break
    out = {"U": U, "Vv": Vv, "Vh": Vh, "status": status, "problem": pb, "schedule_stop": stop,
           "h_stop": h_stop, **st}
    if record:
        rec["x"].append((U.copy(), Vv.copy(), Vh.copy()))
        out["record"] = rec
    return out


# --------------------------------------------------------------------------------------------
# Sec. 4.5: evaluation helpers
# --------------------------------------------------------------------------------------------
def best_shift_error(U, Xu):
    """E(U, Xu) = Xu - (U + alpha), alpha = mean(Xu - U) (Sec. 4.5)."""
    alpha = float(np.mean(Xu - U))
    return Xu - (U + alpha)


def round_congruent(U, X, c=None):
    """'Rounded IRLS' (Sec. 4.5): the output moved to the nearest image that is 2pi-congruent to
    the input.  The global offset of U is free (the model is shift invariant), so U is first
    aligned with X by the circular mean c = arg sum exp(i (U - X)) (float64); then
    K = rint((U - c - X) / 2pi) and U_round = X + 2pi K.  The integer K is decided in float32,
    one correctly rounded operation at a time (the precision of the library's kernel):
    t = (U - c) - X, q = t / 2pi, K = rint(q), U_round = X + (2pi * K).  Returns
    (U_round float32, K int64, c)."""
    U32 = np.asarray(U, dtype=np.float32)
    X32 = np.asarray(X, dtype=np.float32)
    if c is None:
        d = U32.astype(np.float64) - X32.astype(np.float64)
        c = float(math.atan2(np.sum(np.sin(d)), np.sum(np.cos(d))))
    c32 = np.float32(c)
    t = ((U32 - c32).astype(np.float32) - X32).astype(np.float32)
    q = (t / TWO_PI_F32).astype(np.float32)
    K = np.rint(q).astype(np.float32)
    Ur = (X32 + (TWO_PI_F32 * K).astype(np.float32)).astype(np.float32)
    return Ur, K.astype(np.int64), c


def k_map(U, X):
    """Integer ambiguity map of an unwrapped estimate: the global offset c is the circular mean
    of U - X, then K = round((U - c - X) / 2pi).  The paper's 'rounded IRLS' (Sec. 4.5) is
    X + 2pi K + c."""
    X = np.asarray(X, dtype=np.float64)
    c = float(np.angle(np.sum(np.exp(1j * (U - X)))))
    return np.rint((U - c - X) / (2.0 * np.pi)).astype(np.int64)


# --------------------------------------------------------------------------------------------
# Appendix A: explicit Kronecker matrices (tiny grids only)
# --------------------------------------------------------------------------------------------
def dense_operators(N, M):
    """Explicit S_N ((N-1) x N) and T_M (M x (M-1)) from their element definitions (Sec. 2),
    and B = [[I_M (x) S_N, -I, 0], [T_M^T (x) I_N, 0, -I]] (proof of Theorem 'existence').
    Vectorisation is column-major (vec stacks the columns), as in the paper's notation."""
    S = np.zeros((N - 1, N))
    for i in range(N - 1):
        for j in range(N):
            if j == i + 1:
                S[i, j] = 1.0
            elif j == i:
                S[i, j] = -1.0
    T = np.zeros((M, M - 1))
    for i in range(M):
        for j in range(M - 1):
            if i == j + 1:
                T[i, j] = 1.0
            elif i == j:
                T[i, j] = -1.0
    nv, nh = (N - 1) * M, N * (M - 1)
    B = np.zeros((nv + nh, N * M + nv + nh))
    B[:nv, :N * M] = np.kron(np.eye(M), S)
    B[nv:, :N * M] = np.kron(T.T, np.eye(N))
    B[:nv, N * M:N * M + nv] = -np.eye(nv)
    B[nv:, N * M + nv:] = -np.eye(nh)
    return S, T, B


# --------------------------------------------------------------------------------------------
# Adjoint of the IRLS map (X, coherence) -> U, through converged inner solves
# --------------------------------------------------------------------------------------------
def irls_adjoint(X, coherence, dL_dU, *, tau=1e-2, delta=1e-3, outer_iters=10, cg_tol=1e-10,
                 cg_max=5000, adj_tol=None, fwd=None, storage=None):
    """Reverse-mode derivative of L(U(X, coherence)) given dL/dU.

    Model: every outer step of Alg. 1 is taken as its exact solve, x^{k+1} = A_k^+ b with
    A_k = A(D^k), D^k = C^2 / W^k, W^k = sqrt(C^2 (V^k)^2 + delta^2) (Sec. 3.1-3.2), and U zero-mean.
    Then x^{k+1} depends on the previous iterate only through V^k, and for a cotangent xbar of
    x^{k+1}:
        lambda = A_k^+ xbar                       (one solve with the same symmetric operator)
        bbar  += lambda                           (b is linear in G)
        Dbar   = -lambda_V o V^{k+1}              (A depends on D only through diag(0, D))
        Vbar^k = Dbar o dD/dV = Dbar o (-C^4 V^k / W^3)
        Cbar  += Dbar o dD/dC = Dbar o (2 C / W - C^3 (V^k)^2 / W^3)
    and xbar for the previous step is (0, Vbar^k).  Finally V^0 = -G adds -Vbar^0 to Gbar,
    b = ((S^T Gv + Gh T^T)/tau, -Gv/tau, -Gh/tau) gives Gbar_v += (S lambda_U - lambda_Vv)/tau and
    Gbar_h += (lambda_U T - lambda_Vh)/tau, the wrap has derivative 1 almost everywhere so
    Xbar = S^T Gbar_v + Gbar_h T^T, and Cv = (coh_i + coh_i+1)/2 spreads Cbar back to coherence.
    ``storage`` is passed to the forward and adjoint PCG runs (see pcg).
    Returns (dL/dX, dL/dcoherence or None, forward result)."""
    if fwd is None:
        fwd = irls_unwrap(X, coherence, tau=tau, delta=delta, outer_iters=outer_iters,
                          cg_tol=cg_tol, cg_max=cg_max, record=True, storage=storage)
    pb = fwd["problem"]
    N, M = pb.N, pb.M
    xs = fwd["record"]["x"]             # x^0 .. x^K (V parts are the checkpoints)
    K = len(xs) - 1
    adj_tol = cg_tol if adj_tol is None else adj_tol
    Cv, Ch = pb.Cv, pb.Ch
    ubar = np.asarray(dL_dU, dtype=np.float64)
    xbar = (ubar - ubar.mean(), np.zeros((N - 1, M)), np.zeros((N, M - 1)))
    Gbv, Gbh = np.zeros((N - 1, M)), np.zeros((N, M - 1))
    Cbv, Cbh = np.zeros((N - 1, M)), np.zeros((N, M - 1))
    zero = (np.zeros((N, M)), np.zeros((N - 1, M)), np.zeros((N, M - 1)))
    for k in range(K - 1, -1, -1):
        _, Vv_k, Vh_k = xs[k]
        _, Vv_n, Vh_n = xs[k + 1]
        Wv, Wh = reweight(Vv_k, Vh_k, Cv, Ch, delta)
        dv, dh = diag_d(Cv, Ch, Wv, Wh)
        lam, _, _, _ = pcg(zero, xbar, dv, dh, tau, pb.basis_N, pb.basis_M, adj_tol, cg_max,
                           storage=storage)
        lu, lv, lh = lam
        Gbv += (S_op(lu) - lv) / tau
        Gbh += (T_op(lu) - lh) / tau
        Dbv, Dbh = -lv * Vv_n, -lh * Vh_n
        Vbv = Dbv * dD_dV(Cv, Vv_k, Wv)
        Vbh = Dbh * dD_dV(Ch, Vh_k, Wh)
        Cbv += Dbv * dD_dC(Cv, Vv_k, Wv)
        Cbh += Dbh * dD_dC(Ch, Vh_k, Wh)
        xbar = (np.zeros((N, M)), Vbv, Vbh)
    # V^0 = -G
    Gbv -= xbar[1]
    Gbh -= xbar[2]
    Xbar = St_op(Gbv, N) + Tt_op(Gbh, M)
    cbar = None
    if coherence is not None:
        cbar = np.zeros((N, M))
        cbar[:-1, :] += 0.5 * Cbv
        cbar[1:, :] += 0.5 * Cbv
        cbar[:, :-1] += 0.5 * Cbh
        cbar[:, 1:] += 0.5 * Cbh
    return Xbar, cbar, fwd



# --------------------------------------------------------------------------------------------
# Tiled unwrapping of a large image (the paper's future-work remark on very large images,
# Sec. 5, with the 4000 x M images of Sec. 4.5): overlapping tiles solved independently by
# Alg. 1, then each tile's free constant fixed by agreement on the overlaps.  The paper gives
# no procedure; the readings are:
#   * tile starts along a side of n pixels with tile t and overlap o: 0, t - o, 2 (t - o), ...
#     while the tile ends before n, then a last tile ending flush at n (every tile is t long;
#     one tile of n when n <= t);
#   * the offset between tiles s and t that are neighbours in the tile grid (same row of tiles,
#     next column, or same column, next row) is the mean of U_t - U_s over their overlap,
#     taken again over the pixels within pi of that first mean (pixels where the two tiles
#     unwrapped a different number of cycles do not pull it);
#   * constants c minimising sum over neighbour pairs of n_st (c_s - c_t - d_ts)^2 with
#     d_ts = offset(U_t - U_s) and c_0 = 0 (weights n_st: the pixels the second mean used);
#   * each pixel is taken from the tile whose core holds it: consecutive tiles split their
#     overlap at (start of the next + end of this) // 2; the stitched image is made zero-mean.
# --------------------------------------------------------------------------------------------
def tile_starts(n, t, o):
    """Starts of the tiles along a side of n pixels (tile t, overlap o, 0 <= o < t)."""
    if n <= t:
        return [0]
    s, out = t - o, []
    a = 0
    while a + t < n:
        out.append(a)
        a += s
    out.append(n - t)
    return out


def tile_cores(starts, t, n):
    """[lo, hi) of each tile's core along one side: consecutive tiles split their overlap at
    (start of the next + end of this) // 2."""
    t = min(t, n)
    bounds = [0] + [(starts[a + 1] + starts[a] + t) // 2 for a in range(len(starts) - 1)] + [n]
    return [(bounds[a], bounds[a + 1]) for a in range(len(starts))]


def overlap_offset(Ut, Us):
    """Robust mean of Ut - Us over an overlap (both arrays of the overlap's shape): the mean,
    then the mean again over the pixels within pi of it.  Returns (offset, pixel count)."""
    d = (Ut - Us).ravel()
    m0 = float(d.mean())
    keep = np.abs(d - m0) < np.pi
    if not keep.any():
        return m0, d.size
    return float(d[keep].mean()), int(keep.sum())


def stitch_tiles(sol, rs, cs, th, tw, H, W):
    """Fixes the constants of tile solutions sol[t] (tile t = a * len(cs) + b at rows
    rs[a]:rs[a]+th, columns cs[b]:cs[b]+tw) by least squares on the neighbour offsets and
    stitches the cores into a zero-mean H x W image.  Returns (U, constants, pairs)."""
    nc = len(cs)
    pairs = []
    for a in range(len(rs)):
        for b in range(nc):
            t = a * nc + b
            for (a2, b2) in ((a, b + 1), (a + 1, b)):
                if a2 >= len(rs) or b2 >= nc:
                    continue
                s = a2 * nc + b2
                r0, c0 = max(rs[a], rs[a2]), max(cs[b], cs[b2])
                r1, c1 = min(rs[a], rs[a2]) + th, min(cs[b], cs[b2]) + tw
                if r1 <= r0 or c1 <= c0:
                    continue
                Ut = sol[t][r0 - rs[a]:r1 - rs[a], c0 - cs[b]:c1 - cs[b]]
                Us = sol[s][r0 - rs[a2]:r1 - rs[a2], c0 - cs[b2]:c1 - cs[b2]]
                d, n = overlap_offset(Ut, Us)
                pairs.append((t, s, d, n))
    T = len(rs) * nc
    c = np.zeros(T)
    if T > 1:
        # normal equations of sum n (c_s - c_t - d)^2 with c_0 fixed at 0
        A = np.zeros((T, T))
        rhs = np.zeros(T)
        for t, s, d, n in pairs:
            A[t, t] += n
            A[s, s] += n
            A[t, s] -= n
            A[s, t] -= n
            rhs[s] += n * d
            rhs[t] -= n * d
        c[1:] = np.linalg.solve(A[1:, 1:], rhs[1:])
    U = np.zeros((H, W))
    rc, cc = tile_cores(rs, th, H), tile_cores(cs, tw, W)
    for a, (lo_r, hi_r) in enumerate(rc):
        for b, (lo_c, hi_c) in enumerate(cc):
            t = a * nc + b
            U[lo_r:hi_r, lo_c:hi_c] = (sol[t][lo_r - rs[a]:hi_r - rs[a], lo_c - cs[b]:hi_c - cs[b]]
                                       + c[t])
    U -= U.mean()
    return U, c, pairs


def irls_unwrap_tiled(X, coherence=None, *, tile=256, overlap=32, **kw):
    """Unwraps X tile by tile (Alg. 1 on each overlapping tile, keyword arguments as in
    irls_unwrap), fixes the tiles' constants by least squares on the neighbour offsets and
    stitches the cores.  Returns a dict with U (zero mean), the tiles' solutions and constants."""
    X = np.asarray(X, dtype=np.float32)
    H, W = X.shape
    rs, cs = tile_starts(H, tile, overlap), tile_starts(W, tile, overlap)
    th, tw = min(tile, H), min(tile, W)
    tiles = [(r, c) for r in rs for c in cs]
    sol = []
    for r, c in tiles:
        co = None if coherence is None else np.asarray(coherence)[r:r + th, c:c + tw]
        out = irls_unwrap(X[r:r + th, c:c + tw], co, **kw)
        sol.append(out["U"])
    U, c, pairs = stitch_tiles(sol, rs, cs, th, tw, H, W)
    return {"U": U, "tiles": tiles, "tile_U": sol, "constants": c, "pairs": pairs,
            "row_starts": rs, "col_starts": cs}
