"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Every check here compares the oracle with something other than itself: explicit Kronecker
matrices built from the element definitions (Sec. 2, Appendix A), the gradient of the objective
of problem (alt1) by central differences, the closed-form DCT eigenpairs against a library
eigensolver, a dense pseudo-inverse, a least-squares solve, an LP solve of problem (main), a
damped-Newton minimiser of F_delta, the paper's printed Gershgorin figures, and the theorems of
Sec. 3.1 used as invariants.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import irls as O
import synthetic

HERE = os.path.dirname(os.path.abspath(__file__))


def vecF(a):
    """Column-major vectorisation, the paper's vec (Sec. 1, notation)."""
    return np.asarray(a).flatten(order="F")


def pack(x):
    return np.concatenate([vecF(a) for a in x])


def unpack(v, N, M):
    nu, nv = N * M, (N - 1) * M
    return (v[:nu].reshape((N, M), order="F"), v[nu:nu + nv].reshape((N - 1, M), order="F"),
            v[nu + nv:].reshape((N, M - 1), order="F"))


def dense_A(N, M, dv, dh, tau):
    """A of eq. (matrix-soft-constraints), written block by block from the Kronecker forms."""
    S, T, _ = O.dense_operators(N, M)
    IN, IM = np.eye(N), np.eye(M)
    nu, nv, nh = N * M, (N - 1) * M, N * (M - 1)
    A = np.zeros((nu + nv + nh, nu + nv + nh))
    A[:nu, :nu] = (np.kron(IM, S.T @ S) + np.kron(T @ T.T, IN)) / tau
    A[:nu, nu:nu + nv] = -np.kron(IM, S.T) / tau
    A[:nu, nu + nv:] = -np.kron(T, IN) / tau
    A[nu:nu + nv, :nu] = -np.kron(IM, S) / tau
    A[nu:nu + nv, nu:nu + nv] = np.diag(vecF(dv)) + np.eye(nv) / tau
    A[nu + nv:, :nu] = -np.kron(T.T, IN) / tau
    A[nu + nv:, nu + nv:] = np.diag(vecF(dh)) + np.eye(nh) / tau
    return A


def rand_state(N, M, rng):
    U = rng.standard_normal((N, M))
    Vv = rng.standard_normal((N - 1, M))
    Vh = rng.standard_normal((N, M - 1))
    return U, Vv, Vh


def rand_problem(N, M, rng, tau=1e-2):
    X = rng.uniform(-np.pi, np.pi, size=(N, M)).astype(np.float32)
    coh = rng.uniform(0.05, 1.0, size=(N, M)).astype(np.float32)
    return O.Problem(X, coh, tau=tau)


# ------------------------------------------------------------------------------------------
# Sec. 2: wrap
# ------------------------------------------------------------------------------------------
def test_wrap_special_values():
    two_pi = np.float32(2 * np.pi)
    t = np.array([0.0, 3.0, -3.0, 4.0, -4.0, 7.0, 10.0], dtype=np.float32)
    w = O.wrap_f32(t)
    assert w[0] == 0.0 and w[1] == np.float32(3.0) and w[2] == np.float32(-3.0)
    np.testing.assert_allclose(w[3], np.float32(4.0) - two_pi, rtol=0, atol=1e-6)
    np.testing.assert_allclose(w[4], np.float32(-4.0) + two_pi, rtol=0, atol=1e-6)
    np.testing.assert_allclose(w[5], np.float32(7.0) - two_pi, rtol=0, atol=1e-6)
    np.testing.assert_allclose(w[6], np.float32(10.0) - 2 * two_pi, rtol=0, atol=2e-6)
    # the half-open convention: +pi maps to -pi
    assert O.wrap_f32(np.float32(np.pi)) < 0


def test_wrap_range_and_congruence():
    rng = np.random.default_rng(1)
    t = rng.uniform(-2 * np.pi, 2 * np.pi, size=100000).astype(np.float32)
    w = O.wrap_f32(t).astype(np.float64)
    assert np.all(w >= -np.pi - 1e-6) and np.all(w < np.pi + 1e-6)
    k = (t.astype(np.float64) - w) / (2 * np.pi)
    np.testing.assert_allclose(k, np.rint(k), atol=1e-5)
    # differences that already lie well inside (-pi, pi) are returned unchanged
    s = rng.uniform(-3.0, 3.0, size=1000).astype(np.float32)
    assert np.array_equal(O.wrap_f32(s), s)


def test_wrapped_gradients_of_wrapped_smooth_phase_are_true_gradients():
    # Itoh's condition: |true difference| < pi  =>  wrapped difference == true difference
    X, phi = synthetic.smooth_phase(20, 17, seed=3, max_step=2.0)
    Gv, Gh = O.wrapped_gradients(X)
    np.testing.assert_allclose(Gv, np.diff(phi, axis=0), atol=2e-5)
    np.testing.assert_allclose(Gh, np.diff(phi, axis=1), atol=2e-5)


# ------------------------------------------------------------------------------------------
# Sec. 3.2: the matrix A, the right-hand side b, and the gradient of H_delta
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N,M", [(2, 2), (3, 5), (5, 4), (1, 6), (6, 1)])
def test_matvec_equals_kronecker_matrix(N, M):
    rng = np.random.default_rng(N * 10 + M)
    tau = 0.3
    dv = rng.uniform(0.1, 5.0, size=(N - 1, M))
    dh = rng.uniform(0.1, 5.0, size=(N, M - 1))
    A = dense_A(N, M, dv, dh, tau)
    x = rand_state(N, M, rng)
    q = O.apply_A(x, dv, dh, tau)
    np.testing.assert_allclose(pack(q), A @ pack(x), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N,M", [(3, 4), (4, 4)])
def test_A_equals_hessian_of_penalty_plus_D(N, M):
    # proof of the rate theorem: the Hessian of s is (1/tau) B^T B; A adds diag(0, Dv, Dh)
    rng = np.random.default_rng(5)
    tau = 0.7
    dv = rng.uniform(0.1, 2.0, size=(N - 1, M))
    dh = rng.uniform(0.1, 2.0, size=(N, M - 1))
    _, _, B = O.dense_operators(N, M)
    Ad = B.T @ B / tau
    Ad[N * M:, N * M:] += np.diag(np.concatenate([vecF(dv), vecF(dh)]))
    np.testing.assert_allclose(dense_A(N, M, dv, dh, tau), Ad, atol=1e-12)


def test_gershgorin_figures_printed_in_the_paper():
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))["gershgorin"]
    N, M, tau = 5, 6, 0.25
    _, _, B = O.dense_operators(N, M)
    H = B.T @ B / tau
    diag = np.diag(H)
    off = np.abs(H).sum(axis=1) - np.abs(diag)
    assert math.isclose(diag.max() * tau, g["max_diagonal_times_tau"], rel_tol=1e-12)
    assert math.isclose(off.max() * tau, g["max_offdiagonal_row_sum_times_tau"], rel_tol=1e-12)
    row = N + 2 - 1   # 'line N+2' of the paper, 1-based
    assert math.isclose(diag[row] * tau, 4.0) and math.isclose(off[row] * tau, 8.0)
    assert np.linalg.eigvalsh(H).max() * tau <= g["L_s_bound_times_tau"] + 1e-12


@pytest.mark.parametrize("N,M", [(3, 4), (4, 2)])
def test_residual_is_gradient_of_H_delta(N, M):
    """A x - b = grad_x H_delta(x, W) at fixed W (Prop. 'linear system' is the stationarity
    condition of problem (alt1)); checked by central differences of H_delta itself."""
    rng = np.random.default_rng(7)
    tau, delta = 0.2, 0.05
    pb = rand_problem(N, M, rng, tau)
    x = rand_state(N, M, rng)
    Wv = rng.uniform(0.1, 1.0, size=(N - 1, M))
    Wh = rng.uniform(0.1, 1.0, size=(N, M - 1))
    dv, dh = O.diag_d(pb.Cv, pb.Ch, Wv, Wh)
    res = pack(O.apply_A(x, dv, dh, tau)) - pack(pb.b)

    def H(v):
        U, Vv, Vh = unpack(v, N, M)
        return O.H_delta_value(U, Vv, Vh, Wv, Wh, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta)

    v0 = pack(x)
    h = 1e-5
    grad = np.array([(H(v0 + h * e) - H(v0 - h * e)) / (2 * h) for e in np.eye(v0.size)])
    np.testing.assert_allclose(res, grad, rtol=1e-6, atol=1e-6)


def test_b_in_range_of_A():
    rng = np.random.default_rng(2)
    pb = rand_problem(9, 7, rng)
    assert abs(pb.b[0].sum()) < 1e-9 * np.abs(pb.b[0]).sum()


# ------------------------------------------------------------------------------------------
# Sec. 3.3: the preconditioner
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 8, 13])
def test_dct_basis_diagonalises_neumann_laplacian(N):
    P, lam = O.dct_basis(N)
    S, _, _ = O.dense_operators(N, 2)
    L = S.T @ S
    np.testing.assert_allclose(P.T @ P, np.eye(N), atol=1e-13)
    np.testing.assert_allclose(L @ P, P * lam[None, :], atol=1e-12)
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(L), atol=1e-12)


@pytest.mark.parametrize("N,M", [(4, 4), (5, 3), (1, 7), (6, 9)])
def test_preconditioner_equals_dense_pseudo_inverse(N, M):
    rng = np.random.default_rng(N + 100 * M)
    tau = 0.1
    S, T, _ = O.dense_operators(N, M)
    Lap = np.kron(np.eye(M), S.T @ S) + np.kron(T @ T.T, np.eye(N))
    dv = rng.uniform(0, 10, size=(N - 1, M))
    dh = rng.uniform(0, 10, size=(N, M - 1))
    r = rand_state(N, M, rng)
    z = O.precond_apply(r, dv, dh, tau, O.dct_basis(N), O.dct_basis(M))
    zu_ref = np.linalg.pinv(Lap, rcond=1e-10, hermitian=True) @ (tau * vecF(r[0]))
    np.testing.assert_allclose(vecF(z[0]), zu_ref, atol=1e-10)
    np.testing.assert_allclose(z[1], r[1] / (dv + 1 / tau), rtol=1e-14)
    np.testing.assert_allclose(z[2], r[2] / (dh + 1 / tau), rtol=1e-14)


# ------------------------------------------------------------------------------------------
# Alg. 2: PCG reaches the least-squares solution
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("rule", ["fr", "pr"])
def test_pcg_matches_lstsq(rule):
    N, M, tau = 6, 5, 1e-2
    rng = np.random.default_rng(11)
    pb = rand_problem(N, M, rng, tau)
    Wv = rng.uniform(1e-3, 1.0, size=(N - 1, M))
    Wh = rng.uniform(1e-3, 1.0, size=(N, M - 1))
    dv, dh = O.diag_d(pb.Cv, pb.Ch, Wv, Wh)
    A = dense_A(N, M, dv, dh, tau)
    x_ref = np.linalg.lstsq(A, pack(pb.b), rcond=None)[0]
    x0 = rand_state(N, M, rng)
    x, it, rel, st = O.pcg(x0, pb.b, dv, dh, tau, pb.basis_N, pb.basis_M, 1e-13, 500, rule)
    assert st == 0 and rel <= 1e-13 and it > 0
    U = x[0] - x[0].mean()
    xs = pack((U, x[1], x[2]))
    np.testing.assert_allclose(xs, x_ref, atol=1e-9 * np.abs(x_ref).max())


def test_pcg_stops_on_tolerance_and_cap():
    N, M, tau = 8, 8, 1e-2
    rng = np.random.default_rng(12)
    pb = rand_problem(N, M, rng, tau)
    dv, dh = np.ones((N - 1, M)), np.ones((N, M - 1))
    z0 = (np.zeros((N, M)), np.zeros((N - 1, M)), np.zeros((N, M - 1)))
    _, it, rel, _ = O.pcg(z0, pb.b, dv, dh, tau, pb.basis_N, pb.basis_M, 0.0, 3)
    assert it == 3
    _, it0, _, _ = O.pcg(z0, pb.b, dv, dh, tau, pb.basis_N, pb.basis_M, 10.0, 100)
    assert it0 == 0


# ------------------------------------------------------------------------------------------
# Sec. 3.1: theorems as invariants along the IRLS trajectory
# ------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_run():
    d = synthetic.config_small(seed=0, H=40, W=36)
    res = O.irls_unwrap(d["X"], None, tau=1e-2, delta=1e-3, outer_iters=8, cg_tol=1e-9,
                        cg_max=400)
    return d, res


def test_H_delta_monotone(small_run):
    _, res = small_run
    hb, hd, ha = res["h_before"], res["h_delta"], res["h_after_rw"]
    for k in range(len(hd)):
        assert hd[k] <= hb[k] * (1 + 1e-12)          # CG decreases the quadratic in (U, V)
        assert ha[k] <= hd[k] * (1 + 1e-12)          # exact W-minimisation (closed form)
        if k + 1 < len(hb):
            assert math.isclose(hb[k + 1], ha[k], rel_tol=1e-12)


def test_sufficient_decrease_condition_holds(small_run):
    """Eq. (sufficient-decrease): H_delta(x^{k+1}, W^k) <= H_delta(candidate, W^k); the paper
    reports it always held in practice (remark after the rate theorem)."""
    d, _ = small_run
    tau, delta = 1e-2, 1e-3
    pb = O.Problem(d["X"], None, tau=tau)
    U = np.zeros((pb.N, pb.M))
    Vv, Vh = O.S_op(U) - pb.Gv, O.T_op(U) - pb.Gh
    for k in range(4):
        Wv, Wh = O.reweight(Vv, Vh, pb.Cv, pb.Ch, delta)
        dv, dh = O.diag_d(pb.Cv, pb.Ch, Wv, Wh)
        cand = O.gradient_candidate(U, Vv, Vh, Wv, Wh, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta)
        h_cand = O.H_delta_value(*cand, Wv, Wh, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta)
        (U, Vv, Vh), _, _, _ = O.pcg((U, Vv, Vh), pb.b, dv, dh, tau, pb.basis_N, pb.basis_M,
                                     1e-3, 5)
        U = U - U.mean()
        h_new = O.H_delta_value(U, Vv, Vh, Wv, Wh, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, delta)
        assert h_new <= h_cand


def test_F_vs_F_delta_bound(small_run):
    """Theorem 'F vs F_delta': F <= F_delta <= F + delta ((N-1) M + N (M-1))."""
    d, res = small_run
    pb = res["problem"]
    N, M = pb.N, pb.M
    E = (N - 1) * M + N * (M - 1)
    rng = np.random.default_rng(4)
    for delta in (1e-3, 0.5):
        for x in [(res["U"], res["Vv"], res["Vh"]), rand_state(N, M, rng)]:
            F = O.F_value(*x, pb.Gv, pb.Gh, pb.Cv, pb.Ch, 1e-2)
            Fd = O.F_delta_value(*x, pb.Gv, pb.Gh, pb.Cv, pb.Ch, 1e-2, delta)
            assert F <= Fd <= F + delta * E * (1 + 1e-12)


def test_L1_objective_decreases_on_the_small_workload(small_run):
    _, res = small_run
    l1 = res["l1_obj"]
    assert all(l1[k + 1] <= l1[k] * (1 + 1e-9) for k in range(len(l1) - 1))
    assert np.allclose(res["U"].mean(), 0.0, atol=1e-12)


# ------------------------------------------------------------------------------------------
# Exact recovery, LP brute force, Newton minimiser, Schur complement
# ------------------------------------------------------------------------------------------
def test_exact_recovery_on_itoh_phase():
    X, phi = synthetic.smooth_phase(24, 20, seed=9, max_step=1.5)
    res = O.irls_unwrap(X, None, tau=1e-2, delta=1e-3, outer_iters=12, cg_tol=1e-10,
                        cg_max=500)
    err = O.best_shift_error(res["U"], phi)
    assert np.abs(err).max() < 1e-4
    K = O.k_map(res["U"], X)
    assert np.all(K - K.flat[0] == O.k_map(phi, X) - O.k_map(phi, X).flat[0])
    assert res["l1_obj"][-1] < 1e-3


def _lp_l1(pb):
    from scipy.optimize import linprog
    from scipy.sparse import csr_matrix, hstack, vstack, identity, kron, eye
    N, M = pb.N, pb.M
    S, T, _ = O.dense_operators(N, M)
    D = vstack([kron(eye(M), csr_matrix(S)), kron(csr_matrix(T.T), eye(N))]).tocsr()
    g = np.concatenate([vecF(pb.Gv), vecF(pb.Gh)])
    c = np.concatenate([vecF(pb.Cv), vecF(pb.Ch)])
    E = g.size
    # variables [u (NM), e+ (E), e- (E)];  D u - e+ + e- = g
    A_eq = hstack([D, -identity(E), identity(E)]).tocsr()
    cost = np.concatenate([np.zeros(N * M), c, c])
    bounds = [(None, None)] * (N * M) + [(0, None)] * (2 * E)
    bounds[0] = (0.0, 0.0)
    r = linprog(cost, A_eq=A_eq, b_eq=g, bounds=bounds, method="highs-ds")
    assert r.status == 0
    u = r.x[:N * M].reshape((N, M), order="F")
    return r.fun, u, D, g


def test_irls_objective_within_lp_bound_6x6():
    """L1* <= L1(U_irls) <= L1* + E (tau C_max^2 / 2 + delta) (Huber form of min_V F, plus
    the F_delta bound); the LP optimum itself is 2 pi-congruent (Sec. 2, total unimodularity)."""
    rng = np.random.default_rng(21)
    X = rng.uniform(-np.pi, np.pi, size=(6, 6)).astype(np.float32)
    coh = rng.uniform(0.3, 1.0, size=(6, 6)).astype(np.float32)
    tau, delta = 1e-4, 1e-6
    pb = O.Problem(X, coh, tau=tau)
    l1_star, u_star, D, g = _lp_l1(pb)
    kk = (D @ vecF(u_star) - g) / (2 * np.pi)
    np.testing.assert_allclose(kk, np.rint(kk), atol=1e-7)
    res = O.irls_unwrap(X, coh, tau=tau, delta=delta, outer_iters=200, cg_tol=1e-12,
                        cg_max=2000)
    E = g.size
    cmax = max(pb.Cv.max(), pb.Ch.max())
    l1 = res["l1_obj"][-1]
    assert l1_star - 1e-9 <= l1 <= l1_star + E * (tau * cmax ** 2 / 2 + delta) + 1e-6


def _newton_F_delta(pb, tau, delta, iters=200):
    N, M = pb.N, pb.M
    _, _, B = O.dense_operators(N, M)
    nu = N * M
    g = np.concatenate([vecF(pb.Gv), vecF(pb.Gh)])
    c = np.concatenate([vecF(pb.Cv), vecF(pb.Ch)])
    one = np.zeros(B.shape[1])
    one[:nu] = 1.0 / math.sqrt(nu)

    def f(x):
        v = x[nu:]
        r = B @ x - g
        return np.sum(np.sqrt(c * c * v * v + delta * delta)) + r @ r / (2 * tau)

    x = np.zeros(B.shape[1])
    x[nu:] = -g
    for _ in range(iters):
        v = x[nu:]
        s = np.sqrt(c * c * v * v + delta * delta)
        grad = B.T @ (B @ x - g) / tau
        grad[nu:] += c * c * v / s
        Hm = B.T @ B / tau
        Hm[nu:, nu:] += np.diag(c * c * delta * delta / s ** 3)
        Hm += np.outer(one, one)          # fixes the constant mode of U (C0)
        step = np.linalg.solve(Hm, grad)
        t = 1.0
        f0 = f(x)
        while f(x - t * step) > f0 - 1e-4 * t * (grad @ step) and t > 1e-12:
            t *= 0.5
        x = x - t * step
        if np.abs(step).max() * t < 1e-15:
            break
    u = x[:nu].reshape((N, M), order="F")
    return u - u.mean()


@pytest.mark.parametrize("n,delta,outer", [(6, 1.0, 200), (8, 3.0, 80)])
def test_irls_converges_to_newton_minimiser_of_F_delta(n, delta, outer):
    """IRLS with tight inner solves reaches the unique minimiser of F_delta (theorems of
    Sec. 3.1).  A large delta keeps the sublinear outer rate short on random phases."""
    rng = np.random.default_rng(33 + n)
    X = rng.uniform(-np.pi, np.pi, size=(n, n)).astype(np.float32)
    tau = 1e-2
    pb = O.Problem(X, None, tau=tau)
    u_star = _newton_F_delta(pb, tau, delta)
    res = O.irls_unwrap(X, None, tau=tau, delta=delta, outer_iters=outer, cg_tol=1e-13,
                        cg_max=2000)
    np.testing.assert_allclose(res["U"], u_star, atol=1e-8)


def test_schur_complement_equivalence():
    """Eliminating V from the linear system gives D^T Omega D U = D^T Omega G with
    Omega = C^2 / (W + tau C^2) (the sandwiched form of the remark at the end of Sec. 3.3)."""
    N, M, tau = 5, 6, 1e-2
    rng = np.random.default_rng(8)
    pb = rand_problem(N, M, rng, tau)
    Wv = rng.uniform(1e-3, 1.0, size=(N - 1, M))
    Wh = rng.uniform(1e-3, 1.0, size=(N, M - 1))
    dv, dh = O.diag_d(pb.Cv, pb.Ch, Wv, Wh)
    A = dense_A(N, M, dv, dh, tau)
    x = np.linalg.lstsq(A, pack(pb.b), rcond=None)[0]
    U_full = unpack(x, N, M)[0]
    S, T, _ = O.dense_operators(N, M)
    D = np.vstack([np.kron(np.eye(M), S), np.kron(T.T, np.eye(N))])
    Om = np.concatenate([vecF(pb.Cv ** 2 / (Wv + tau * pb.Cv ** 2)),
                         vecF(pb.Ch ** 2 / (Wh + tau * pb.Ch ** 2))])
    g = np.concatenate([vecF(pb.Gv), vecF(pb.Gh)])
    u = np.linalg.lstsq(D.T @ (Om[:, None] * D), D.T @ (Om * g), rcond=None)[0]
    u = u.reshape((N, M), order="F")
    np.testing.assert_allclose(U_full - U_full.mean(), u - u.mean(), atol=1e-10)


def test_schur_operators_equal_kronecker_forms():
    """schur_matvec = D^T diag(Om) D and schur_rhs = D^T diag(Om) g with D = [I (x) S; T^T (x) I]
    from the element definitions, Om = C^2 / (W + tau C^2) = D_w / (1 + tau D_w), and the V
    recovered from U solves the V rows of the full system."""
    N, M, tau = 6, 5, 1e-2
    rng = np.random.default_rng(18)
    pb = rand_problem(N, M, rng, tau)
    Wv = rng.uniform(1e-3, 1.0, size=(N - 1, M))
    Wh = rng.uniform(1e-3, 1.0, size=(N, M - 1))
    dv, dh = O.diag_d(pb.Cv, pb.Ch, Wv, Wh)
    Ov, Oh = O.schur_weights(dv, dh, tau)
    np.testing.assert_allclose(Ov, pb.Cv ** 2 / (Wv + tau * pb.Cv ** 2), rtol=1e-13)
    S, T, _ = O.dense_operators(N, M)
    D = np.vstack([np.kron(np.eye(M), S), np.kron(T.T, np.eye(N))])
    Om = np.concatenate([vecF(Ov), vecF(Oh)])
    U = rng.standard_normal((N, M))
    np.testing.assert_allclose(vecF(O.schur_matvec(U, Ov, Oh)), D.T @ (Om * (D @ vecF(U))),
                               atol=1e-12)
    g = np.concatenate([vecF(pb.Gv), vecF(pb.Gh)])
    np.testing.assert_allclose(vecF(O.schur_rhs(pb.Gv, pb.Gh, Ov, Oh, N, M)), D.T @ (Om * g),
                               atol=1e-12)
    Vv, Vh = O.schur_recover_v(U, pb.Gv, pb.Gh, dv, dh, tau)
    q = dense_A(N, M, dv, dh, tau) @ pack((U, Vv, Vh)) - pack(pb.b)
    nu = N * M
    assert np.abs(q[nu:]).max() < 1e-9 * np.abs(pack(pb.b)).max()


def test_pcg_schur_matches_lstsq():
    N, M, tau = 7, 6, 1e-2
    rng = np.random.default_rng(19)
    pb = rand_problem(N, M, rng, tau)
    Wv = rng.uniform(1e-2, 1.0, size=(N - 1, M))
    Wh = rng.uniform(1e-2, 1.0, size=(N, M - 1))
    dv, dh = O.diag_d(pb.Cv, pb.Ch, Wv, Wh)
    Ov, Oh = O.schur_weights(dv, dh, tau)
    f = O.schur_rhs(pb.Gv, pb.Gh, Ov, Oh, N, M)
    U, it, rel, st = O.pcg_schur(np.zeros((N, M)), f, Ov, Oh, tau, O.dct_basis(N), O.dct_basis(M),
                                 1e-13, 500)
    S, T, _ = O.dense_operators(N, M)
    D = np.vstack([np.kron(np.eye(M), S), np.kron(T.T, np.eye(N))])
    Om = np.concatenate([vecF(Ov), vecF(Oh)])
    u = np.linalg.lstsq(D.T @ (Om[:, None] * D), vecF(f), rcond=None)[0].reshape((N, M), order="F")
    assert st == 0 and rel <= 1e-13
    np.testing.assert_allclose(U - U.mean(), u - u.mean(), atol=1e-9)


def test_schur_irls_equals_full_irls_with_converged_solves():
    """With every inner solve converged, the U-only form and the paper's (U, V) form follow the
    same IRLS trajectory (the Schur complement is exact): same U, same objectives."""
    d = synthetic.make_phase(20, 18, 3, ramp=10.0, n_bumps=2, noise=0.6, coherence=True)
    kw = dict(tau=1e-2, delta=1e-2, outer_iters=5, cg_tol=1e-13, cg_max=5000)
    full = O.irls_unwrap(d["X"], d["coherence"], **kw)
    schur = O.irls_unwrap(d["X"], d["coherence"], system="schur", **kw)
    np.testing.assert_allclose(schur["U"], full["U"], atol=1e-7)
    np.testing.assert_allclose(schur["l1_obj"], full["l1_obj"], rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(schur["h_delta"], full["h_delta"], rtol=1e-8, atol=1e-9)


# ------------------------------------------------------------------------------------------
# Invariances
# ------------------------------------------------------------------------------------------
def test_invariances():
    d = synthetic.config_small(seed=1, H=20, W=18)
    X = d["X"]
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-10, cg_max=300)
    base = O.irls_unwrap(X, None, **kw)["U"]
    # transposition
    tr = O.irls_unwrap(X.T.copy(), None, **kw)["U"]
    np.testing.assert_allclose(tr.T, base, atol=1e-8)
    # 2 pi integer field and a constant added to X (float32 rounding perturbs G slightly)
    rng = np.random.default_rng(0)
    X2 = (X.astype(np.float64) + 2 * np.pi * rng.integers(-2, 3, size=X.shape) + 0.7)
    u2 = O.irls_unwrap(X2.astype(np.float32), None, **kw)["U"]
    np.testing.assert_allclose(u2, base, atol=1e-4)
    # scaling: C -> sC, delta -> s delta, tau -> tau / s leaves the trajectory unchanged
    s = 3.0
    pb = O.Problem(X, None)
    us = O.irls_unwrap(X, None, Cv=s * pb.Cv, Ch=s * pb.Ch, tau=1e-2 / s, delta=1e-3 * s,
                       outer_iters=4, cg_tol=1e-10, cg_max=300)["U"]
    np.testing.assert_allclose(us, base, atol=1e-8)


def test_preconditioner_clusters_spectrum():
    """Sec. 3.3.2: C* A C* has a far smaller condition number than A (N = M = 8 here)."""
    N = M = 8
    tau, delta = 1e-2, 1e-6
    rng = np.random.default_rng(0)
    dv = rng.uniform(0, 1 / delta, size=(N - 1, M))
    dh = rng.uniform(0, 1 / delta, size=(N, M - 1))
    A = dense_A(N, M, dv, dh, tau)
    S, T, _ = O.dense_operators(N, M)
    Dm = np.zeros_like(A)
    nu = N * M
    Dm[:nu, :nu] = A[:nu, :nu]
    Dm[nu:, nu:] = np.diag(np.diag(A)[nu:])
    w, V = np.linalg.eigh(Dm)
    keep = w > 1e-9 * w.max()
    Cs = (V[:, keep] / np.sqrt(w[keep])) @ V[:, keep].T
    def kappa(Mx):
        e = np.linalg.eigvalsh((Mx + Mx.T) / 2)
        e = e[e > 1e-9 * e.max()]
        return e.max() / e.min()
    assert kappa(Cs @ A @ Cs) < 1e-3 * kappa(A)


# ------------------------------------------------------------------------------------------
# Planted mistakes: each pin above must catch a plausible slip in the oracle
# ------------------------------------------------------------------------------------------
def _matvec_matches(apply):
    rng = np.random.default_rng(3)
    N, M, tau = 4, 5, 0.3
    dv = rng.uniform(0.1, 5.0, size=(N - 1, M))
    dh = rng.uniform(0.1, 5.0, size=(N, M - 1))
    x = rand_state(N, M, rng)
    return np.allclose(pack(apply(x, dv, dh, tau)), dense_A(N, M, dv, dh, tau) @ pack(x))


def test_planted_sign_error_in_matvec_is_caught():
    def bad(x, dv, dh, tau):
        qU, qV, qH = O.apply_A(x, dv, dh, tau)
        return qU, qV + 2 * O.S_op(x[0]) / tau, qH     # flips the sign of the -S U / tau term
    assert _matvec_matches(O.apply_A) and not _matvec_matches(bad)


def test_planted_transposed_dct_is_caught():
    N, M = 5, 4
    rng = np.random.default_rng(0)
    S, T, _ = O.dense_operators(N, M)
    Lap = np.kron(np.eye(M), S.T @ S) + np.kron(T @ T.T, np.eye(N))
    r = rand_state(N, M, rng)
    PN, lN = O.dct_basis(N)
    PM, lM = O.dct_basis(M)
    z_bad = O.precond_apply(r, np.ones((N - 1, M)), np.ones((N, M - 1)), 1.0, (PN.T, lN),
                            (PM, lM))
    ref = np.linalg.pinv(Lap, rcond=1e-10, hermitian=True) @ vecF(r[0])
    assert not np.allclose(vecF(z_bad[0]), ref, atol=1e-6)


def test_planted_missing_tau_in_rhs_is_caught():
    rng = np.random.default_rng(7)
    N, M, tau = 3, 3, 0.2
    pb = rand_problem(N, M, rng, tau)
    b_bad = (pb.b[0] * tau, pb.b[1], pb.b[2])       # drops the 1/tau of B1
    x = rand_state(N, M, rng)
    W = (np.ones((N - 1, M)), np.ones((N, M - 1)))
    dv, dh = O.diag_d(pb.Cv, pb.Ch, *W)
    res_bad = pack(O.apply_A(x, dv, dh, tau)) - pack(b_bad)

    def H(v):
        U, Vv, Vh = unpack(v, N, M)
        return O.H_delta_value(U, Vv, Vh, *W, pb.Gv, pb.Gh, pb.Cv, pb.Ch, tau, 0.1)

    v0 = pack(x)
    grad = np.array([(H(v0 + 1e-5 * e) - H(v0 - 1e-5 * e)) / 2e-5 for e in np.eye(v0.size)])
    assert not np.allclose(res_bad, grad, rtol=1e-6, atol=1e-6)


def test_paper_parameters_fixture():
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    assert g["tau"] == 1e-2 and g["delta"] == 1e-6
    assert g["max_iter_CG_start"] == 5 and g["increase_CG_iteration_factor"] == 1.7


# ------------------------------------------------------------------------------------------
# Sec. 4.3: CG budget and IRLS stop
# ------------------------------------------------------------------------------------------
def test_paper_cg_cap_rules():
    """The three cases of Sec. 4.3, with its parameters m_CG(0) = 5, eps_tol = 1e-3, alpha = 1.7,
    on a hand-worked sequence of relative improvements."""
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    m0, tol, a = g["max_iter_CG_start"], g["rel_improvement_tol"], g["increase_CG_iteration_factor"]
    # case 1: significant improvement keeps the budget
    assert O.paper_cg_cap(0.5, 5, False, tol, a) == (5, False)
    assert O.paper_cg_cap(0.5, 8, True, tol, a) == (8, False)
    # case 3: not significant, budget not raised last time -> times alpha (5 * 1.7 = 8.5 -> 8)
    assert O.paper_cg_cap(1e-4, 5, False, tol, a) == (8, True)
    assert O.paper_cg_cap(tol, 13, False, tol, a) == (22, True)      # boundary: Delta <= tol
    # case 2: not significant right after a raise -> stop
    assert O.paper_cg_cap(1e-4, 8, True, tol, a)[0] is None
    # a whole run: Delta_{k-1,k} for k = 1..6
    deltas = [0.5, 0.1, 5e-4, 0.2, 5e-4, 5e-4]
    m, raised, caps = m0, False, [m0]
    for d in deltas:
        m_next, raised = O.paper_cg_cap(d, m, raised, tol, a)
        if m_next is None:
            break
        m = m_next
        caps.append(m)
    assert caps == [5, 5, 5, 8, 8, 13] and m_next is None


@pytest.fixture(scope="module")
def schedule_case():
    d = synthetic.config_small(3, H=24, W=20)
    return d["X"], dict(tau=1e-2, delta=1e-3, outer_iters=12, cg_tol=1e-10, cg_max=1000)


def test_paper_schedule_special_cases(schedule_case):
    """eps_tol < 0 never finds an improvement insignificant: the run is the fixed schedule with
    every solve capped at m_CG(0).  eps_tol = inf finds every improvement insignificant: the
    budget is raised once at k = 1 (5 -> 8) and the run stops at k = 2, returning U^2."""
    X, kw = schedule_case
    keep = O.irls_unwrap(X, None, cg_schedule="paper", eps_tol=-1.0, **kw)
    fixed = O.irls_unwrap(X, None, **dict(kw, cg_max=5))
    assert keep["cg_cap"] == [5] * kw["outer_iters"] and not keep["schedule_stop"]
    assert np.array_equal(keep["U"], fixed["U"])
    stop = O.irls_unwrap(X, None, cg_schedule="paper", eps_tol=np.inf, **kw)
    assert stop["cg_cap"] == [5, 8] and stop["schedule_stop"]
    assert len(stop["cg_iters"]) == 2 and stop["cg_iters"][1] <= 8


def test_paper_schedule_follows_the_rule(schedule_case):
    """With the paper's parameters, the caps and the stop follow the rule applied to the run's
    own Delta_{k-1,k} = (H(x^k, W^{k-1}) - H(x^k, W^k)) / H(x^k, W^{k-1}), and every Delta is
    >= 0 (reweighting minimises H over W, Sec. 3.1)."""
    X, kw = schedule_case
    r = O.irls_unwrap(X, None, cg_schedule="paper", **kw)
    assert r["cg_cap"][0] == 5
    assert all(d >= -1e-12 for d in r["delta_rel"])
    h_now = r["h_before"] + ([r["h_stop"]] if r["schedule_stop"] else [])
    for k, d in enumerate(r["delta_rel"], start=1):
        ref = (r["h_delta"][k - 1] - h_now[k]) / r["h_delta"][k - 1]
        assert d == ref
    m, raised = 5, False
    for k, d in enumerate(r["delta_rel"], start=1):
        m, raised = O.paper_cg_cap(d, m, raised, 1e-3, 1.7)
        if m is None:
            assert r["schedule_stop"] and len(r["cg_cap"]) == k
            break
        assert r["cg_cap"][k] == m
    assert all(it <= cap for it, cap in zip(r["cg_iters"], r["cg_cap"]))


# ------------------------------------------------------------------------------------------
# Sec. 4.5: rounded IRLS and the best-shift error
# ------------------------------------------------------------------------------------------
def test_round_congruent_recovers_planted_integers():
    """U = X + 2pi K0 + c0 + small noise: the planted K0 and offset come back exactly, and the
    rounded image is X + 2pi K0 (congruent to X to float32 rounding)."""
    rng = np.random.default_rng(4)
    X = rng.uniform(-np.pi, np.pi, (40, 30)).astype(np.float32)
    K0 = rng.integers(-20, 21, (40, 30))
    c0 = 1.234
    U = (X + 2 * np.pi * K0 + c0 + 0.3 * rng.standard_normal(X.shape)).astype(np.float32)
    Ur, K, c = O.round_congruent(U, X)
    assert abs(c - c0) < 0.1
    assert np.array_equal(K, K0)
    assert np.abs(Ur.astype(np.float64) - X - 2 * np.pi * K0).max() <= 4e-6 * np.abs(Ur).max()
    # a multiple of 2pi added to U moves K by the same integer; a constant shift moves only c
    _, K2, _ = O.round_congruent((U + np.float32(2 * np.pi) * 3).astype(np.float32), X)
    assert np.array_equal(K2, K0 + 3)
    _, K3, c3 = O.round_congruent((U + np.float32(0.5)).astype(np.float32), X)
    assert np.array_equal(K3, K0) and abs(c3 - c - 0.5) < 1e-6


def test_rounded_irls_matches_true_ambiguities_on_an_easy_image():
    """On a low-noise smooth phase the unwrapped output rounds to the true integer map (the
    planted phase's own ambiguities), up to one global integer."""
    d = synthetic.make_phase(48, 40, 9, ramp=30.0, n_bumps=2, noise=0.05)
    r = O.irls_unwrap(d["X"], None, tau=1e-2, delta=1e-3, outer_iters=8, cg_tol=1e-9)
    _, K, _ = O.round_congruent(r["U"], d["X"])
    # the planted phase's own ambiguities (its constant offset aligned the same way)
    _, Ktrue, _ = O.round_congruent(d["phi_true"], d["X"])
    diff = K - Ktrue
    assert np.all(diff == diff.flat[0])


def test_best_shift_error_definition():
    """E = Xu - (U + alpha) with alpha the least-squares shift (Sec. 4.5): E has zero mean, and
    no other shift gives a smaller norm."""
    rng = np.random.default_rng(5)
    Xu = rng.standard_normal((20, 16)) * 5
    U = Xu + 3.7 + 0.1 * rng.standard_normal(Xu.shape)
    E = O.best_shift_error(U, Xu)
    assert abs(E.mean()) < 1e-12
    n0 = np.linalg.norm(E)
    for s in (-1e-3, 1e-3):
        assert np.linalg.norm(E - s) > n0


# ------------------------------------------------------------------------------------------
# Adjoint of the IRLS map: central differences of the oracle's own forward map
# ------------------------------------------------------------------------------------------
def _adjoint_case():
    N, M = 12, 10
    d = synthetic.make_phase(N, M, 5, ramp=6.0, n_bumps=1, noise=1.0, coherence=True)
    X = d["X"].astype(np.float64)
    coh = d["coherence"].astype(np.float64)
    Uref = np.random.default_rng(0).standard_normal((N, M))
    kw = dict(tau=1e-2, delta=0.05, outer_iters=3, cg_tol=1e-13, cg_max=5000)
    return X, coh, Uref, kw


def _adjoint_fd_mismatches(X, coh, Uref, kw):
    """Compares the oracle adjoint's dL/dX and dL/dcoherence (L = sum (U - U_ref)^2 through 3
    IRLS steps with converged solves) with central differences of the oracle's own forward map.
    X: Richardson-extrapolated central differences with steps 2e-2 and 1e-2 (the float32 wrap
    rounds X +- h, so smaller steps only add noise; pixels whose incident wrapped differences
    stay below pi - 0.05); coherence: steps of 1e-3.  Returns the pixels that disagree and the
    number of X pixels checked."""
    def L(Xa, ca):
        return float(np.sum((O.irls_unwrap(Xa, ca, **kw)["U"] - Uref) ** 2))

    r0 = O.irls_unwrap(X, coh, **kw)
    gX, gC, _ = O.irls_adjoint(X, coh, 2 * (r0["U"] - Uref), **kw)
    Gv, Gh = O.wrapped_gradients(X)
    N, M = X.shape
    checked, bad = 0, []
    for i, j in [(3, 4), (6, 2), (0, 0), (11, 9), (5, 5), (8, 1)]:
        inc = [abs(Gv[i - 1, j]) if i > 0 else 0, abs(Gv[i, j]) if i < N - 1 else 0,
               abs(Gh[i, j - 1]) if j > 0 else 0, abs(Gh[i, j]) if j < M - 1 else 0]
        if max(inc) < np.pi - 0.05:
            def cd(h):
                Xp, Xm = X.copy(), X.copy()
                Xp[i, j] += h
                Xm[i, j] -= h
                return (L(Xp, coh) - L(Xm, coh)) / (2 * h)
            # Richardson extrapolation of steps 2e-2 and 1e-2 (cancels the O(h^2) term)
            fd = (4.0 * cd(1e-2) - cd(2e-2)) / 3.0
            # float32 rounding of X +- h and of the wrapped difference leaves ~2e-4 of noise
            if abs(fd - gX[i, j]) > 5e-4 * max(1.0, abs(fd)):
                bad.append(("X", i, j, fd, gX[i, j]))
            checked += 1
        h = 1e-3
        cp, cm = coh.copy(), coh.copy()
        cp[i, j] += h
        cm[i, j] -= h
        fdc = (L(X, cp) - L(X, cm)) / (2 * h)
        if abs(fdc - gC[i, j]) > 1e-5 * max(1.0, abs(fdc)):
            bad.append(("coh", i, j, fdc, gC[i, j]))
    return bad, checked


def test_adjoint_matches_central_differences():
    X, coh, Uref, kw = _adjoint_case()
    bad, checked = _adjoint_fd_mismatches(X, coh, Uref, kw)
    assert not bad, bad
    assert checked >= 3


def test_planted_wrong_reweighting_derivative_is_caught(monkeypatch):
    """Dropping the C^3 V^2 / W^3 term of dD/dC (D = C^2 / W with W = sqrt(C^2 V^2 + delta^2),
    Sec. 3.1) must break the central-difference check of the coherence gradient; a sign slip
    in dD/dV must break the check of dL/dX (it reaches X through V^0 = -G)."""
    X, coh, Uref, kw = _adjoint_case()
    monkeypatch.setattr(O, "dD_dC", lambda C, V, W: 2.0 * C / W)
    bad, _ = _adjoint_fd_mismatches(X, coh, Uref, kw)
    assert any(b[0] == "coh" for b in bad)
    monkeypatch.undo()
    monkeypatch.setattr(O, "dD_dV", lambda C, V, W: (C ** 4) * V / W ** 3)
    bad, _ = _adjoint_fd_mismatches(X, coh, Uref, kw)
    assert any(b[0] == "X" for b in bad)


# ------------------------------------------------------------------------------------------
# Edge weights from coherence (reading of Sec. 2's weights for a per-pixel coherence map)
# ------------------------------------------------------------------------------------------
def _edges_touched_by_pixel(fn, N, M, i, j):
    """Which edge weights change when only pixel (i, j)'s coherence changes."""
    rng = np.random.default_rng(i * 31 + j)
    c = rng.uniform(0.05, 1.0, size=(N, M))
    Cv0, Ch0 = fn(c, N, M)
    c2 = c.copy()
    c2[i, j] += 0.25
    Cv1, Ch1 = fn(c2, N, M)
    return set(map(tuple, np.argwhere(Cv1 != Cv0))), set(map(tuple, np.argwhere(Ch1 != Ch0)))


def _edge_weight_pins_hold(fn):
    """An edge's weight depends on the coherence of its two end pixels only, equally on both:
    raising one pixel's coherence by h raises exactly its (up to) four incident edges, each by
    h / 2; uniform coherence c gives uniform weights c on every edge that exists."""
    for N, M in ((7, 7), (6, 9)):
        for i, j in ((0, 0), (3, 5), (N - 1, M - 1), (2, 0), (N - 1, 4)):
            tv, th = _edges_touched_by_pixel(fn, N, M, i, j)
            want_v = {(a, j) for a in (i - 1, i) if 0 <= a < N - 1}
            want_h = {(i, b) for b in (j - 1, j) if 0 <= b < M - 1}
            if tv != want_v or th != want_h:
                return False
        Cv, Ch = fn(np.full((N, M), 0.3), N, M)
        if Cv.shape != (N - 1, M) or Ch.shape != (N, M - 1):
            return False
        if not (np.allclose(Cv, 0.3) and np.allclose(Ch, 0.3)):
            return False
        rng = np.random.default_rng(N)
        c = rng.uniform(0.05, 1.0, size=(N, M))
        c2 = c.copy()
        c2[2, 3] += 0.25
        Cv0, Ch0 = fn(c, N, M)
        Cv1, Ch1 = fn(c2, N, M)
        if not (np.allclose((Cv1 - Cv0)[(Cv1 - Cv0) != 0], 0.125)
                and np.allclose((Ch1 - Ch0)[(Ch1 - Ch0) != 0], 0.125)):
            return False
    return True


def test_edge_weights_are_local_and_symmetric():
    assert _edge_weight_pins_hold(O.edge_weights)
    Cv, Ch = O.edge_weights(None, 5, 4)
    assert np.array_equal(Cv, np.ones((4, 4))) and np.array_equal(Ch, np.ones((5, 3)))


def test_transposition_with_non_symmetric_coherence():
    """Transposing X and the coherence map transposes U (the problem has no preferred axis), with
    a coherence map that is far from symmetric."""
    d = synthetic.make_phase(18, 14, 4, ramp=8.0, n_bumps=2, noise=0.7, coherence=True)
    X = d["X"]
    coh = d["coherence"].copy()
    coh[:, :5] *= 0.2             # a low-coherence band along one side only
    assert np.abs(coh[:14, :14] - coh[:14, :14].T).max() > 0.3
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-11, cg_max=600)
    base = O.irls_unwrap(X, coh, **kw)
    tr = O.irls_unwrap(X.T.copy(), coh.T.copy(), **kw)
    np.testing.assert_allclose(tr["U"].T, base["U"], atol=1e-8)
    np.testing.assert_allclose(tr["l1_obj"], base["l1_obj"], rtol=1e-6)


def test_planted_axis_swap_in_edge_weights_is_caught(monkeypatch):
    """Averaging along the wrong axis (on a square image the shapes still fit): the locality pin
    fails.  A swap of both planes (weights taken from the transposed coherence) keeps the
    transposition invariance, so that check alone could not catch it; a swap of one plane
    breaks both."""
    def both_swapped(coherence, N, M):
        c = np.asarray(coherence, dtype=np.float64)
        return 0.5 * (c[:, 1:] + c[:, :-1]).T, 0.5 * (c[1:, :] + c[:-1, :]).T

    def one_swapped(coherence, N, M):
        c = np.asarray(coherence, dtype=np.float64)
        return 0.5 * (c[:, 1:] + c[:, :-1]).T, 0.5 * (c[:, 1:] + c[:, :-1])

    square = lambda fn: (lambda c, N, M: fn(c, N, M) if N == M else O.edge_weights(c, N, M))  # noqa
    assert not _edge_weight_pins_hold(square(both_swapped))
    assert not _edge_weight_pins_hold(square(one_swapped))
    d = synthetic.make_phase(14, 14, 4, ramp=8.0, n_bumps=2, noise=0.7, coherence=True)
    X, coh = d["X"], d["coherence"].copy()
    coh[:, :5] *= 0.2
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=3, cg_tol=1e-11, cg_max=600)
    monkeypatch.setattr(O, "edge_weights", one_swapped)
    base = O.irls_unwrap(X, coh, **kw)
    tr = O.irls_unwrap(X.T.copy(), coh.T.copy(), **kw)
    assert np.abs(tr["U"].T - base["U"]).max() > 1e-6
