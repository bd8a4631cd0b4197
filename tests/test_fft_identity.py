"""The identities the fast-transform preconditioner (IRLS_DCT_FFT) is built on, restated in
numpy float64 and checked against the oracle's dense DCT basis and preconditioner (no GPU):

  * DCT-II through an FFT of the even/odd-reordered sequence (Makhoul): with v_m = x_2m,
    v_(N-1-m) = x_(2m+1) and V = DFT(v), (P^T x)_k = c_k Re(exp(-i pi k / 2N) V_k);
  * two real sequences in one complex transform (a + i b), separated by the conjugate symmetry
    of a real sequence's DFT;
  * the fused step per frequency pair (k, N-k): one complex product per sequence gives both
    coefficients, the division by the eigenvalues, and one product per sequence gives both
    inverse spectra; the inverse sum by a forward FFT of the conjugate;
  * the Stockham auto-sort stage formula with radix 16, 8, 4, 2 and 5 stages;
  * the shared-memory layouts: every map is a bijection, and the access patterns of a stage fall
    on distinct banks (the swizzled column strip and the padded pair layout)."""
import numpy as np
import pytest

from oracle import irls as O


def radices(n):
    rs = []
    while n > 1:
        r = 16 if n % 16 == 0 else 8 if n % 8 == 0 else 4 if n % 4 == 0 else 2 if n % 2 == 0 \
            else 5
        rs.append(r)
        n //= r
    return rs


def stockham(x):
    """Forward DFT by the auto-sort stages: butterfly j of a stage with sub-length ns reads
    x[j + r N/R], multiplies by exp(-2 pi i k r / (ns R)) (k = j mod ns), takes a length-R DFT
    and writes y[(j // ns) ns R + k + r ns]."""
    n = len(x)
    x = np.asarray(x, dtype=complex).copy()
    ns = 1
    for R in radices(n):
        y = np.empty_like(x)
        nj = n // R
        q = np.arange(R)
        F = np.exp(-2j * np.pi * np.outer(q, q) / R)
        for j in range(nj):
            k = j % ns
            v = x[j + q * nj] * np.exp(-2j * np.pi * k * q / (ns * R))
            y[(j // ns) * ns * R + k + q * ns] = F @ v
        x = y
        ns *= R
    return x


def reorder(x):
    n = len(x)
    v = np.empty(n)
    v[:(n + 1) // 2] = x[0::2]
    v[n - 1 - np.arange(n // 2)] = x[1::2]
    return v


def ck(n):
    c = np.full(n, np.sqrt(2.0 / n))
    c[0] = np.sqrt(1.0 / n)
    return c


@pytest.mark.parametrize("n", [2, 16, 64, 128, 256, 2048, 2000, 4000])
def test_stockham_stages_are_the_dft(n):
    x = np.random.default_rng(n).standard_normal(n) + 1j * np.random.default_rng(n + 1).standard_normal(n)
    assert np.allclose(stockham(x), np.fft.fft(x), atol=1e-10 * np.sqrt(n))


@pytest.mark.parametrize("n", [64, 128, 512, 2000])
def test_dct2_of_two_sequences_by_one_fft(n):
    P = O.dct_basis(n)[0]
    rng = np.random.default_rng(n)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    Z = stockham(reorder(a) + 1j * reorder(b))
    Zc = np.conj(Z[(-np.arange(n)) % n])
    t = np.exp(-1j * np.pi * np.arange(n) / (2 * n))
    Xa = ck(n) * np.real(t * (Z + Zc) / 2)
    Xb = ck(n) * np.real(t * (Z - Zc) / 2j)
    assert np.allclose(Xa, P.T @ a, atol=1e-12)
    assert np.allclose(Xb, P.T @ b, atol=1e-12)


def fused_column_solve(T, tau, lam_n, lam_m):
    """The column pass as the kernel arranges it: columns in pairs, forward transform, the
    per-pair fused step, inverse by the conjugate forward transform; also rho_U by Parseval."""
    n, w = T.shape
    t = np.exp(-1j * np.pi * np.arange(n) / (2 * n))
    c = ck(n)
    out = np.zeros_like(T)
    rho = 0.0
    for ja in range(0, w, 2):
        jb = ja + 1
        Z = stockham(reorder(T[:, ja]) + 1j * reorder(T[:, jb]))
        S = np.zeros(n, dtype=complex)
        for k in range(n // 2 + 1):
            kc = (n - k) % n
            va = 0.5 * complex(Z[k].real + Z[kc].real, Z[k].imag - Z[kc].imag)
            vb = 0.5 * complex(Z[k].imag + Z[kc].imag, -(Z[k].real - Z[kc].real))
            wa, wb = t[k] * va, t[k] * vb
            x = {(0, k): c[k] * wa.real, (1, k): c[k] * wb.real}
            if kc != k:
                x.update({(0, kc): -c[kc] * wa.imag, (1, kc): -c[kc] * wb.imag})
            s = {}
            for (q, kk), v in x.items():
                j = ja + q
                s[(q, kk)] = 0.0 if (kk == 0 and j == 0) else v / (lam_n[kk] + lam_m[j])
            rho += sum(x[e] * s[e] for e in x) / tau
            if k == 0:
                S[0] = complex(c[0] * s[(0, 0)], -c[0] * s[(1, 0)])
                continue
            pa = np.conj(t[k]) * complex(c[k] * s[(0, k)], -c[kc] * s[(0, kc)]) * 0.5
            pb = np.conj(t[k]) * complex(c[k] * s[(1, k)], -c[kc] * s[(1, kc)]) * 0.5
            S[k] = complex(pa.real - pb.imag, -(pa.imag + pb.real))
            if kc != k:
                S[kc] = complex(pa.real + pb.imag, pa.imag - pb.real)
        z = stockham(S)
        m = np.array([n - 1 - (i >> 1) if i & 1 else i >> 1 for i in range(n)])
        out[:, ja] = z[m].real
        out[:, jb] = -z[m].imag
    return out, rho


@pytest.mark.parametrize("n,w", [(16, 8), (64, 32), (32, 64)])
def test_fused_column_step_is_the_laplacian_block(n, w):
    """Row transforms (as the oracle's basis) then the fused column pass then the inverse row
    transforms reproduce the oracle's preconditioner; rho equals r^T z."""
    tau = 1e-2
    R = np.random.default_rng(n * w).standard_normal((n, w))
    Pn, Pm = O.dct_basis(n)[0], O.dct_basis(w)[0]
    lam_n = 2 - 2 * np.cos(np.pi * np.arange(n) / n)
    lam_m = 2 - 2 * np.cos(np.pi * np.arange(w) / w)
    T = tau * R @ Pm
    Tc, rho = fused_column_solve(T, tau, lam_n, lam_m)
    Z = Tc @ Pm.T
    z_ref = O.precond_apply((R, np.zeros((n - 1, w)), np.zeros((n, w - 1))), np.zeros((n - 1, w)),
                           np.zeros((n, w - 1)), tau, O.dct_basis(n), O.dct_basis(w))[0]
    assert np.abs(Z - z_ref).max() <= 1e-12 * np.abs(z_ref).max()
    assert abs(rho - float(np.sum(R * z_ref))) <= 1e-12 * abs(rho)


def strip_row_two(m):
    g = m >> 3
    return m ^ (((g >> 1) + (g & 1)) & 7)


def pair_slot(m):
    return m + (m >> 4)


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
def test_shared_layouts_are_bijective_and_conflict_free(n):
    """Sides of 1024 and more (column strips of two transforms).
    Column strip of two transforms (16-byte rows, swizzled): the eight rows of a half-warp
    hit eight different 16-byte bank groups for consecutive rows, the first stage's reordered
    reads (rows two apart) and its writes (rows sixteen apart).  Row pairs (8-byte slots, one
    slot of padding every 16): a half-warp's sixteen slots hit sixteen bank pairs for
    consecutive elements, the first stage's writes and the reordered stores of the load."""
    rows = [strip_row_two(m) for m in range(n)]
    assert sorted(rows) == list(range(n))
    src = lambda m: 2 * m if m < n // 2 else 2 * n - 1 - 2 * m   # noqa: E731
    nj = n // 16
    for j0 in range(0, nj, 8):
        for r in range(16):
            for ms in ([j + r * nj for j in range(j0, j0 + 8)],
                       [src(j + r * nj) for j in range(j0, j0 + 8)],
                       [16 * j + r for j in range(j0, j0 + 8)]):
                assert len({strip_row_two(m) & 7 for m in ms}) == 8
    for j0 in range(0, nj, 16):
        for r in range(16):
            for ms in ([j + r * nj for j in range(j0, j0 + 16)],
                       [16 * j + r for j in range(j0, min(j0 + 16, nj))]):
                assert len({pair_slot(m) % 16 for m in ms}) == len(ms)
    # the load's reordered stores: thread t stores elements 4t .. 4t+3 of a row
    pos = lambda i: n - 1 - (i >> 1) if i & 1 else i >> 1   # noqa: E731
    for t0 in range(0, n // 4, 16):
        for c in range(4):
            slots = {pair_slot(pos(4 * t + c)) % 16 for t in range(t0, t0 + 16)}
            assert len(slots) == 16
