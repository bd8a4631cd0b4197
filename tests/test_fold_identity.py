"""The even / odd fold of the DCT-II basis that the folded preconditioner is built on, for even
and odd sides (numpy, float64; no GPU): P[n-1-a][k] = (-1)^k P[a][k], so

  forward:  (P^T r)[2b]   = sum_{a < ceil(n/2)} P[a][2b]   s[a],  s[a] = r[a] + r[n-1-a] (a < n/2),
                                                                   s[mid] = r[mid] (odd n);
            (P^T r)[2b+1] = sum_{a < floor(n/2)} P[a][2b+1] d[a], d[a] = r[a] - r[n-1-a];
  inverse:  (P g)[a] = E[a] + O[a], (P g)[n-1-a] = E[a] - O[a] with E, O the products of the
            even and odd halves, and O[mid] = 0 for odd n (the middle row of the odd-frequency
            half is zero), so the middle entry is written consistently twice."""
import numpy as np
import pytest

from oracle import irls as O


@pytest.mark.parametrize("n", [2, 7, 8, 255, 256, 257, 300, 301])
def test_fold_forward_and_inverse(n):
    P = O.dct_basis(n)[0]                       # P[a][k], orthonormal DCT-II
    rng = np.random.default_rng(n)
    r = rng.standard_normal(n)
    g = rng.standard_normal(n)
    he, ho = (n + 1) // 2, n // 2               # even / odd frequencies and spatial half sides
    a = np.arange(he)
    # mirror symmetry of the basis
    for k in range(n):
        assert np.allclose(P[n - 1 - np.arange(n), k], (-1) ** k * P[:, k], atol=1e-13)
    # folded residual: sums (middle counted once) and differences (middle zero)
    s = r[a] + r[n - 1 - a]
    d = r[a] - r[n - 1 - a]
    if n % 2:
        s[he - 1] = r[he - 1]
        d[he - 1] = 0.0
    Pe = P[:he, 0::2]                           # he x he: spatial half, even frequencies
    Po = P[:he, 1::2]                           # he x ho: spatial half, odd frequencies
    full = P.T @ r
    assert np.allclose(full[0::2], Pe.T @ s, atol=1e-12)
    assert np.allclose(full[1::2], Po.T @ d, atol=1e-12)
    # inverse: E + O on the first half, E - O on the mirrored half
    E = Pe @ g[0::2]
    Od = Po @ g[1::2]
    z = P @ g
    assert np.allclose(z[a], E + Od, atol=1e-12)
    assert np.allclose(z[n - 1 - a], E - Od, atol=1e-12)
    if n % 2:
        # middle row of the odd half: zero (up to the cosine's rounding here; the library's basis
        # build stores exact zeros there)
        assert np.all(np.abs(Po[he - 1]) < 1e-13)
