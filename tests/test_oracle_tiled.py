"""Pins of the oracle's tiled unwrapping (the paper's future-work step for very large images,
Sec. 5, on the 4000 x M images of Sec. 4.5), CPU only: the layout partitions the image, one
tile is the plain method, known constants come back exactly, and an Itoh-satisfying phase is
recovered exactly through the tiles."""
import numpy as np
import pytest

from oracle import irls as O
import synthetic


@pytest.mark.parametrize("n,t,o", [(1000, 256, 32), (256, 256, 32), (200, 256, 32), (257, 256, 32),
                                   (4000, 1024, 64), (16000, 1024, 64), (1, 8, 2), (513, 128, 1)])
def test_layout_covers_and_partitions(n, t, o):
    st = O.tile_starts(n, t, o)
    tt = min(t, n)
    assert st[0] == 0 and st[-1] + tt == n
    assert all(b > a for a, b in zip(st, st[1:]))
    assert all(a + tt > b for a, b in zip(st, st[1:])), "consecutive tiles overlap or touch"
    assert all(b - a <= t - o for a, b in zip(st, st[1:]))
    cores = O.tile_cores(st, t, n)
    assert cores[0][0] == 0 and cores[-1][1] == n
    for (lo, hi), (lo2, _) in zip(cores, cores[1:]):
        assert hi == lo2
    for a, (lo, hi) in zip(st, cores):
        assert a <= lo < hi <= a + tt, "every core lies inside its tile"


def test_one_tile_is_the_plain_method():
    d = synthetic.config_2048(seed=3, H=40, W=36)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=3, cg_tol=1e-8, cg_max=1000)
    a = O.irls_unwrap(d["X"], d["coherence"], **kw)
    b = O.irls_unwrap_tiled(d["X"], d["coherence"], tile=64, overlap=8, **kw)
    assert len(b["tiles"]) == 1
    np.testing.assert_allclose(b["U"], a["U"] - a["U"].mean(), atol=1e-12)


def _planted(seed=0, H=90, W=70, t=32, o=10, slip=0):
    rng = np.random.default_rng(seed)
    truth = np.cumsum(np.cumsum(rng.standard_normal((H, W)), 0), 1) * 0.05
    rs, cs = O.tile_starts(H, t, o), O.tile_starts(W, t, o)
    sol, k = [], 0
    for r in rs:
        for c in cs:
            u = truth[r:r + t, c:c + t] + rng.uniform(-50, 50)
            # a few pixels a tile unwrapped with another number of cycles
            m = rng.random(u.shape) < 0.02
            u = u + 2 * np.pi * m * rng.choice([-1, 1], size=u.shape)
            sol.append(u)
            k += 1
    return truth, sol, rs, cs


def test_known_constants_come_back():
    """Tile solutions equal to one image plus a random constant each (and 2 % of their pixels
    off by one cycle): the stitched image is that image outside the off pixels, whatever the
    constants."""
    truth, sol, rs, cs = _planted()
    H, W = truth.shape
    U, c, pairs = O.stitch_tiles(sol, rs, cs, 32, 32, H, W)
    d = U - (truth - truth.mean())
    d -= np.median(d)
    assert np.mean(np.abs(d) < 1e-9) > 0.95
    assert len(pairs) == (len(rs) - 1) * len(cs) + len(rs) * (len(cs) - 1)


def test_planted_sign_slip_in_the_constants_is_caught(monkeypatch):
    """Reading the offset the wrong way round (U_s - U_t) must break the recovery above."""
    truth, sol, rs, cs = _planted()
    H, W = truth.shape
    real = O.overlap_offset
    monkeypatch.setattr(O, "overlap_offset", lambda a, b: real(b, a))
    U, _, _ = O.stitch_tiles(sol, rs, cs, 32, 32, H, W)
    d = U - (truth - truth.mean())
    d -= np.median(d)
    assert np.mean(np.abs(d) < 1e-9) < 0.5


def test_exact_recovery_through_tiles():
    """An Itoh-satisfying smooth phase without noise (|gradient| < pi everywhere) is recovered up
    to a constant by every tile, so the stitched result is the phase up to a constant."""
    X, phi = synthetic.smooth_phase(80, 72, 3, max_step=2.0)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-11, cg_max=2000)
    r = O.irls_unwrap_tiled(X, None, tile=40, overlap=8, **kw)
    truth = phi - phi.mean()
    assert len(r["tiles"]) == 6
    assert np.abs(r["U"] - truth).max() < 1e-5
