"""Tiled unwrapping of one large image on the batched form (irls_tiled_*): against the oracle's
tiled method on a small image cut into four tiles, and against a single-plan solve of a larger
image (the integer ambiguity maps)."""
import numpy as np
import pytest

from oracle import irls as O
import synthetic
from test_gpu_parity import assert_unwrap_parity, k_agreement

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def irls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_09961_gb300 as m
    m.lib()
    return m


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("law,H,W,tile,overlap", [("coherence", 200, 180, 128, 32),
                                                  ("mixed", 290, 280, 160, 30)])
def test_tiled_matches_oracle_tiled(irls, law, H, W, tile, overlap):
    """Four tiles (2 x 2), solves tight enough (cg_tol 1e-8) that the tiles' solutions are
    determined: U, the L1 objective of the stitched image and its integer map as for a single
    image, with no envelope; the tiles' constants within the U bar."""
    gen = synthetic.config_2048 if law == "coherence" else synthetic.config_4096_mixed
    d = gen(seed=50, H=H, W=W)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-8, cg_max=3000)
    ref = O.irls_unwrap_tiled(d["X"], d["coherence"], tile=tile, overlap=overlap, **kw)
    assert len(ref["tiles"]) == 4
    with irls.Tiled(H, W, tile=tile, overlap=overlap, tau=1e-2, delta=1e-3, outer_iters=4,
                    cg_tol=1e-8, cg_max_iter=3000) as t:
        assert t.n_tiles == 4 and t.n_pairs == 4
        U, st, c = t.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    pb = O.Problem(d["X"], d["coherence"])
    l1o = O.l1_objective(ref["U"], pb.Gv, pb.Gh, pb.Cv, pb.Ch)
    Ug = U.cpu().numpy().astype(np.float64)
    l1g = O.l1_objective(Ug, pb.Gv, pb.Gh, pb.Cv, pb.Ch)
    assert_unwrap_parity(Ug, ref["U"], l1g, l1o, d["X"], ref={"U": ref["U"], "problem": pb},
                         strict=True, case=f"{H}x{W} {law}-law tiled 2x2 ({tile}, {overlap}) "
                                           "bf16x3 tol 1e-8")
    assert np.abs(np.array(c) - ref["constants"]).max() <= 1e-3
    assert all(s["outer_done"] == 4 for s in st)


def test_tiled_against_single_plan(irls):
    """A 2048 x 4096 image of the coherence law, tiles of 1024 with 64 pixels of overlap (3 x 5
    tiles), against the same image solved by one plan: the integer ambiguity maps agree on
    >= 99.9 % of the pixels (up to one global integer), and the L1 objectives are stated."""
    import parity_log
    H, W = 2048, 4096
    d = synthetic.config_2048(seed=60, H=H, W=W)
    X, C = cuda(d["X"]), cuda(d["coherence"])
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=20, cg_tol=1e-6, cg_max_iter=1000)
    with irls.Tiled(H, W, tile=1024, overlap=64, precision="bf16x3", **kw) as t:
        assert t.n_tiles == 15
        Ut, st, _ = t.unwrap(X, C)
    with irls.Plan(H, W, precision="bf16x3", **kw) as p:
        Us, ss = p.unwrap(X, C)
    Ut = Ut.cpu().numpy().astype(np.float64)
    Us = Us.cpu().numpy().astype(np.float64)
    pb = O.Problem(d["X"], d["coherence"])
    l1t = O.l1_objective(Ut, pb.Gv, pb.Gh, pb.Cv, pb.Ch)
    l1s = O.l1_objective(Us, pb.Gv, pb.Gh, pb.Cv, pb.Ch)
    kag = k_agreement(Ut, Us, d["X"])
    parity_log.record(case=f"{H}x{W} tiled (1024, 64) vs single plan, bf16x3", err_u=float("nan"),
                      atol=float("nan"), dl1_rel=(l1t - l1s) / l1s, l1_bar_rel=float("nan"),
                      k_agree=kag, l1=l1s, bars=f"L1 tiled {l1t:.6g}, single {l1s:.6g}")
    assert kag >= 0.999, kag
