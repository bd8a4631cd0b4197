"""Large non-square images 4000 x M (the paper's scaling shapes, Sec. 4.4): the folded
tensor-core preconditioner with halves padded to multiples of 256 (and the direct form on
request), against the oracle where it finishes in seconds and against invariants beyond that."""
import numpy as np
import pytest

from oracle import irls as O
import synthetic
from test_gpu_parity import assert_unwrap_parity

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


@pytest.mark.parametrize("form", ["folded", "direct"])
def test_4000x2000_first_outer_matches_oracle(irls, form):
    """4000 x 2000 (8 Mpix), split-bf16: one outer step of 4 CG iterations element by element
    (bound as for the 2048 x 2048 truncated run: 4 x 5e-5 x max|U|), both preconditioner forms."""
    d = synthetic.config_4096_mixed(seed=40, H=4000, W=2000)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=1, cg_tol=1e-6, cg_max=4)
    ref = O.irls_unwrap(d["X"], d["coherence"], **kw)
    with irls.Plan(4000, 2000, delta=1e-3, outer_iters=1, cg_tol=1e-6, cg_max_iter=4,
                   precision="bf16x3", dct_form=form) as p:
        assert p.folded == (form == "folded")
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["cg_iters"] == [4]
    atol = max(1e-3, 4 * 5e-5 * np.abs(ref["U"]).max())
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         atol=atol, ref=ref, case=f"4000x2000 mixed-law bf16x3 ({form}) 1 step x 4 CG",
                         truncated=True)


@pytest.mark.parametrize("W", [8000, 16000])
def test_4000xM_invariants(irls, W):
    """4000 x 8000 and 4000 x 16000 (64 Mpix, about 12 GB of device memory): three outer steps;
    the monotone quantities of Sec. 3.1 hold on the device statistics, U has zero mean, the plan
    runs the folded form with padded halves (2000 -> 2048), and the solve reports no error."""
    d = synthetic.config_4096_mixed(seed=41, H=4000, W=W)
    with irls.Plan(4000, W, delta=1e-3, outer_iters=3, cg_tol=1e-6, precision="bf16x3") as p:
        assert p.folded
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["return_code"] in (0, 1)
    f, h = st["f_delta"], st["h_delta"]
    for k in range(len(h)):
        assert h[k] <= f[k] * (1 + 1e-5)
        if k + 1 < len(f):
            assert f[k + 1] <= h[k] * (1 + 1e-5)
    assert st["l1_obj"][-1] < st["l1_obj"][0]
    assert abs(float(U.double().mean())) < 1e-3
