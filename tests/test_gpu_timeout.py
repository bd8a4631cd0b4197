"""Failure detection on the GPU without a fault: the folded preconditioner's bounded dependency
waits run out (a row-panel count that never arrives, set by a test hook), the launch returns the
timeout status, and the context and the plan stay usable."""
import time

import numpy as np
import pytest

import synthetic

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


OPTS = dict(tau=1e-2, delta=1e-3, outer_iters=1, cg_tol=1e-6, cg_max_iter=50, precision="bf16x3")


def test_stalled_dependency_wait_times_out_and_recovers(irls):
    d = synthetic.config_2048(seed=90, H=512, W=512)
    X, C = cuda(d["X"]), cuda(d["coherence"])
    with irls.Plan(512, 512, **OPTS) as ref:
        U_ref, s_ref = ref.unwrap(X, C)
    with irls.Plan(512, 512, **OPTS) as p:
        assert p.folded
        assert irls.lib().irls_debug_stall_fold(p.handle, 1) == 0
        t0 = time.perf_counter()
        with pytest.raises(irls.IrlsError) as e:
            p.unwrap(X, C)
        elapsed = time.perf_counter() - t0
        assert e.value.code == -6                     # IRLS_ERR_TIMEOUT
        assert elapsed < 30.0                          # bounded: one wait budget (about 2 s)
        torch.cuda.synchronize()                       # the context is usable
        assert float(torch.ones(4, device="cuda").sum()) == 4.0
        assert irls.lib().irls_debug_stall_fold(p.handle, 0) == 0
        U, s = p.unwrap(X, C)                          # the same plan solves normally again
        assert torch.equal(U, U_ref)
        assert s["cg_iters"] == s_ref["cg_iters"]


def test_stall_hook_needs_the_folded_form(irls):
    with irls.Plan(200, 300, **OPTS) as p:
        assert not p.folded
        assert irls.lib().irls_debug_stall_fold(p.handle, 1) == -8
