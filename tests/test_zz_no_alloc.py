"""The allocation-free preconditioner entry point, checked against the plan-based one.

irls_precond_laplacian_noalloc serves callers that cannot allocate device memory (plug-ins
whose framework owns all device memory, latency-critical code that must avoid cudaMalloc's
implicit synchronisation).  It keeps its scratch in a fixed buffer inside the library, which
every call reuses; the calls below are consecutive and of different shapes so that leftovers
of an earlier call would show.  This file sorts last so that a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def irls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_09961_gb300 as m
    m.lib()
    return m


def test_noalloc_matches_plan_entry_point_on_consecutive_calls(irls):
    L = irls.lib()
    tau = 1e-2
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for H, W, seed in [(200, 150, 0), (96, 256, 1), (200, 150, 2), (256, 256, 3)]:
        g = torch.Generator(device="cuda").manual_seed(seed)
        R = torch.randn(H, W, device="cuda", generator=g)
        with irls.Plan(H, W, tau=tau, precision="fp32") as plan:
            Z_ref = irls.precond_laplacian(plan, R)
        Z = torch.full_like(R, float("nan"))
        rc = L.irls_precond_laplacian_noalloc(ctypes.c_void_p(R.data_ptr()),
                                              ctypes.c_void_p(Z.data_ptr()), H, W,
                                              ctypes.c_float(tau), stream)
        assert rc == 0, rc
        torch.cuda.synchronize()
        scale = float(Z_ref.abs().max())
        # the float32 preconditioner tolerance used against the oracle: 2e-5 of the largest output
        assert float((Z - Z_ref).abs().max()) <= 2e-5 * scale


def _noalloc(irls, R, tau):
    L = irls.lib()
    H, W = R.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Z = torch.full_like(R, float("nan"))
    rc = L.irls_precond_laplacian_noalloc(ctypes.c_void_p(R.data_ptr()),
                                          ctypes.c_void_p(Z.data_ptr()), H, W,
                                          ctypes.c_float(tau), stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return Z.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("H,W", [(17, 33), (1, 200), (255, 3), (256, 255), (255, 256), (200, 1)])
def test_noalloc_matches_oracle(irls, H, W):
    """Against the FP64 oracle's Laplacian block (Sec. 3.3: the Sylvester solve in the DCT
    eigenbasis, zero frequency dropped), at the float32 preconditioner's bound: 2e-5 of the
    largest output.  (1, 200) and (200, 1) have a single eigenvalue 0 along one side, (255, 3)
    and (17, 33) are odd and ragged, and (256, 255) / (255, 256) use the whole buffer: the
    entry point refuses any shape whose layout would not fit it (IRLS_ERR_SHAPE), so a change of
    the layout shows here as a refusal, never as a write beyond the buffer."""
    from oracle import irls as O
    tau = 1e-2
    R = np.random.default_rng(H * 1000 + W).standard_normal((H, W)).astype(np.float32)
    Z = _noalloc(irls, torch.as_tensor(R).cuda(), tau)
    z_ref = O.precond_apply((R.astype(np.float64), np.zeros((H - 1, W)), np.zeros((H, W - 1))),
                            np.zeros((H - 1, W)), np.zeros((H, W - 1)), tau, O.dct_basis(H),
                            O.dct_basis(W))[0]
    scale = np.abs(z_ref).max() + 1e-30
    assert np.abs(Z - z_ref).max() <= 2e-5 * scale


def test_noalloc_rejects_sizes_beyond_its_buffer(irls):
    L = irls.lib()
    R = torch.zeros(300, 300, device="cuda")
    Z = torch.zeros_like(R)
    p, q = ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(Z.data_ptr())
    assert L.irls_precond_laplacian_noalloc(p, q, 257, 10, ctypes.c_float(1e-2), None) == -2
    assert L.irls_precond_laplacian_noalloc(p, q, 10, 300, ctypes.c_float(1e-2), None) == -2
    assert L.irls_precond_laplacian_noalloc(p, q, 0, 10, ctypes.c_float(1e-2), None) == -2
    assert L.irls_precond_laplacian_noalloc(None, q, 10, 10, ctypes.c_float(1e-2), None) == -1
    assert L.irls_precond_laplacian_noalloc(p, q, 10, 10, ctypes.c_float(0.0), None) == -1
