"""The U-only (Schur complement) system on the GPU against the FP64 oracle's U-only form, and
against the paper's (U, V) form where both solves converge."""
import numpy as np
import pytest

from oracle import irls as O
import synthetic
from test_gpu_parity import assert_unwrap_parity, oracle_with_envelope, parity_atol

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


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("H,W,seed", [(96, 80, 3), (256, 256, 5), (130, 257, 6)])
def test_schur_matches_oracle(irls, H, W, seed, prec):
    d = synthetic.config_2048(seed=seed, H=H, W=W)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=6, cg_tol=1e-6, cg_max=1000, system="schur")
    ref, env = oracle_with_envelope(d["X"], d["coherence"], kw)
    U, st = irls.unwrap(cuda(d["X"]), cuda(d["coherence"]), eps=1e-3, outer_iters=6,
                        cg_tol=1e-6, precision=prec, system="schur", return_stats=True)
    assert st["return_code"] == 0
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         atol=parity_atol(env), ref=ref, env=env,
                         case=f"{H}x{W} coherence U-only {prec} tol 1e-6")
    # the objectives of Sec. 3.1 recorded along the way agree too
    np.testing.assert_allclose(st["h_delta"], ref["h_delta"], rtol=2e-4)


def test_schur_equals_full_when_converged(irls):
    """Both systems solved to 1e-9 give the same IRLS iterates (the elimination is exact)."""
    d = synthetic.config_2048(seed=9, H=64, W=48)
    outs = {}
    for system in ("full", "schur"):
        U, st = irls.unwrap(cuda(d["X"]), cuda(d["coherence"]), eps=1e-2, outer_iters=4,
                            cg_tol=1e-9, cg_max_iter=5000, system=system, return_stats=True)
        outs[system] = (U.cpu().numpy().astype(np.float64), st)
    (Uf, sf), (Us, ss) = outs["full"], outs["schur"]
    assert np.abs((Uf - Uf.mean()) - (Us - Us.mean())).max() < 2e-3
    np.testing.assert_allclose(ss["l1_obj"], sf["l1_obj"], rtol=1e-4)


def test_schur_2048_first_outer_matches_oracle(irls):
    """2048 x 2048 coherence-weighted workload, split-bf16 (folded) preconditioner: one outer step
    of 4 CG iterations element by element (bound of the truncated-run tests: 4 x 5e-5 x max|U|)."""
    d = synthetic.config_2048(seed=10)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=1, cg_tol=1e-6, cg_max=4, system="schur")
    ref = O.irls_unwrap(d["X"], d["coherence"], **kw)
    U, st = irls.unwrap(cuda(d["X"]), cuda(d["coherence"]), eps=1e-3, outer_iters=1,
                        cg_tol=1e-6, cg_max_iter=4, precision="bf16x3", system="schur",
                        return_stats=True)
    assert st["cg_iters"] == [4]
    atol = max(1e-3, 4 * 5e-5 * np.abs(ref["U"]).max())
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         atol=atol, ref=ref)


def test_schur_rejected_where_unsupported(irls):
    with pytest.raises(irls.IrlsError) as e:
        irls.Batch([(64, 64)], system="schur")
    assert e.value.code == -8
    from paper_2401_09961_gb300.autograd import unwrap_record
    X = cuda(synthetic.config_small(1, H=32, W=32)["X"])
    with irls.Plan(32, 32, system="schur") as p:
        with pytest.raises(irls.IrlsError) as e:
            unwrap_record(p, X, None)
        assert e.value.code == -8
