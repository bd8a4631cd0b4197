"""The hand-written adjoint (irls_unwrap_forward_record / irls_unwrap_backward) against the FP64
oracle's adjoint and against central differences of the GPU forward map."""
import numpy as np
import pytest

from oracle import irls as O
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


def gpu_grads(irls, X, coh, dLdU, prec="fp32", **kw):
    from paper_2401_09961_gb300.autograd import unwrap_record, unwrap_backward
    H, W = X.shape
    with irls.Plan(H, W, precision=prec, **kw) as plan:
        U, tape, _ = unwrap_record(plan, cuda(X), cuda(coh))
        dX, dc, st = unwrap_backward(tape, cuda(dLdU(U.cpu().numpy().astype(np.float64))))
        tape.free()
        return U.cpu().numpy(), dX.cpu().numpy(), dc.cpu().numpy(), st


def oracle_grads(X, coh, dLdU, storage=None, **kw):
    fwd = O.irls_unwrap(X, coh, record=True, storage=storage, **kw)
    gX, gC, _ = O.irls_adjoint(X, coh, dLdU(fwd["U"]), fwd=fwd, storage=storage, **kw)
    return fwd["U"], gX, gC


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_adjoint_matches_oracle_adjoint(irls, prec):
    """48 x 40 image of the 1024 x 1024 adjoint workload's law, 4 outer steps."""
    d = synthetic.config_adjoint_1024(seed=30, H=48, W=40)
    assert_grads_match_oracle(irls, d["X"], d["coherence"], d["phi_true"], prec, 4, 1e-7,
                              "law of the 1024^2 workload")


def assert_grads_match_oracle(irls, X, coh, Uref, prec, outer, cg_tol, case, **plan_kw):
    """GPU adjoint (dL/dX, dL/dcoherence of L = sum (U - mean U - U_ref)^2) against the FP64
    oracle adjoint, both from their own forward runs.  Bar: max(2e-3 of the largest gradient,
    2 x the spread between the FP64 oracle and the same oracle with float32 vector storage)."""
    import parity_log
    dLdU = lambda U: 2.0 * (U - U.mean() - Uref)  # noqa: E731
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=outer, cg_tol=cg_tol, cg_max=3000)
    _, gX, gC = oracle_grads(X, coh, dLdU, **kw)
    _, gX32, gC32 = oracle_grads(X, coh, dLdU, storage=np.float32, **kw)
    H, W = X.shape
    with irls.Plan(H, W, precision=prec, tau=1e-2, delta=1e-3, outer_iters=outer,
                   cg_tol=cg_tol, cg_max_iter=3000, **plan_kw) as p:
        form = p.dct_form_name
    U, dX, dc, st = gpu_grads(irls, X, coh, dLdU, prec=prec, tau=1e-2, delta=1e-3,
                              outer_iters=outer, cg_tol=cg_tol, cg_max_iter=3000, **plan_kw)
    assert st["outer_done"] == outer and np.all(np.isfinite(dX)) and np.all(np.isfinite(dc))
    for name, g, r, r32 in (("dL/dX", dX, gX, gX32), ("dL/dcoh", dc, gC, gC32)):
        env = np.abs(r32 - r).max()
        tol = max(2e-3 * np.abs(r).max(), 2.0 * env)
        err = np.abs(g - r).max()
        parity_log.record(case=f"adjoint {name} {H}x{W} {outer} steps {prec} ({form}) {case}",
                          err_u=err / np.abs(r).max(), atol=tol / np.abs(r).max(),
                          dl1_rel=float("nan"), l1_bar_rel=float("nan"), k_agree=float("nan"),
                          l1=float("nan"), bars=f"relative to max|grad| {np.abs(r).max():.3g}; "
                                                f"float32-storage spread {env / np.abs(r).max():.1e}")
        assert err <= tol, (name, err, tol, env)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_adjoint_256_matches_oracle_adjoint(irls, prec):
    """256 x 256 image of the 1024 x 1024 adjoint workload's law, 4 outer steps: the split-bf16
    plan runs the folded preconditioner (the form the 1024 x 1024 adjoint runs) in the forward
    solves and in the adjoint solves."""
    d = synthetic.config_adjoint_1024(seed=30, H=256, W=256)
    assert_grads_match_oracle(irls, d["X"], d["coherence"], d["phi_true"], prec, 4, 1e-7,
                              "law of the 1024^2 workload")


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_adjoint_128_crop_of_1024_workload(irls, prec):
    """The 128 x 128 crop (top-left corner) of the 1024 x 1024 adjoint workload, with its 15
    outer steps, against the FP64 oracle adjoint of the same crop."""
    d = synthetic.config_adjoint_1024(seed=30)
    X = np.ascontiguousarray(d["X"][:128, :128])
    coh = np.ascontiguousarray(d["coherence"][:128, :128])
    Uref = d["phi_true"][:128, :128]
    assert_grads_match_oracle(irls, X, coh, Uref - Uref.mean(), prec, 15, 1e-7,
                              "crop of the 1024^2 workload")


def test_adjoint_matches_gpu_central_differences(irls):
    """Central differences of the GPU forward map itself.  A residue-rich image (noise 1 rad) with
    delta = 0.05 so that the coherence gradient is not negligible (on well-unwrapped images
    D-bar = -lambda_V o V ~ 0) and the map is smooth at the step size; X steps of 2e-2 (float32
    X), coherence steps of 1e-2, pixels whose incident wrapped differences stay below pi - 0.1.
    Differences of a float32 forward resolve about 1 % of the largest gradient, hence the bar."""
    d = synthetic.make_phase(40, 36, 7, ramp=10.0, n_bumps=1, noise=1.0, coherence=True)
    X, coh = d["X"], d["coherence"]
    Uref = d["phi_true"]
    kw = dict(tau=1e-2, delta=0.05, outer_iters=3, cg_tol=1e-7, cg_max_iter=3000)
    H, W = X.shape
    with irls.Plan(H, W, **kw) as plan:
        def L(Xa, ca):
            U, _ = plan.unwrap(cuda(Xa), cuda(ca))
            U = U.cpu().numpy().astype(np.float64)
            return float(np.sum((U - U.mean() - Uref) ** 2))

        from paper_2401_09961_gb300.autograd import unwrap_record, unwrap_backward
        U, tape, _ = unwrap_record(plan, cuda(X), cuda(coh))
        Ud = U.cpu().numpy().astype(np.float64)
        dX, dc, _ = unwrap_backward(tape, cuda(2.0 * (Ud - Ud.mean() - Uref)))
        tape.free()
        dX, dc = dX.cpu().numpy(), dc.cpu().numpy()
        Gv, Gh = O.wrapped_gradients(X)
        rng = np.random.default_rng(3)
        pts = [tuple(p) for p in rng.integers(1, min(H, W) - 1, size=(40, 2))]
        n = 0
        sx, sc = np.abs(dX).max(), np.abs(dc).max()
        for i, j in pts:
            inc = max(abs(Gv[i - 1, j]), abs(Gv[i, j]), abs(Gh[i, j - 1]), abs(Gh[i, j]))
            if inc >= np.pi - 0.1:
                continue
            h = 2e-2
            Xp, Xm = X.copy(), X.copy()
            Xp[i, j] += h
            Xm[i, j] -= h
            fd = (L(Xp, coh) - L(Xm, coh)) / (2 * h)
            hc = 1e-2
            cp, cm = coh.copy(), coh.copy()
            cp[i, j] += hc
            cm[i, j] -= hc
            fdc = (L(X, cp) - L(X, cm)) / (2 * hc)
            assert abs(fd - dX[i, j]) <= 2e-2 * sx, (i, j, fd, dX[i, j], sx)
            assert abs(fdc - dc[i, j]) <= 2e-2 * sc, (i, j, fdc, dc[i, j], sc)
            n += 1
            if n >= 8:
                break
        assert n >= 4


def test_autograd_function(irls):
    d = synthetic.config_adjoint_1024(seed=32, H=32, W=40)
    X = cuda(d["X"]).requires_grad_(True)
    C = cuda(d["coherence"]).requires_grad_(True)
    Uref = cuda(d["phi_true"])
    with irls.Plan(32, 40, tau=1e-2, delta=1e-3, outer_iters=3, cg_tol=1e-6) as plan:
        U = irls.unwrap_differentiable(X, C, plan)
        loss = ((U - U.mean() - Uref) ** 2).sum()
        loss.backward()
        from paper_2401_09961_gb300.autograd import unwrap_record, unwrap_backward
        U2, tape, _ = unwrap_record(plan, X.detach(), C.detach())
        dX, dc, _ = unwrap_backward(tape, (2.0 * (U2 - U2.mean() - Uref)).contiguous())
        tape.free()
    # the autograd graph forms dL/dU with torch's own float32 ops (U - mean(U) differentiated),
    # so the adjoint solves start from a right-hand side rounded differently
    assert float((X.grad - dX).abs().max()) <= 1e-3 * float(dX.abs().max())
    assert float((C.grad - dc).abs().max()) <= 1e-3 * float(dc.abs().max()) + 1e-9


def test_adjoint_1024_workload(irls):
    """The 1024 x 1024 adjoint workload (15 outer steps, split-bf16 folded preconditioner)
    against central differences of the GPU forward itself, with solves tight enough (cg_tol
    1e-8) that the forward map is the converged-solve map the adjoint differentiates:
      * dL/dX at 32 random pixels whose incident wrapped differences stay below pi - 0.1, step
        h = 0.05 (X is float32: at h = 1e-3 the difference of two forwards over 1M pixels is
        rounding noise, about 0.5 in the quotient; at 0.05 the quotient agrees with the adjoint
        to ~0.3 % of the largest gradient), bar 2 % of max |dL/dX|;
      * dL/dcoherence along the direction v = sign(dL/dcoh) on the pixels where |dL/dcoh| is
        above 1 % of its maximum (elsewhere the coherence gradient is below the forward's noise),
        step 0.03: (L(c + h v) - L(c - h v)) / 2h against sum v dL/dcoh within 5 %;
      * dL/dX sums to zero (the loss is invariant to a constant added to X)."""
    import parity_log
    from paper_2401_09961_gb300.autograd import unwrap_record, unwrap_backward
    d = synthetic.config_adjoint_1024(seed=30)
    X, coh, Uref = d["X"], d["coherence"], d["phi_true"]
    H, W = X.shape
    with irls.Plan(H, W, precision="bf16x3", tau=1e-2, delta=1e-3, outer_iters=15, cg_tol=1e-8,
                   cg_max_iter=3000) as plan:
        assert plan.folded
        U, tape, st = unwrap_record(plan, cuda(X), cuda(coh))
        Ud = U.cpu().numpy().astype(np.float64)
        dX, dc, sb = unwrap_backward(tape, cuda(2.0 * (Ud - Ud.mean() - Uref)))
        tape.free()
        dX, dc = dX.cpu().numpy().astype(np.float64), dc.cpu().numpy().astype(np.float64)
        assert st["outer_done"] == 15 and sb["outer_done"] == 15
        assert np.all(np.isfinite(dX)) and np.all(np.isfinite(dc))
        assert abs(dX.sum()) <= 1e-4 * np.abs(dX).sum()

        def L(Xa, ca):
            Ua, _ = plan.unwrap(cuda(Xa), cuda(ca))
            Ua = Ua.cpu().numpy().astype(np.float64)
            return float(np.sum((Ua - Ua.mean() - Uref) ** 2))

        Gv, Gh = O.wrapped_gradients(X)
        rng = np.random.default_rng(5)
        pts = []
        while len(pts) < 32:
            i, j = (int(v) for v in rng.integers(1, H - 1, size=2))
            if max(abs(Gv[i - 1, j]), abs(Gv[i, j]), abs(Gh[i, j - 1]), abs(Gh[i, j])) < np.pi - 0.1:
                pts.append((i, j))
        h = 0.05
        sx = np.abs(dX).max()
        worst = 0.0
        for i, j in pts:
            Xp, Xm = X.copy(), X.copy()
            Xp[i, j] += h
            Xm[i, j] -= h
            fd = (L(Xp, coh) - L(Xm, coh)) / (2 * h)
            worst = max(worst, abs(fd - dX[i, j]) / sx)
        v = np.where(np.abs(dc) > 0.01 * np.abs(dc).max(), np.sign(dc), 0.0)
        pred = float(np.sum(v * dc))
        hc = 0.03
        fdc = (L(X, coh + hc * v) - L(X, coh - hc * v)) / (2 * hc)
    parity_log.record(case="adjoint 1024x1024 15 steps bf16x3 (folded) vs GPU central differences",
                      err_u=worst, atol=2e-2, dl1_rel=float("nan"), l1_bar_rel=float("nan"),
                      k_agree=float("nan"), l1=float("nan"),
                      bars=f"dL/dX: 32 pixels, h {h}, max err / max|grad|; dL/dcoh along "
                           f"sign(grad) on {int(np.abs(v).sum())} pixels: FD {fdc:.4g} vs "
                           f"adjoint {pred:.4g} ({abs(fdc - pred) / abs(pred):.1%})")
    assert worst <= 2e-2, worst
    assert abs(fdc - pred) <= 0.05 * abs(pred), (fdc, pred)
