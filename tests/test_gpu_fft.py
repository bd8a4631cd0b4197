"""The fast-transform form of the Sec. 3.3 Laplacian block (IRLS_DCT_FFT: every orthonormal
DCT-II / DCT-III of the map through a float32 complex FFT of the same length, r_U^T z_U from the
spectrum) against the FP64 oracle, through the C ABI.

Bars as for the float32 dense form: the preconditioner within 2e-5 of its largest output (its
rounding is a few float32 ulps times log2 of the length per coefficient, amplified like any
error by tau / (l_i + m_j) at the lowest frequencies, which carry the largest outputs), and
unwraps at the acceptance bars of the method (assert_unwrap_parity)."""
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


def dense_reference(R, tau):
    H, W = R.shape
    return O.precond_apply((R.astype(np.float64), np.zeros((H - 1, W)), np.zeros((H, W - 1))),
                           np.zeros((H - 1, W)), np.zeros((H, W - 1)), tau, O.dct_basis(H),
                           O.dct_basis(W))[0]


@pytest.mark.parametrize("H,W", [(64, 64), (64, 128), (128, 64), (256, 256), (512, 1024),
                                 (1024, 512), (2048, 256), (256, 2048)])
def test_fft_precond_matches_oracle(irls, H, W):
    """Every row and column length of the form (64 ... 2048) against the oracle's dense
    products in FP64."""
    rng = np.random.default_rng(H * 7 + W)
    R = rng.standard_normal((H, W)).astype(np.float32)
    tau = 1e-2
    with irls.Plan(H, W, tau=tau, precision="fp32", dct_form="fft") as plan:
        assert plan.dct_form_name == "fft"
        Z = irls.precond_laplacian(plan, cuda(R)).cpu().numpy().astype(np.float64)
        Z2 = irls.precond_laplacian(plan, cuda(R)).cpu().numpy().astype(np.float64)
    z_ref = dense_reference(R, tau)
    scale = np.abs(z_ref).max()
    rel2 = np.linalg.norm(Z - z_ref) / np.linalg.norm(z_ref)
    assert np.abs(Z - z_ref).max() <= 2e-5 * scale and rel2 <= 1e-5, rel2
    assert np.array_equal(Z, Z2)


@pytest.mark.parametrize("H,W", [(4096, 4096), (8192, 64), (64, 16384), (8192, 1024),
                                 (1024, 16384)])
def test_fft_precond_large(irls, H, W):
    """The benchmarked size and the extreme lengths (8192 columns, 16384 rows) against the
    float64 DCT reference of scipy (pinned to the oracle's dense products in
    tests/test_gpu_parity.py)."""
    from test_gpu_parity import precond_reference_fft
    R = np.random.default_rng(H + 3 * W).standard_normal((H, W)).astype(np.float32)
    with irls.Plan(H, W, tau=1e-2, precision="fp32", dct_form="fft") as plan:
        Z = irls.precond_laplacian(plan, cuda(R)).cpu().numpy().astype(np.float64)
    z_ref = precond_reference_fft(R, 1e-2)
    rel2 = np.linalg.norm(Z - z_ref) / np.linalg.norm(z_ref)
    assert np.abs(Z - z_ref).max() <= 2e-5 * np.abs(z_ref).max() and rel2 <= 1e-5, rel2


@pytest.mark.parametrize("H,W", [(4000, 2000), (2000, 4000), (8000, 64), (64, 16000),
                                 (4000, 16000)])
def test_fft_precond_composite_lengths(irls, H, W):
    """The lengths 2^a 5^3 (2000, 4000, 8000, 16000: radix-5 stages after the radix-2^k ones),
    the sides of the paper's 4000 x M images, against the float64 DCT reference."""
    from test_gpu_parity import precond_reference_fft
    R = np.random.default_rng(H + 5 * W).standard_normal((H, W)).astype(np.float32)
    with irls.Plan(H, W, tau=1e-2, precision="fp32", dct_form="fft") as plan:
        assert plan.dct_form_name == "fft"
        Z = irls.precond_laplacian(plan, cuda(R)).cpu().numpy().astype(np.float64)
    z_ref = precond_reference_fft(R, 1e-2)
    rel2 = np.linalg.norm(Z - z_ref) / np.linalg.norm(z_ref)
    assert np.abs(Z - z_ref).max() <= 2e-5 * np.abs(z_ref).max() and rel2 <= 1e-5, rel2


def test_fft_unwrap_4000x2000_first_outer_matches_oracle(irls):
    """4000 x 2000 (composite lengths), one outer step truncated at 4 CG iterations, element by
    element against the oracle (the form's relative error, about 1e-6, is far inside 1e-3)."""
    from test_gpu_parity import assert_unwrap_parity
    d = synthetic.config_4096_mixed(seed=40, H=4000, W=2000)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=1, cg_tol=1e-6, cg_max=4)
    ref = O.irls_unwrap(d["X"], d["coherence"], **kw)
    with irls.Plan(4000, 2000, precision="fp32", dct_form="fft", tau=1e-2, delta=1e-3,
                   outer_iters=1, cg_tol=1e-6, cg_max_iter=4) as p:
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["cg_iters"] == [4]
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         atol=1e-3, ref=ref, case="4000x2000 fp32 (fft) 1 step x 4 CG",
                         truncated=True)


def test_fft_form_only_where_allowed(irls):
    """Power-of-two sides in range (and the compiled-in 2^a 5^3 lengths) and float32 only;
    batches do not take it."""
    for H, W in ((100, 128), (128, 100), (32, 64), (16384, 64), (64, 32768), (3000, 2000),
                 (16000, 64)):
        with pytest.raises(irls.IrlsError):
            irls.Plan(H, W, precision="fp32", dct_form="fft")
    with pytest.raises(irls.IrlsError):
        irls.Plan(256, 256, precision="bf16x3", dct_form="fft")
    with pytest.raises(irls.IrlsError):
        irls.Batch([(256, 256), (128, 256)], precision="fp32", dct_form="fft")
    with irls.Plan(256, 512, precision="fp32") as p:
        assert p.dct_form_name == "simt"
        p.set_opts(dct_form="fft")
        assert p.dct_form_name == "fft"
        p.set_opts(dct_form="auto")
        assert p.dct_form_name == "simt"


@pytest.mark.parametrize("law,H,W,seed,outer", [("coherence", 256, 512, 5, 6),
                                                ("mixed", 128, 64, 12, 4),
                                                ("mixed", 256, 256, 12, 4)])
def test_fft_unwrap_determined_matches_oracle(irls, law, H, W, seed, outer):
    """Full unwraps solved to cg_tol 1e-8 (the determined trajectory) at the strict bars."""
    from test_gpu_parity import assert_history, assert_unwrap_parity, determined_reference
    d, ref = determined_reference(law, H, W, seed, outer)
    with irls.Plan(H, W, precision="fp32", dct_form="fft", tau=1e-2, delta=1e-3,
                   outer_iters=outer, cg_tol=1e-8, cg_max_iter=3000) as p:
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["return_code"] == 0
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         ref=ref, strict=True,
                         case=f"{H}x{W} {law}-law fp32 (fft) tol 1e-8")
    assert_history(st, ref, l1=(law == "mixed"))


def test_fft_unwrap_4096_first_outer_step_matches_oracle(irls):
    """The 4096 x 4096 benchmark input, one outer step truncated at 4 CG iterations, element by
    element against the oracle: the form's own relative error (about 1e-6) reaches U about once
    per iteration, far inside 1e-3 rad."""
    from test_gpu_parity import assert_unwrap_parity
    d = synthetic.config_4096_mixed(seed=20, H=4096, W=4096)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=1, cg_tol=1e-6, cg_max=4)
    ref = O.irls_unwrap(d["X"], d["coherence"], **kw)
    with irls.Plan(4096, 4096, precision="fp32", dct_form="fft", tau=1e-2, delta=1e-3,
                   outer_iters=1, cg_tol=1e-6, cg_max_iter=4) as p:
        p.autotune()
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["cg_iters"] == [4]
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         atol=1e-3, ref=ref, case="4096x4096 bench input fp32 (fft) 1 step x 4 CG",
                         truncated=True)


def test_fft_u_only_system_matches_oracle(irls):
    """The U-only (Schur) system with the fast-transform preconditioner, determined solve."""
    from test_gpu_parity import assert_unwrap_parity
    d = synthetic.config_4096_mixed(seed=12, H=256, W=256)
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-8, cg_max=3000)
    ref = O.irls_unwrap(d["X"], d["coherence"], system="schur", **kw)
    with irls.Plan(256, 256, precision="fp32", dct_form="fft", system="schur", tau=1e-2,
                   delta=1e-3, outer_iters=4, cg_tol=1e-8, cg_max_iter=3000) as p:
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["return_code"] == 0
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         ref=ref, strict=True, case="256x256 mixed-law U-only fp32 (fft) tol 1e-8")


def test_fft_adjoint_matches_oracle_adjoint(irls):
    """The adjoint's solves through the fast-transform preconditioner, 128 x 128 image of the
    1024 x 1024 adjoint workload's law, 4 outer steps."""
    from test_gpu_adjoint import assert_grads_match_oracle
    d = synthetic.config_adjoint_1024(seed=30, H=128, W=128)
    assert_grads_match_oracle(irls, d["X"], d["coherence"], d["phi_true"], "fp32", 4, 1e-7,
                              "law of the 1024^2 workload", dct_form="fft")


def test_fft_and_dense_float32_forms_reach_the_same_unwrap(irls):
    """1024 x 1024 mixed-law image, 20 outer steps at the benchmark's cg_tol 1e-6: the fast
    transforms and the float32 dense products are two roundings of one map, so the unwraps
    agree to the trajectory noise of float32 CG (L1 within 1e-5 relative, integer maps on
    99.9 % of the pixels) and take the same number of CG iterations within 2 %."""
    d = synthetic.config_4096_mixed(seed=21, H=1024, W=1024)
    out = {}
    for form in ("auto", "fft"):
        with irls.Plan(1024, 1024, precision="fp32", dct_form=form, tau=1e-2, delta=1e-3,
                       outer_iters=20, cg_tol=1e-6, cg_max_iter=1000) as p:
            U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
            out[form] = (U.cpu().numpy().astype(np.float64), st)
    (Ua, sa), (Uf, sf) = out["auto"], out["fft"]
    Gv, Gh = O.wrapped_gradients(d["X"])
    Cv, Ch = O.edge_weights(d["coherence"], 1024, 1024)
    la, lf = O.l1_objective(Ua, Gv, Gh, Cv, Ch), O.l1_objective(Uf, Gv, Gh, Cv, Ch)
    assert abs(la - lf) <= 1e-5 * la, (la, lf)
    from test_gpu_parity import k_agreement
    assert k_agreement(Uf, Ua, d["X"]) >= 0.999
    assert abs(sa["cg_total"] - sf["cg_total"]) <= 0.02 * sa["cg_total"], (sa["cg_total"],
                                                                            sf["cg_total"])


def test_fft_paper_schedule_matches_oracle(irls):
    """The CG budget and IRLS stop of Sec. 4.3 with the fast-transform preconditioner: the same
    caps and stop as the oracle (whose Delta values sit at least 4.5e-4 from eps_tol on this
    image), and U within the measured spread of valid executions (preconditioner output rounded
    at 5e-7 relative, the form's measured rounding)."""
    from test_gpu_parity import assert_unwrap_parity, parity_atol
    from test_gpu_schedule import check_rule, schedule_envelope
    d = synthetic.config_2048(seed=29, H=128, W=64)
    kw = dict(tau=1e-2, delta=0.05, outer_iters=60, cg_tol=1e-8, cg_max=1000,
              cg_schedule="paper")
    ref, env = schedule_envelope(d["X"], d["coherence"], kw, 5e-7)
    assert ref["schedule_stop"] and max(ref["cg_cap"]) > 5
    assert all(abs(x - 1e-3) > 2e-5 for x in ref["delta_rel"])
    with irls.Plan(128, 64, precision="fp32", dct_form="fft", tau=1e-2, delta=0.05,
                   outer_iters=60, cg_tol=1e-8, cg_schedule="paper") as p:
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["cg_cap"] == ref["cg_cap"] and st["schedule_stop"] == ref["schedule_stop"]
    check_rule(st)
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         atol=parity_atol(env), ref=ref, env=env,
                         case="128x64 Sec. 4.3 CG schedule fp32 (fft)")


def test_fft_flexible_ratio_matches_oracle(irls):
    """The Polak-Ribiere ratio with the fast-transform preconditioner, on the determined
    trajectory (cg_tol 1e-8), at the strict bars."""
    from test_gpu_parity import assert_unwrap_parity, determined_reference
    d, ref = determined_reference("mixed", 256, 256, 12, 4)
    with irls.Plan(256, 256, precision="fp32", dct_form="fft", flexible_cg=1, tau=1e-2,
                   delta=1e-3, outer_iters=4, cg_tol=1e-8, cg_max_iter=3000) as p:
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["return_code"] == 0
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         ref=ref, strict=True, case="256x256 mixed-law fp32 (fft, flexible) tol 1e-8")


@pytest.mark.parametrize("H,W", [(8192, 8192), (4000, 16000)])
def test_fft_large_solve_invariants(irls, H, W):
    """The largest column length (8192) and the composite 4000 x 16000 in a full solve of three
    outer steps: the monotone quantities of Sec. 3.1 hold on the device statistics, U has zero
    mean, the solve reports no error, and the L1 objective falls."""
    d = synthetic.config_4096_mixed(seed=43, H=H, W=W)
    with irls.Plan(H, W, precision="fp32", dct_form="fft", delta=1e-3, outer_iters=3,
                   cg_tol=1e-6) as p:
        assert p.dct_form_name == "fft"
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert st["return_code"] in (0, 1)
    f, h = st["f_delta"], st["h_delta"]
    for k in range(len(h)):
        assert h[k] <= f[k] * (1 + 1e-5)
        if k + 1 < len(f):
            assert f[k + 1] <= h[k] * (1 + 1e-5)
    assert st["l1_obj"][-1] < st["l1_obj"][0]
    assert abs(float(U.double().mean())) < 1e-3
