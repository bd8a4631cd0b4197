"""The batched form (one launch per phase over many images of uneven sizes) against the
single-image path and the FP64 oracle."""
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


OPTS = dict(tau=1e-2, delta=1e-3, outer_iters=5, cg_tol=1e-6, cg_max_iter=1000)
# single-image plans in the grouped form's (direct) preconditioner, for bit-identical comparisons
DIRECT = dict(OPTS, dct_form="direct")


def test_batched_equals_single_image_path(irls):
    """Same kernels, same per-image block decomposition and reduction order: bit-identical."""
    shapes = [(128, 128), (256, 384), (384, 128), (200, 150), (128, 256), (96, 80)]
    tiles = [synthetic.config_2048(seed=100 + t, H=h, W=w) for t, (h, w) in enumerate(shapes)]
    Xs = [cuda(d["X"]) for d in tiles]
    Cs = [cuda(d["coherence"]) for d in tiles]
    with irls.Batch(shapes, precision="bf16x3", **OPTS) as b:
        Us, st = b.unwrap(Xs, Cs)
        Us = [u.clone() for u in Us]
        assert b.uses_graphs
        Us2, st2 = b.unwrap(Xs, Cs)   # a second call on the same batch (graph replay)
    for t, (h, w) in enumerate(shapes):
        with irls.Plan(h, w, precision="bf16x3", **DIRECT) as p:
            U, s1 = p.unwrap(Xs[t], Cs[t])
        assert torch.equal(Us[t], U), t
        assert torch.equal(Us2[t], U), t
        assert st[t]["cg_iters"] == s1["cg_iters"]
        assert st[t]["l1_obj"] == s1["l1_obj"]


def test_batched_per_image_convergence_masks(irls):
    """Images that converge at very different iteration counts (a constant image needs none)."""
    shapes = [(128, 128), (256, 256), (128, 384)]
    flat = np.full((128, 128), 0.5, dtype=np.float32)
    hard = synthetic.config_4096_mixed(seed=7, H=256, W=256)
    easy = synthetic.config_small(seed=3, H=128, W=384)
    Xs = [cuda(flat), cuda(hard["X"]), cuda(easy["X"])]
    Cs = [cuda(np.ones((128, 128), np.float32)), cuda(hard["coherence"]),
          cuda(np.ones((128, 384), np.float32))]
    with irls.Batch(shapes, precision="bf16x3", **OPTS) as b:
        Us, st = b.unwrap(Xs, Cs)
    assert st[0]["cg_iters"] == [0] * 5 and float(Us[0].abs().max()) == 0.0
    assert sum(st[1]["cg_iters"]) > 5 * sum(st[2]["cg_iters"])
    for t, (h, w) in enumerate(shapes):
        with irls.Plan(h, w, precision="bf16x3", **DIRECT) as p:
            U, s1 = p.unwrap(Xs[t], Cs[t])
        assert torch.equal(Us[t], U) and st[t]["cg_iters"] == s1["cg_iters"]


def test_batched_matches_oracle(irls):
    shapes = [(64, 96), (80, 64)]
    tiles = [synthetic.config_2048(seed=200 + t, H=h, W=w) for t, (h, w) in enumerate(shapes)]
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-6, cg_max=1000)
    with irls.Batch(shapes, precision="bf16x3", tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-6,
                    cg_max_iter=1000) as b:
        Us, st = b.unwrap([cuda(d["X"]) for d in tiles], [cuda(d["coherence"]) for d in tiles])
    for t, d in enumerate(tiles):
        ref, env = oracle_with_envelope(d["X"], d["coherence"], kw)
        assert_unwrap_parity(Us[t].cpu().numpy(), ref["U"], st[t]["l1_obj"][-1],
                             ref["l1_obj"][-1], d["X"], atol=parity_atol(env), ref=ref, env=env,
                             case=f"batch of 2, image {t} {d['X'].shape} bf16x3 (direct) tol 1e-6")


def test_batched_folded_form_only_where_every_image_allows_it(irls):
    """The folded form needs the split precision and sides >= 256 in every image."""
    for shapes, prec in (([(256, 256), (256, 250)], "bf16x3"), ([(256, 256), (255, 256)], "bf16x3"),
                         ([(256, 256)], "bf16")):
        with pytest.raises(irls.IrlsError) as e:
            irls.Batch(shapes, precision=prec, dct_form="folded", **OPTS)
        assert e.value.code == -8
    with irls.Batch([(256, 256), (256, 250)], precision="bf16x3", **OPTS) as b:
        assert not b.folded    # auto: direct, one image does not allow the fold
    with irls.Batch([(256, 256), (258, 512)], precision="bf16x3", **OPTS) as b:
        assert b.folded
    with irls.Batch([(256, 256)], precision="bf16x3", **DIRECT) as b:
        assert not b.folded


# sides >= 256: halves padded to multiples of 256 (129 -> 256, 150 -> 256, 384 -> 512), odd sides
# (middle row or column its own mirror), non-square, one side shared by several images, one
# shape twice
FOLD_SHAPES = [(256, 256), (258, 300), (512, 384), (384, 768), (256, 256), (1024, 512),
               (257, 301), (511, 256)]


def test_batched_folded_equals_single_image_path(irls):
    """Folded preconditioner over all images in one fused launch: per image the same tiles, the same
    per-tile r^T z slots and the same reduction order as a plan of its own, so bit-identical."""
    tiles = [synthetic.config_2048(seed=300 + t, H=h, W=w) for t, (h, w) in enumerate(FOLD_SHAPES)]
    Xs = [cuda(d["X"]) for d in tiles]
    Cs = [cuda(d["coherence"]) for d in tiles]
    with irls.Batch(FOLD_SHAPES, precision="bf16x3", **OPTS) as b:
        assert b.folded
        Us, st = b.unwrap(Xs, Cs)
        Us = [u.clone() for u in Us]
        Us2, st2 = b.unwrap(Xs, Cs)
    for t, (h, w) in enumerate(FOLD_SHAPES):
        with irls.Plan(h, w, precision="bf16x3", **OPTS) as p:
            assert p.folded
            U, s1 = p.unwrap(Xs[t], Cs[t])
        assert torch.equal(Us[t], U), t
        assert torch.equal(Us2[t], U), t
        assert st[t]["cg_iters"] == s1["cg_iters"] == st2[t]["cg_iters"], t
        assert st[t]["l1_obj"] == s1["l1_obj"], t


def test_batched_folded_per_image_masks(irls):
    """A constant image stops at once and an easy one early, while a hard one runs on: the
    stopped images' tiles drop out of the pair GEMMs and their fold."""
    shapes = [(256, 256), (512, 512), (256, 384)]
    flat = np.full((256, 256), 0.5, dtype=np.float32)
    hard = synthetic.config_4096_mixed(seed=8, H=512, W=512)
    easy = synthetic.config_small(seed=4, H=256, W=384)
    Xs = [cuda(flat), cuda(hard["X"]), cuda(easy["X"])]
    Cs = [cuda(np.ones((256, 256), np.float32)), cuda(hard["coherence"]),
          cuda(np.ones((256, 384), np.float32))]
    with irls.Batch(shapes, precision="bf16x3", **OPTS) as b:
        assert b.folded
        Us, st = b.unwrap(Xs, Cs)
    assert st[0]["cg_iters"] == [0] * 5 and float(Us[0].abs().max()) == 0.0
    assert sum(st[1]["cg_iters"]) > 3 * sum(st[2]["cg_iters"])
    for t, (h, w) in enumerate(shapes):
        with irls.Plan(h, w, precision="bf16x3", **OPTS) as p:
            U, s1 = p.unwrap(Xs[t], Cs[t])
        assert torch.equal(Us[t], U) and st[t]["cg_iters"] == s1["cg_iters"], t


def test_batched_folded_matches_oracle(irls):
    """The folded batched form (the 64-tile workload's form) on two images of the coherence law
    with solves tight enough (cg_tol 1e-8) that U is determined: no envelope, per-outer H_delta
    history too.  (At cg_tol 1e-6 the oracle's own U on the 256 x 320 image moves by 1.9e-3 rad
    between solves cut at 1e-6 and at 1e-8, so a truncated comparison would measure where a
    solve stops, not the batched form.)"""
    from test_gpu_parity import assert_history
    shapes = [(256, 256), (256, 320)]
    tiles = [synthetic.config_2048(seed=400 + t, H=h, W=w) for t, (h, w) in enumerate(shapes)]
    kw = dict(tau=1e-2, delta=1e-3, outer_iters=3, cg_tol=1e-8, cg_max=3000)
    with irls.Batch(shapes, precision="bf16x3", tau=1e-2, delta=1e-3, outer_iters=3, cg_tol=1e-8,
                    cg_max_iter=3000) as b:
        assert b.folded
        Us, st = b.unwrap([cuda(d["X"]) for d in tiles], [cuda(d["coherence"]) for d in tiles])
    for t, d in enumerate(tiles):
        ref = O.irls_unwrap(d["X"], d["coherence"], **kw)
        assert_unwrap_parity(Us[t].cpu().numpy(), ref["U"], st[t]["l1_obj"][-1],
                             ref["l1_obj"][-1], d["X"], ref=ref, strict=True,
                             case=f"batch of 2, image {t} {d['X'].shape} bf16x3 (folded) tol 1e-8")
        assert_history(st[t], ref, l1=False)


@pytest.mark.parametrize("form", ["auto", "direct"])
def test_batched_64_uneven_tiles(irls, form):
    """The 64-tile workload: sides drawn from {256, 384, ..., 1536}, one batch (folded where every
    image allows it, else direct); a few tiles are re-solved alone and must agree bit for bit."""
    tiles = synthetic.batched_tiles(n=64)
    shapes = [d["X"].shape for d in tiles]
    Xs = [cuda(d["X"]) for d in tiles]
    Cs = [cuda(d["coherence"]) for d in tiles]
    opts = dict(tau=1e-2, delta=1e-3, outer_iters=3, cg_tol=1e-6, cg_max_iter=1000, dct_form=form)
    with irls.Batch(shapes, precision="bf16x3", **opts) as b:
        assert b.folded == (form == "auto")
        Us, st = b.unwrap(Xs, Cs)
    assert all(s["outer_done"] == 3 for s in st)
    for t in (0, 17, 63):
        h, w = shapes[t]
        with irls.Plan(h, w, precision="bf16x3", **opts) as p:
            U, _ = p.unwrap(Xs[t], Cs[t])
        assert torch.equal(Us[t], U), t
