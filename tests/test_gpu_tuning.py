"""Stencil tile shapes of the CG kernels: settable, autotuned, cached, and the solve stays at
parity with the oracle whatever the shape (only the reductions' summation order changes)."""
import numpy as np
import pytest

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


KW = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-6, cg_max=1000)
OPTS = dict(tau=1e-2, delta=1e-3, outer_iters=4, cg_tol=1e-6, cg_max_iter=1000)


def test_set_get_and_invalid_rows(irls):
    with irls.Plan(64, 96, **OPTS) as p:
        assert p.tiles == (24, 32)
        p.set_tiles(8, 16)
        assert p.tiles == (8, 16)
        p.set_tiles(0, 24)                  # 0 keeps the direction kernel's value
        assert p.tiles == (8, 24)
        for bad in [(7, 8), (8, 65), (-8, 8), (100, 8)]:
            with pytest.raises(irls.IrlsError) as e:
                p.set_tiles(*bad)
            assert e.value.code == -1
        assert p.tiles == (8, 24)
        p.set_tiles(22, 27)                 # any count from 8 to 64 for a plan
        assert p.tiles == (22, 27)


_REF = {}


def ragged_case():
    if not _REF:
        d = synthetic.config_2048(seed=77, H=203, W=613)
        _REF["d"] = d
        _REF["ref"] = oracle_with_envelope(d["X"], d["coherence"], KW)
    return _REF["d"], _REF["ref"][0], _REF["ref"][1]


@pytest.mark.parametrize("tiles", [(8, 8), (16, 24), (32, 16), (22, 27), (13, 50)])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_unwrap_parity_any_tile_shape(irls, tiles, prec):
    """Ragged shapes (rows not a multiple of any tile height, several column blocks)."""
    d, ref, env = ragged_case()
    with irls.Plan(203, 613, precision=prec, **OPTS) as p:
        p.set_tiles(*tiles)
        U, st = p.unwrap(cuda(d["X"]), cuda(d["coherence"]))
    assert_unwrap_parity(U.cpu().numpy(), ref["U"], st["l1_obj"][-1], ref["l1_obj"][-1], d["X"],
                         atol=parity_atol(env), ref=ref, env=env,
                         case=f"203x613 coherence {prec} tiles {tiles} tol 1e-6")


def test_tile_shape_changes_rounding_only(irls):
    """A shape is repeatable bit for bit; across shapes only rounding moves (CG totals within a
    few per cent, U within a loose bound: the oracle parity bar is the test above)."""
    d = synthetic.config_2048(seed=78, H=512, W=512)
    X, C = cuda(d["X"]), cuda(d["coherence"])
    out = {}
    with irls.Plan(512, 512, precision="bf16x3", **OPTS) as p:
        for tiles in [(24, 32), (8, 8), (32, 24), (16, 16)]:
            p.set_tiles(*tiles)
            U, st = p.unwrap(X, C)
            out[tiles] = (U.clone(), st)
        p.set_tiles(8, 8)
        U2, _ = p.unwrap(X, C)
    assert torch.equal(U2, out[(8, 8)][0])
    U0, s0 = out[(24, 32)]
    scale = float(U0.abs().max())
    for tiles, (U, st) in out.items():
        assert abs(sum(st["cg_iters"]) - sum(s0["cg_iters"])) <= 0.05 * sum(s0["cg_iters"]), tiles
        assert float((U - U0).abs().max()) <= 1e-2 * scale, tiles


def test_autotune_and_cache(irls, tmp_path):
    cache = str(tmp_path / "tiles.json")
    d = synthetic.config_2048(seed=79, H=1024, W=768)
    X, C = cuda(d["X"]), cuda(d["coherence"])
    with irls.Plan(1024, 768, precision="bf16x3", **OPTS) as p:
        U_def, s_def = p.unwrap(X, C)
        r = p.autotune(cache=cache)
        assert not r["cached"] and r["tiles"] == p.tiles
        assert all(t in (8, 16, 24, 32) for t in r["tiles"])
        ms = r["ms"]
        assert len(ms) == 8 and all(m > 0 for m in ms)
        # the choice is the fastest of each kernel's timings
        rows = (8, 16, 24, 32)
        assert r["tiles"] == (rows[int(np.argmin(ms[:4]))], rows[int(np.argmin(ms[4:]))])
        U, st = p.unwrap(X, C)          # the plan solves as before after the timing runs
        assert float((U - U_def).abs().max()) <= 1e-2 * float(U_def.abs().max())
        p.set_tiles(24, 32)
        U3, _ = p.unwrap(X, C)          # and bit for bit as before with the default shapes
        assert torch.equal(U3, U_def)
    with irls.Plan(1024, 768, precision="bf16x3", **OPTS) as q:
        r2 = q.autotune(cache=cache)
        assert r2["cached"] and r2["ms"] is None and q.tiles == r["tiles"]


@pytest.mark.parametrize("form", ["auto", "direct"])
def test_batched_tiles_equal_single_plans(irls, form):
    """A batch run with non-default tile shapes equals single-image plans with the same shapes,
    bit for bit; changing the shapes between runs re-captures the CG graphs."""
    shapes = [(256, 256), (384, 512), (512, 256)]
    tiles = [synthetic.config_2048(seed=500 + t, H=h, W=w) for t, (h, w) in enumerate(shapes)]
    Xs = [cuda(d["X"]) for d in tiles]
    Cs = [cuda(d["coherence"]) for d in tiles]
    opts = dict(OPTS, dct_form=form)
    with irls.Batch(shapes, precision="bf16x3", **opts) as b:
        assert b.tiles == (24, 32)
        Ud, _ = b.unwrap(Xs, Cs)
        Ud = [u.clone() for u in Ud]
        b.set_tiles(8, 16)
        assert b.tiles == (8, 16)
        Us, st = b.unwrap(Xs, Cs)
        assert b.uses_graphs
        Us = [u.clone() for u in Us]
        with pytest.raises(irls.IrlsError):
            b.set_tiles(10, 16)
    for t, (h, w) in enumerate(shapes):
        with irls.Plan(h, w, precision="bf16x3", **opts) as p:
            p.set_tiles(8, 16)
            U, s1 = p.unwrap(Xs[t], Cs[t])
            p.set_tiles(24, 32)
            U0, _ = p.unwrap(Xs[t], Cs[t])
        assert torch.equal(Us[t], U), t
        assert st[t]["cg_iters"] == s1["cg_iters"], t
        assert torch.equal(Ud[t], U0), t


def test_batched_autotune_and_cache(irls, tmp_path):
    cache = str(tmp_path / "tiles.json")
    tiles = synthetic.batched_tiles(n=8)
    shapes = [d["X"].shape for d in tiles]
    Xs = [cuda(d["X"]) for d in tiles]
    Cs = [cuda(d["coherence"]) for d in tiles]
    with irls.Batch(shapes, precision="bf16x3", **OPTS) as b:
        r = b.autotune(cache=cache)
        assert not r["cached"] and len(r["ms"]) == 8 and all(m > 0 for m in r["ms"])
        rows = (8, 16, 24, 32)
        assert r["tiles"] == (rows[int(np.argmin(r["ms"][:4]))], rows[int(np.argmin(r["ms"][4:]))])
        Us, st = b.unwrap(Xs, Cs)
        assert all(s["outer_done"] == 4 for s in st)
    for t in (0, 5):
        h, w = shapes[t]
        with irls.Plan(h, w, precision="bf16x3", **OPTS) as p:
            p.set_tiles(*r["tiles"])
            U, _ = p.unwrap(Xs[t], Cs[t])
        assert torch.equal(Us[t], U), t
    with irls.Batch(shapes, precision="bf16x3", **OPTS) as b2:
        r2 = b2.autotune(cache=cache)
        assert r2["cached"] and b2.tiles == r["tiles"]
