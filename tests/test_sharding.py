"""Splitting independent tiles across ranks (LPT greedy) and its agreement across gloo ranks.
Host arithmetic only; no GPU."""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_2401_09961_gb300 import sharding


def _brute_makespan(costs, m):
    """The optimal makespan by trying every assignment (tiny cases only)."""
    best = float("inf")
    for a in itertools.product(range(m), repeat=len(costs)):
        loads = [0.0] * m
        for c, p in zip(costs, a):
            loads[p] += c
        best = min(best, max(loads))
    return best


def test_every_index_once_and_deterministic():
    rng = np.random.default_rng(0)
    costs = rng.uniform(0, 10, 37).tolist()
    for m in (1, 2, 3, 5, 8, 40):
        parts = sharding.lpt_partition(costs, m)
        assert len(parts) == m
        assert sorted(i for p in parts for i in p) == list(range(37))
        assert all(p == sorted(p) for p in parts)
        assert parts == sharding.lpt_partition(list(costs), m)


def test_one_part_keeps_input_order_and_empty_input():
    assert sharding.lpt_partition([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
    assert sharding.lpt_partition([], 3) == [[], [], []]


def test_hand_worked_example():
    # sorted 7, 5, 4, 3, 2 (index order on ties) onto 2 parts:
    # 7 -> p0; 5 -> p1; 4 -> p1 (9); 3 -> p0 (10); 2 -> p1 (11)
    costs = [4.0, 7.0, 2.0, 5.0, 3.0]
    assert sharding.lpt_partition(costs, 2) == [[1, 4], [0, 2, 3]]
    # equal costs: part order follows index order, equal loads go to the lowest part
    assert sharding.lpt_partition([1.0] * 5, 2) == [[0, 2, 4], [1, 3]]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("m", (2, 3))
def test_graham_bound_against_brute_force(seed, m):
    costs = np.random.default_rng(seed).uniform(0.1, 10, 7).tolist()
    parts = sharding.lpt_partition(costs, m)
    lpt = max(sum(costs[i] for i in p) for p in parts)
    opt = _brute_makespan(costs, m)
    assert opt <= lpt <= (4 / 3 - 1 / (3 * m)) * opt + 1e-12


def test_bad_arguments():
    with pytest.raises(ValueError):
        sharding.lpt_partition([1.0], 0)
    with pytest.raises(ValueError):
        sharding.lpt_partition([1.0, float("nan")], 2)
    with pytest.raises(ValueError):
        sharding.lpt_partition([-1.0], 2)
    with pytest.raises(ValueError):
        sharding.shard_tiles([(8, 8)], 2, 2)
    with pytest.raises(ValueError):
        sharding.tile_cost(0, 5)


def test_tile_cost_model():
    # monotone in each side; the folded form halves the transform work at equal padded size
    assert sharding.tile_cost(512, 512) < sharding.tile_cost(512, 640) < sharding.tile_cost(640, 640)
    # a 256 side folds into halves of 128, padded to 256 like those of a 512 side: the two
    # differ by the stencil work alone
    d = sharding.tile_cost(512, 512) - sharding.tile_cost(256, 256)
    assert d == pytest.approx((512 * 512 - 256 * 256) * sharding._STENCIL_S_PER_PX)
    # at 4096 x 4096 the estimate is the calibration: 0.490 + 0.331 ms per CG iteration
    assert sharding.tile_cost(4096, 4096) == pytest.approx(0.821e-3)
    # odd sides pad their halves: 513 -> halves 257 and 256, padded to 512 -> 1024 a side, so
    # the transform part is 8 times that of 512 x 512
    def dct(n):
        return sharding.tile_cost(n, n) - n * n * sharding._STENCIL_S_PER_PX
    assert dct(513) == pytest.approx(8 * dct(512))


def test_benchmark_tiles_balance():
    """The 64 tiles per GPU of the batched benchmark: the estimated loads of the ranks agree
    within a few per cent, and the union of 64 N tiles is exactly the shards."""
    import synthetic
    for world in (1, 2, 4, 8):
        shapes = synthetic.batched_tile_shapes(n=64 * world, seed_base=1000)
        parts = [sharding.shard_tiles(shapes, r, world) for r in range(world)]
        assert sorted(i for p in parts for i in p) == list(range(64 * world))
        loads = sharding.part_loads(shapes, parts)
        assert max(loads) <= 1.03 * (sum(loads) / world)
    assert sharding.shard_tiles(synthetic.batched_tile_shapes(64, 1000), 0, 1) == list(range(64))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synthetic
        shapes = synthetic.batched_tile_shapes(n=64 * world, seed_base=1000)
        mine = sharding.shard_tiles(shapes, rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        out.put((rank, mine, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_without_exchange():
    """Each rank derives its share on its own; gathered afterwards, the shares are disjoint,
    cover every tile and equal what each rank would compute for the other."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    (_, m0, g0), (_, m1, g1) = res
    assert g0 == g1 == [m0, m1]
    assert not set(m0) & set(m1) and sorted(m0 + m1) == list(range(128))
    import synthetic
    shapes = synthetic.batched_tile_shapes(n=128, seed_base=1000)
    assert [m0, m1] == sharding.lpt_partition([sharding.tile_cost(*s) for s in shapes], 2)


class FakeBatch:
    """Stands in for the GPU batch: records what it was given and returns X + 1 as U."""
    made = []

    def __init__(self, shapes, **opts):
        self.shapes, self.opts, self.closed = list(shapes), opts, False
        FakeBatch.made.append(self)

    def unwrap(self, Xs, cohs=None):
        assert [tuple(X.shape) for X in Xs] == self.shapes
        assert all(X.dtype.is_floating_point and X.is_contiguous() for X in Xs)
        self.cohs = cohs
        return [X + 1 for X in Xs], [{"cg_total": int(X.numel())} for X in Xs]

    def close(self):
        self.closed = True


def _images(n=9, seed=0):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.integers(256, 700)), int(rng.integers(256, 700))) for _ in range(n)]
    return [torch.full(s, float(i), dtype=torch.float64) for i, s in enumerate(shapes)]


def test_unwrap_sharded_takes_this_ranks_share():
    Xs = _images()
    cohs = [X * 0 + 0.5 for X in Xs]
    got = {}
    for r in range(3):
        FakeBatch.made.clear()
        idx, Us, st = sharding.unwrap_sharded(Xs, cohs, rank=r, world=3, device="cpu",
                                              batch=FakeBatch, precision="bf16x3")
        assert idx == sharding.shard_tiles([tuple(X.shape) for X in Xs], r, 3)
        b, = FakeBatch.made
        assert b.closed and b.opts == {"precision": "bf16x3"} and len(b.cohs) == len(idx)
        for i, U in zip(idx, Us):
            assert U.dtype.is_floating_point and float(U[0, 0]) == i + 1
            got[i] = U
        assert [s["cg_total"] for s in st] == [Xs[i].numel() for i in idx]
    assert sorted(got) == list(range(len(Xs)))


def test_unwrap_sharded_edges():
    Xs = _images(2)
    idx, Us, st = sharding.unwrap_sharded(Xs, rank=3, world=4, device="cpu", batch=FakeBatch)
    assert (idx, Us, st) == ([], [], [])
    with pytest.raises(ValueError):
        sharding.unwrap_sharded(Xs, [Xs[0]], rank=0, world=1, device="cpu", batch=FakeBatch)
    with pytest.raises(ValueError):
        sharding.unwrap_sharded([Xs[0][0]], rank=0, world=1, device="cpu", batch=FakeBatch)
    # no process group: the whole list on one rank
    idx, _, _ = sharding.unwrap_sharded(Xs, device="cpu", batch=FakeBatch)
    assert idx == [0, 1]


def _unwrap_rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Xs = _images(11, seed=5)
        idx, Us, _ = sharding.unwrap_sharded(Xs, device="cpu", batch=FakeBatch)
        vals = [float(U[0, 0]) for U in Us]
        out.put((rank, idx, vals))
    finally:
        dist.destroy_process_group()


def test_unwrap_sharded_under_two_gloo_ranks():
    """rank and world come from the process group; the two shares cover every image once."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_unwrap_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    assert sorted(res[0][1] + res[1][1]) == list(range(11))
    assert not set(res[0][1]) & set(res[1][1])
    for _, idx, vals in res:
        assert vals == [i + 1.0 for i in idx]
