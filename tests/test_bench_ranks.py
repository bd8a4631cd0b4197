"""The multi-rank path of bench.py on CPU: two gloo ranks, the timing aggregation (slowest rank,
whole-job units) and the reference arm's rank-0-only rule.  No GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r took (r + 1) * 100 ms for its steps and processed 16.78 * (r + 1) Mpix
        ms = bench.rank_max((rank + 1) * 100.0, world, device="cpu")
        mpix = bench.rank_sum(16.78 * (rank + 1), world, device="cpu")
        ref = bench.reference_arm(None, rank, world, 4096, "bf16x3") if rank == 1 else "skipped"
        out.put((rank, ms, mpix, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, ms, mpix, ref in got:
        assert ms == 200.0                           # the slowest rank's time, on every rank
        assert mpix == pytest.approx(16.78 * 3)      # both ranks' pixels
    assert got[1][3] is None                         # rank 1 of the reference arm: no work


def test_single_rank_is_the_identity():
    import bench
    assert bench.rank_max(3.5, 1) == 3.5 and bench.rank_sum(2.0, 1) == 2.0
