"""unwrap_sharded on the GPU: a rank's share of a tile list, solved by the batched form, equals
the same tiles solved by a Batch built directly (bit for bit), and the shares cover the list."""
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


OPTS = dict(precision="bf16x3", tau=1e-2, delta=1e-3, outer_iters=3, cg_tol=1e-6,
            cg_max_iter=1000)


def host(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32))


def test_share_equals_a_batch_of_the_same_tiles(irls):
    from paper_2401_09961_gb300 import sharding
    shapes = [(256, 256), (300, 256), (256, 320), (128, 200), (384, 256)]
    tiles = [synthetic.config_2048(seed=700 + t, H=h, W=w) for t, (h, w) in enumerate(shapes)]
    Xh = [host(d["X"]) for d in tiles]           # stay in host memory: the share is copied
    Ch = [host(d["coherence"]) for d in tiles]
    seen = []
    for rank in range(2):
        idx, Us, st = sharding.unwrap_sharded(Xh, Ch, rank=rank, world=2, **OPTS)
        assert idx == sharding.shard_tiles(shapes, rank, 2) and len(idx) > 0
        seen += idx
        with irls.Batch([shapes[i] for i in idx], **OPTS) as b:
            Ur, sr = b.unwrap([Xh[i].cuda() for i in idx], [Ch[i].cuda() for i in idx])
        torch.cuda.synchronize()
        for a, r in zip(Us, Ur):
            assert a.is_cuda and torch.equal(a, r)
        assert [s["cg_total"] for s in st] == [s["cg_total"] for s in sr]
        assert all(s["status"] >= 0 for s in st)
    assert sorted(seen) == list(range(len(shapes)))
