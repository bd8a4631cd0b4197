"""Rounded IRLS output and best-shift error (Sec. 4.5) on the GPU against the oracle."""
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


def planted(H, W, seed, noise=0.3):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-np.pi, np.pi, (H, W)).astype(np.float32)
    K0 = rng.integers(-200, 201, (H, W))
    U = (X + 2 * np.pi * K0 + 0.77 + noise * rng.standard_normal((H, W))).astype(np.float32)
    return X, U, K0


@pytest.mark.parametrize("H,W", [(1, 1), (37, 53), (300, 200), (4096, 4096)])
def test_round_congruent_matches_oracle(irls, H, W):
    """The integer map is bit-exact against the oracle's float32 recipe given the same offset,
    the rounded image is bit-exact, and the offset agrees with the oracle's FP64 sum."""
    X, U, K0 = planted(H, W, H + W)
    with irls.Plan(H, W) as p:
        Ur, K, c = irls.round_congruent(p, cuda(U), cuda(X))
    Ur_o, K_o, c_o = O.round_congruent(U, X, c=c)
    assert abs(c - O.round_congruent(U, X)[2]) < 1e-9
    assert np.array_equal(K.cpu().numpy().astype(np.int64), K_o)
    assert np.array_equal(Ur.cpu().numpy(), Ur_o)
    assert np.array_equal(K_o, K0)


def test_rounded_unwrap_output(irls):
    """The rounded output of a GPU unwrap: same integers as the oracle's rounding of the same U,
    and the planted phase's own ambiguities up to one global integer on >= 99.9 % of pixels."""
    d = synthetic.config_small(4, H=128, W=96)
    with irls.Plan(128, 96, delta=1e-3, outer_iters=10, cg_tol=1e-6) as p:
        U, _ = p.unwrap(cuda(d["X"]))
        _, K, c = irls.round_congruent(p, U, cuda(d["X"]))
    Ug = U.cpu().numpy()
    _, K_o, _ = O.round_congruent(Ug, d["X"], c=c)
    K = K.cpu().numpy().astype(np.int64)
    assert np.array_equal(K, K_o)
    _, Kt, _ = O.round_congruent(d["phi_true"], d["X"])
    diff = K - Kt
    vals, counts = np.unique(diff, return_counts=True)
    assert counts.max() >= 0.999 * diff.size


@pytest.mark.parametrize("H,W", [(37, 53), (1024, 768)])
def test_best_shift_error_matches_oracle(irls, H, W):
    rng = np.random.default_rng(H * W)
    Xu = (rng.standard_normal((H, W)) * 30).astype(np.float32)
    U = (Xu - 12.5 + 0.2 * rng.standard_normal((H, W))).astype(np.float32)
    with irls.Plan(H, W) as p:
        E, alpha, rms = irls.best_shift_error(p, cuda(U), cuda(Xu))
    E_o = O.best_shift_error(U.astype(np.float64), Xu.astype(np.float64))
    a_o = float(np.mean(Xu.astype(np.float64) - U.astype(np.float64)))
    assert abs(alpha - a_o) <= 1e-12 * max(1.0, abs(a_o)) + 1e-12
    assert abs(rms - np.sqrt(np.mean(E_o ** 2))) <= 1e-9 * rms
    # float32 output: (Xu - U) rounded, minus alpha rounded to float32
    assert np.abs(E.cpu().numpy() - E_o).max() <= 4e-6 * np.abs(Xu).max()
