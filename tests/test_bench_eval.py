"""The bench's result evaluators (FP64 L1 of problem (main), Sec. 2, and the 2pi-multiple
agreement of two unwraps) against the oracle's definitions."""
import numpy as np

import bench
import oracle.irls as O
import synthetic


def test_l1_fp64_matches_oracle_objective():
    d = synthetic.config_4096_mixed(seed=3, H=120, W=97)
    rng = np.random.default_rng(0)
    U = (d["X"].astype(np.float64) + 2 * np.pi * rng.integers(-2, 3, size=d["X"].shape)
         + 0.01 * rng.standard_normal(d["X"].shape))
    Gv, Gh = O.wrapped_gradients(d["X"])
    Cv, Ch = O.edge_weights(d["coherence"], *d["X"].shape)
    ref = O.l1_objective(U, Gv, Gh, Cv, Ch)
    assert abs(bench.l1_fp64(U, d["X"], d["coherence"]) - ref) <= 1e-12 * ref


def test_k_agreement_counts_2pi_jumps_and_ignores_constants():
    rng = np.random.default_rng(1)
    U = rng.standard_normal((64, 50)) * 20
    assert bench.k_agreement(U, U + 3.0) == 1.0
    jumps = rng.random(U.shape) < 0.05
    a = bench.k_agreement(U, U - 1.0 + 2 * np.pi * jumps)
    assert abs(a - (1.0 - jumps.mean())) < 1e-12
