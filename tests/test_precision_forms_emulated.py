"""Precision forms of the Laplacian block's DCT solve (Sec. 3.3), emulated on the CPU inside the
oracle's PCG (Alg. 2): the three products per stage evaluated with operands rounded to bfloat16
(one pass), to split bfloat16 (hi + lo, three products), or to float16 with every stored
intermediate scaled to its own maximum first; accumulation in float64 (the tensor cores
accumulate in float32).  The CG iteration counts of the first outer system show which forms keep
the preconditioner symmetric and accurate enough for cg_tol = 1e-6.  No GPU."""
import numpy as np
import pytest

import synthetic
from oracle import irls as O


def bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16      # round to nearest even, 8-bit mantissa
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def fp16(x):
    return np.asarray(x, dtype=np.float16).astype(np.float64)


def product(A, B, form):
    if form == "bf16x3":
        Ah, Bh = bf16(A), bf16(B)
        return Ah @ Bh + Ah @ bf16(B - Bh) + bf16(A - Ah) @ Bh
    f = bf16 if form == "bf16" else fp16
    return f(A) @ f(B)


def stored(X, form):
    if form == "bf16x3":
        h = bf16(X)
        return h + bf16(X - h)
    if form == "fp16":
        s = max(np.abs(X).max(), 1e-300)          # per-stage scale: the largest value maps to 1
        return fp16(X / s) * s
    return bf16(X)


def emulated_precond(form):
    def apply(r, dv, dh, tau, basis_N, basis_M):
        rU, rVv, rVh = r
        PN, lamN = basis_N
        PM, lamM = basis_M
        den = lamN[:, None] + lamM[None, :]
        keep = den > 0
        keep[0, 0] = False
        R = stored(tau * rU, form)
        T1 = stored(product(PN.T, R, form), form)
        Y = product(T1, PM, form)
        G = np.zeros_like(Y)
        G[keep] = Y[keep] / den[keep]
        T3 = stored(product(PN, stored(G, form), form), form)
        zU = product(T3, PM.T, form)
        return (zU, rVv / (dv + 1.0 / tau), rVh / (dh + 1.0 / tau))
    return apply


def first_solve_iterations(form, monkeypatch, n=256):
    d = synthetic.config_2048(seed=10, H=n, W=n)
    if form != "fp64":
        monkeypatch.setattr(O, "precond_apply", emulated_precond(form))
    r = O.irls_unwrap(d["X"], d["coherence"], tau=1e-2, delta=1e-3, outer_iters=1, cg_tol=1e-6,
                      cg_max=3000)
    monkeypatch.undo()
    return r["cg_iters"][0]


def test_precision_forms_first_solve(monkeypatch):
    """This emulation, first outer system, cg_tol 1e-6 (float64 / split bf16 / single-pass bf16
    / scaled float16): 256 x 256: 256 / 266 / 437 / 298 iterations; 512 x 512: 232 / 242 / 548 /
    276.  Split bf16 stays within 5 % of float64; single-pass bf16 degrades as the size grows
    (tau / lambda_min grows as n^2); float16 with every intermediate scaled to its own maximum
    stays within about 20 %."""
    it = {f: first_solve_iterations(f, monkeypatch) for f in ("fp64", "bf16x3", "bf16", "fp16")}
    assert it["bf16x3"] <= 1.1 * it["fp64"], it
    assert it["fp16"] <= 1.3 * it["fp64"], it
    assert it["bf16"] >= 1.4 * it["fp64"], it
