"""Seeded synthetic interferograms shaped like the paper's workloads.

The paper unwraps Sentinel-1 topographic phases (2048 x 2048 crops and ~4000 x 20000 stitched
bursts, Sec. 4.1) with SNAPHU-derived edge weights (Sec. 4.2).  Neither the data nor SNAPHU is
available, so these generators stand in for them.  They hold none of the unwrapping method's
arithmetic: they only draw a true (unwrapped) phase, a coherence map and the observed wrapped
phase.  Both the FP64 oracle and the CUDA path consume their output.

Recipe (all sizes in pixels, all draws from ``numpy.random.default_rng(seed)``):

* true phase = linear ramp from 0 to ``ramp`` rad across the image along a random direction
  + ``n_bumps`` Gaussian bumps (amplitude U[5, 30] rad, sigma U[10, 60] px, centres uniform);
* optional step discontinuities: ``n_steps`` half-planes bounded by random lines through the
  image, each offset by +3*pi (these violate Itoh's condition on purpose);
* coherence (optional) = uniform noise, Gaussian-blurred with sigma = 16 px (periodic FFT blur),
  affinely rescaled to [0.05, 1]; optional low-coherence elliptic patches covering
  ``patch_frac`` of the pixels where the coherence is redrawn from U[0.05, 0.2];
* observed phase = wrap(true phase + N(0, noise^2)) into (-pi, pi], with the noise standard
  deviation raised to ``patch_noise`` inside the patches;
* X is returned as float32 (the library's input type); the true phase is returned in float64
  with its mean removed.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "make_phase",
    "config_small",
    "config_2048",
    "config_4096_mixed",
    "config_adjoint_1024",
    "batched_tiles",
    "smooth_phase",
]


def _ramp(H, W, ramp, rng):
    theta = rng.uniform(0.0, 2.0 * np.pi)
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    proj = x * np.cos(theta) + y * np.sin(theta)
    lo, hi = proj.min(), proj.max()
    if hi - lo <= 0:
        return np.zeros((H, W))
    return ramp * (proj - lo) / (hi - lo)


def _bumps(H, W, n, rng, amp=(5.0, 30.0), sig=(10.0, 60.0)):
    out = np.zeros((H, W))
    for _ in range(n):
        a = rng.uniform(*amp)
        s = rng.uniform(*sig)
        cy = rng.uniform(0, H)
        cx = rng.uniform(0, W)
        r = int(np.ceil(5.0 * s))
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
        xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
        out[y0:y1, x0:x1] += a * np.exp(-(yy * yy + xx * xx) / (2.0 * s * s))
    return out


def _steps(H, W, n, rng, height=3.0 * np.pi):
    out = np.zeros((H, W))
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(n):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        th = rng.uniform(0, np.pi)
        side = (x - cx) * np.cos(th) + (y - cy) * np.sin(th) > 0
        out += height * side
    return out


def _blur_periodic(a, sigma):
    H, W = a.shape
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    g = np.exp(-2.0 * (np.pi * sigma) ** 2 * (fy * fy + fx * fx))
    return np.fft.irfft2(np.fft.rfft2(a) * g, s=(H, W))


def _coherence(H, W, rng, lo=0.05, hi=1.0, sigma=16.0):
    c = _blur_periodic(rng.uniform(0.0, 1.0, size=(H, W)), sigma)
    cmin, cmax = c.min(), c.max()
    if cmax - cmin <= 0:
        return np.full((H, W), hi)
    return lo + (hi - lo) * (c - cmin) / (cmax - cmin)


def _patches(H, W, frac, rng):
    """Boolean mask of random ellipses covering about ``frac`` of the image."""
    mask = np.zeros((H, W), dtype=bool)
    if frac <= 0:
        return mask
    target = frac * H * W
    side = min(H, W)
    for _ in range(10000):
        if mask.sum() >= target:
            break
        a = rng.uniform(0.02, 0.08) * side
        b = rng.uniform(0.02, 0.08) * side
        th = rng.uniform(0, np.pi)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        r = int(np.ceil(max(a, b))) + 1
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1)[:, None] - cy
        xx = np.arange(x0, x1)[None, :] - cx
        u = xx * np.cos(th) + yy * np.sin(th)
        v = -xx * np.sin(th) + yy * np.cos(th)
        mask[y0:y1, x0:x1] |= (u / a) ** 2 + (v / b) ** 2 <= 1.0
    return mask


def _wrap_observation(phi):
    """Observed phase in (-pi, pi] (the sensor's wrap, not the method's)."""
    return np.angle(np.exp(1j * phi))


def make_phase(H, W, seed, *, ramp, n_bumps, noise, coherence=False, patch_frac=0.0,
               patch_noise=1.2, n_steps=0):
    """Draw one synthetic interferogram.

    Returns a dict with ``X`` (float32 H x W, wrapped to (-pi, pi]), ``coherence`` (float32 H x W
    or None), ``phi_true`` (float64, noise-free unwrapped phase, mean removed) and ``patches``
    (bool mask of the low-coherence patches).
    """
    rng = np.random.default_rng(seed)
    phi = _ramp(H, W, ramp, rng) + _bumps(H, W, n_bumps, rng)
    if n_steps:
        phi = phi + _steps(H, W, n_steps, rng)
    coh = _coherence(H, W, rng) if coherence else None
    mask = _patches(H, W, patch_frac, rng)
    sig = np.full((H, W), float(noise))
    if mask.any():
        sig[mask] = patch_noise
        if coh is not None:
            coh[mask] = rng.uniform(0.05, 0.2, size=int(mask.sum()))
    obs = phi + rng.standard_normal((H, W)) * sig
    X = _wrap_observation(obs).astype(np.float32)
    return {
        "X": X,
        "coherence": None if coh is None else coh.astype(np.float32),
        "phi_true": phi - phi.mean(),
        "patches": mask,
    }


def config_small(seed=0, H=256, W=256):
    """256 x 256: ramp 0-40 rad, 5 bumps, noise 0.3 rad, uniform weights."""
    return make_phase(H, W, seed, ramp=40.0 * max(H, W) / 256.0, n_bumps=5, noise=0.3)


def config_2048(seed=10, H=2048, W=2048):
    """2048 x 2048: ramp 0-400 rad, 40 bumps, noise 0.5 rad, smoothed coherence weights."""
    s = max(H, W) / 2048.0
    return make_phase(H, W, seed, ramp=400.0 * s, n_bumps=max(1, int(round(40 * s))),
                      noise=0.5, coherence=True)


def config_4096_mixed(seed=20, H=4096, W=4096):
    """4096 x 4096: ramp 0-800 rad, 80 bumps, noise 0.5 rad, coherence weights, 20 % of the pixels
    in low-coherence patches (coherence U[0.05, 0.2], noise 1.2 rad), two +3*pi steps."""
    s = max(H, W) / 4096.0
    return make_phase(H, W, seed, ramp=800.0 * s, n_bumps=max(1, int(round(80 * s))),
                      noise=0.5, coherence=True, patch_frac=0.2, patch_noise=1.2, n_steps=2)


def config_adjoint_1024(seed=30, H=1024, W=1024):
    """1024 x 1024: ramp 0-200 rad, 20 bumps, noise 0.5 rad, coherence weights."""
    s = max(H, W) / 1024.0
    return make_phase(H, W, seed, ramp=200.0 * s, n_bumps=max(1, int(round(20 * s))),
                      noise=0.5, coherence=True)


def batched_tile_shapes(n=64, seed_base=1000, sides=tuple(range(256, 1537, 128))):
    """The (H, W) of each tile ``batched_tiles`` draws, without drawing the images."""
    shapes = []
    for t in range(n):
        rng = np.random.default_rng(seed_base + t)
        H = int(rng.choice(sides))
        W = int(rng.choice(sides))
        shapes.append((H, W))
    return shapes


def batched_tiles(n=64, seed_base=1000, sides=tuple(range(256, 1537, 128)), indices=None):
    """``n`` independent tiles with each side drawn uniformly from ``sides`` (non-square allowed),
    tile t seeded with ``seed_base + t`` and drawn with the 2048 x 2048 law scaled to its size.
    With ``indices``, only those tiles (in that order) are drawn."""
    shapes = batched_tile_shapes(n, seed_base, sides)
    idx = range(n) if indices is None else indices
    return [config_2048(seed=seed_base + t, H=shapes[t][0], W=shapes[t][1]) for t in idx]


def smooth_phase(H, W, seed, max_step=2.0):
    """Noise-free smooth phase whose neighbour differences stay below ``max_step`` rad (< pi),
    so Itoh's condition holds everywhere.  Returns (X float32 wrapped, phi float64 mean-free)."""
    rng = np.random.default_rng(seed)
    phi = _ramp(H, W, rng.uniform(0.5, 1.5) * max_step * 0.5 * max(H, W) / 2.0, rng)
    phi += _bumps(H, W, 2, rng, amp=(0.5, 2.0), sig=(max(1.0, min(H, W) / 4.0),
                                                        max(1.5, min(H, W) / 2.0)))
    dv = np.abs(np.diff(phi, axis=0)).max(initial=0.0)
    dh = np.abs(np.diff(phi, axis=1)).max(initial=0.0)
    m = max(dv, dh)
    if m > max_step:
        phi *= max_step / m
    X = _wrap_observation(phi).astype(np.float32)
    return X, phi - phi.mean()
