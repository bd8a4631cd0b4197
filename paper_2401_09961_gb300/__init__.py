"""GB300-native L1 phase unwrapping by IRLS + DCT-preconditioned CG (arXiv 2401.09961).

The compute path is libirls.so (hand-written CUDA for sm_103a behind a C ABI, include/irls.h);
this package marshals torch tensors into it.  PyTorch provides device memory and streams only.

    import torch, paper_2401_09961_gb300 as irls
    U = irls.unwrap(X_cuda, coherence_cuda, eps=1e-3, outer_iters=20, cg_tol=1e-6)
"""
from __future__ import annotations

import ctypes

from ._binding import (CG_SCHEDULES, DCT_FORMS, SYSTEMS, IRLS_MAX_OUTER, PRECISIONS, IrlsError, Opts, Stats, check, default_opts,
                       lib)

__all__ = ["Plan", "Batch", "Tiled", "unwrap", "precond_laplacian", "apply_A", "round_congruent",
           "best_shift_error", "default_opts", "lib", "IrlsError",
           "Opts", "Stats", "PRECISIONS", "unwrap_differentiable"]


def unwrap_differentiable(X, coherence, plan):
    """U(X, coherence) as a torch autograd node (hand-written adjoint, see .autograd)."""
    from .autograd import UnwrapFn
    return UnwrapFn.apply(X, coherence, plan)


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    torch = _torch()
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Owns an irls_plan: device workspace, DCT eigenbases and device-resident solver state
    for one H x W image shape (Sec. 3.3: the eigendecompositions are computed once)."""

    def __init__(self, H, W, **opts):
        self.H, self.W = int(H), int(W)
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        check(lib().irls_plan_create(self.H, self.W, ctypes.byref(self.opts), ctypes.byref(h)),
              "irls_plan_create")
        self._h = h

    @property
    def folded(self):
        """True when the preconditioner runs in the folded (even / odd) form."""
        return lib().irls_plan_dct_form(self.handle) == DCT_FORMS["folded"]

    @property
    def dct_form_name(self):
        """The preconditioner form in use: "folded", "direct" (tensor-core products), "fft"
        (fast transforms) or "simt" (float32 dense products on the CUDA cores)."""
        f = lib().irls_plan_dct_form(self.handle)
        names = {DCT_FORMS["folded"]: "folded", DCT_FORMS["direct"]: "direct",
                 DCT_FORMS["fft"]: "fft", DCT_FORMS["auto"]: "simt"}
        return names.get(f, str(f))

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    @property
    def tiles(self):
        """(direction, update) image rows per block of the CG stencil kernels in use."""
        d, u = ctypes.c_int(), ctypes.c_int()
        check(lib().irls_plan_get_tiles(self.handle, ctypes.byref(d), ctypes.byref(u)),
              "irls_plan_get_tiles")
        return d.value, u.value

    def set_tiles(self, dir_rows=0, upd_rows=0):
        """Sets the stencil tile shapes (image rows per block, 8 to 64; 0 keeps the current
        value)."""
        check(lib().irls_plan_set_tiles(self.handle, int(dir_rows), int(upd_rows)),
              "irls_plan_set_tiles")

    def autotune(self, cache=None, stream=None):
        """Times the stencil kernels' tile shapes on this GPU and keeps the fastest.  With
        `cache` (a JSON file path) a result stored for the same size, precision, system and GPU
        is applied without timing, and a new result is stored.  Returns a dict with the tiles in
        use, the eight timings in ms (None when cached) and whether the cache answered."""
        from . import tuning
        torch = _torch()
        key = tuning.tuning_key(self.H, self.W, self.opts.precision, self.opts.system,
                                torch.cuda.get_device_name())
        hit = tuning.cache_get(cache, key) if cache else None
        if hit is not None:
            self.set_tiles(*hit)
            return {"tiles": self.tiles, "ms": None, "cached": True}
        ms = (ctypes.c_float * 8)()
        check(lib().irls_plan_autotune(self.handle, ms, _stream(stream)), "irls_plan_autotune")
        tiles = self.tiles
        if cache:
            tuning.cache_put(cache, key, tiles, list(ms))
        return {"tiles": tiles, "ms": list(ms), "cached": False}

    def set_opts(self, **kw):
        o = Opts.from_buffer_copy(self.opts)
        for k, v in kw.items():
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            if k == "dct_form" and isinstance(v, str):
                v = DCT_FORMS[v]
            if k == "cg_schedule" and isinstance(v, str):
                v = CG_SCHEDULES[v]
            if k == "system" and isinstance(v, str):
                v = SYSTEMS[v]
            setattr(o, k, v)
        check(lib().irls_plan_set_opts(self.handle, ctypes.byref(o)), "irls_plan_set_opts")
        self.opts = o

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().irls_plan_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self):
        return int(lib().irls_workspace_bytes(self.H, self.W, ctypes.byref(self.opts)))

    def unwrap(self, X, coherence=None, *, Cv=None, Ch=None, U_init=None, Vv_init=None,
               Vh_init=None, out=None, return_slacks=False, stream=None):
        """Run Alg. 1 on device tensors; returns U (and (Vv, Vh) with return_slacks) and stats."""
        torch = _torch()
        H, W = self.H, self.W
        if tuple(X.shape) != (H, W):
            raise ValueError(f"X has shape {tuple(X.shape)}, plan is {(H, W)}")
        dev = X.device
        U = out if out is not None else torch.empty((H, W), device=dev, dtype=torch.float32)
        Vv = Vh = None
        if return_slacks or U_init is not None:
            Vv = torch.empty((max(H - 1, 0), W), device=dev, dtype=torch.float32)
            Vh = torch.empty((H, max(W - 1, 0)), device=dev, dtype=torch.float32)
            if U_init is not None:
                Vv.copy_(Vv_init)
                Vh.copy_(Vh_init)
        st = Stats()
        rc = lib().irls_unwrap_ex(self.handle, _ptr(X), _ptr(coherence), _ptr(Cv), _ptr(Ch),
                                  _ptr(U_init), _ptr(U),
                                  _ptr(Vv) if Vv is not None and Vv.numel() else None,
                                  _ptr(Vh) if Vh is not None and Vh.numel() else None,
                                  ctypes.byref(st), _stream(stream))
        check(rc, "irls_unwrap_ex")
        stats = st.to_dict()
        stats["return_code"] = rc
        if return_slacks:
            return U, Vv, Vh, stats
        return U, stats


def unwrap(X, coherence=None, *, eps=1e-3, outer_iters=20, cg_tol=1e-6, tau=1e-2,
           cg_max_iter=1000, precision="fp32", flexible_cg=None, Cv=None, Ch=None,
           return_stats=False, plan=None, cg_schedule="fixed", system="full"):
    """Unwrap the wrapped phase X (H x W float32) with the L1 IRLS method.

    X and the optional coherence / Cv / Ch may be CUDA tensors (the result stays on the device)
    or host arrays / CPU tensors (they are copied to the current CUDA device and U is copied
    back).  eps is the smoothing delta of F_delta (Sec. 3.1).  cg_schedule "paper" runs the
    adaptive CG budget and IRLS stop of Sec. 4.3 (outer_iters then bounds the number of IRLS
    iterations); system "schur" solves the U-only system left after eliminating V."""
    torch = _torch()
    import numpy as np
    host = not (isinstance(X, torch.Tensor) and X.is_cuda)

    def dev(a):
        if a is None:
            return None
        t = torch.as_tensor(np.asarray(a) if not isinstance(a, torch.Tensor) else a)
        return t.to(device="cuda", dtype=torch.float32).contiguous()

    Xd = dev(X)
    H, W = Xd.shape
    if flexible_cg is None:
        # the single-pass bf16 preconditioner is inexact enough to need the flexible ratio;
        # fp32 and the split bf16x3 form converge like exact arithmetic with the ratio of Alg. 2
        flexible_cg = 1 if precision == "bf16" else 0
    own = plan is None
    if own:
        plan = Plan(H, W, tau=tau, delta=eps, outer_iters=outer_iters, cg_tol=cg_tol,
                    cg_max_iter=cg_max_iter, precision=precision, flexible_cg=flexible_cg,
                    cg_schedule=cg_schedule, system=system)
    try:
        U, stats = plan.unwrap(Xd, dev(coherence), Cv=dev(Cv), Ch=dev(Ch))
    finally:
        if own:
            plan.close()
    if host:
        U = U.cpu()
    return (U, stats) if return_stats else U


class Batch:
    """A batched solve of images of uneven sizes (one launch per phase for all of them)."""

    def __init__(self, shapes, **opts):
        self.shapes = [(int(h), int(w)) for h, w in shapes]
        T = len(self.shapes)
        if "precision" not in opts:
            opts["precision"] = "bf16x3"
        self.opts = default_opts(**opts)
        Hs = (ctypes.c_int * T)(*[h for h, _ in self.shapes])
        Ws = (ctypes.c_int * T)(*[w for _, w in self.shapes])
        h = ctypes.c_void_p()
        check(lib().irls_batch_create(T, Hs, Ws, ctypes.byref(self.opts), ctypes.byref(h)),
              "irls_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().irls_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def uses_graphs(self):
        return lib().irls_batch_uses_graphs(self._h) == 1

    @property
    def folded(self):
        """True when the batch's preconditioner runs in the folded (even / odd) form."""
        return lib().irls_batch_dct_form(self._h) == DCT_FORMS["folded"]

    @property
    def tiles(self):
        """(direction, update) image rows per block of the batched CG stencil launches."""
        d, u = ctypes.c_int(), ctypes.c_int()
        check(lib().irls_batch_get_tiles(self._h, ctypes.byref(d), ctypes.byref(u)),
              "irls_batch_get_tiles")
        return d.value, u.value

    def set_tiles(self, dir_rows=0, upd_rows=0):
        """Sets the stencil tile shapes (one of 8, 16, 24, 32; 0 keeps the current value)."""
        check(lib().irls_batch_set_tiles(self._h, int(dir_rows), int(upd_rows)),
              "irls_batch_set_tiles")

    def autotune(self, cache=None, stream=None):
        """As Plan.autotune, for the batch's launches; the cache key holds the batch's shapes."""
        from . import tuning
        torch = _torch()
        key = tuning.batch_key(self.shapes, self.opts.precision, self.opts.system,
                               torch.cuda.get_device_name())
        hit = tuning.cache_get(cache, key) if cache else None
        if hit is not None:
            self.set_tiles(*hit)
            return {"tiles": self.tiles, "ms": None, "cached": True}
        ms = (ctypes.c_float * 8)()
        check(lib().irls_batch_autotune(self._h, ms, _stream(stream)), "irls_batch_autotune")
        tiles = self.tiles
        if cache:
            tuning.cache_put(cache, key, tiles, list(ms))
        return {"tiles": tiles, "ms": list(ms), "cached": False}

    def unwrap(self, Xs, cohs=None, outs=None, stream=None):
        """Xs, cohs: lists of contiguous float32 CUDA tensors; returns (list of U, list of stats)."""
        torch = _torch()
        T = len(self.shapes)
        if len(Xs) != T:
            raise ValueError("one X per image")
        for X, (h, w) in zip(Xs, self.shapes):
            if tuple(X.shape) != (h, w):
                raise ValueError("image shape does not match the batch")
        Us = outs if outs is not None else [torch.empty_like(X) for X in Xs]
        P = ctypes.c_void_p
        xa = (P * T)(*[_ptr(X) for X in Xs])
        ua = (P * T)(*[_ptr(U) for U in Us])
        ca = (P * T)(*[_ptr(c) for c in cohs]) if cohs is not None else None
        st = (Stats * T)()
        rc = lib().irls_unwrap_batched_ex(self._h, xa, ca, ua, st, _stream(stream))
        check(rc, "irls_unwrap_batched_ex")
        return Us, [x.to_dict() for x in st]


class Tiled:
    """A tiled solve of one large H x W image (irls_tiled_*): overlapping tiles of side `tile`
    with `overlap` pixels in common, solved as one batch, then stitched by constants fixed on
    the overlaps.  Options as for Batch (precision bf16x3 by default)."""

    def __init__(self, H, W, tile=1024, overlap=64, **opts):
        if "precision" not in opts:
            opts["precision"] = "bf16x3"
        self.H, self.W, self.tile, self.overlap = int(H), int(W), int(tile), int(overlap)
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        check(lib().irls_tiled_create(self.H, self.W, self.tile, self.overlap,
                                      ctypes.byref(self.opts), ctypes.byref(h)),
              "irls_tiled_create")
        self._h = h
        n, th, tw, npair = (ctypes.c_int() for _ in range(4))
        check(lib().irls_tiled_info(h, ctypes.byref(n), ctypes.byref(th), ctypes.byref(tw),
                                    ctypes.byref(npair)), "irls_tiled_info")
        self.n_tiles, self.tile_shape, self.n_pairs = n.value, (th.value, tw.value), npair.value

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().irls_tiled_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, stream=None):
        """Times the batched stencil tile shapes on this solve's batch and keeps the fastest."""
        b = ctypes.c_void_p()
        check(lib().irls_tiled_batch(self._h, ctypes.byref(b)), "irls_tiled_batch")
        ms = (ctypes.c_float * 8)()
        check(lib().irls_batch_autotune(b, ms, _stream(stream)), "irls_batch_autotune")
        return list(ms)

    def unwrap(self, X, coherence=None, out=None, stream=None):
        """X, coherence: H x W float32 CUDA tensors; returns (U, per-tile stats, constants)."""
        torch = _torch()
        if tuple(X.shape) != (self.H, self.W):
            raise ValueError("image shape does not match the tiled solve")
        U = out if out is not None else torch.empty_like(X)
        st = (Stats * self.n_tiles)()
        c = (ctypes.c_double * self.n_tiles)()
        rc = lib().irls_unwrap_tiled(self._h, _ptr(X), _ptr(coherence), _ptr(U), st, c,
                                     _stream(stream))
        check(rc, "irls_unwrap_tiled")
        return U, [x.to_dict() for x in st], list(c)


def precond_laplacian(plan, R, stream=None):
    """Z solving S^T S Z + Z T T^T = tau R in the DCT eigenbasis (Sec. 3.3), on device."""
    torch = _torch()
    Z = torch.empty_like(R)
    check(lib().irls_precond_laplacian(plan.handle, _ptr(R), _ptr(Z), _stream(stream)),
          "irls_precond_laplacian")
    return Z


def round_congruent(plan, U, X, stream=None):
    """'Rounded IRLS' (Sec. 4.5): (U_round, K, c) with U_round = X + 2pi K the image
    2pi-congruent to X nearest to U aligned by its circular-mean offset c (device tensors)."""
    torch = _torch()
    Ur = torch.empty_like(U)
    K = torch.empty(U.shape, device=U.device, dtype=torch.int32)
    c = ctypes.c_double()
    check(lib().irls_round_congruent(plan.handle, _ptr(U), _ptr(X), _ptr(Ur),
                                     ctypes.c_void_p(K.data_ptr()), ctypes.byref(c),
                                     _stream(stream)), "irls_round_congruent")
    return Ur, K, c.value


def best_shift_error(plan, U, Xu, stream=None):
    """Best-shift error of Sec. 4.5: (E, alpha, rms) with E = (Xu - U) - alpha on the device."""
    torch = _torch()
    E = torch.empty_like(U)
    a, r = ctypes.c_double(), ctypes.c_double()
    check(lib().irls_best_shift_error(plan.handle, _ptr(U), _ptr(Xu), _ptr(E), ctypes.byref(a),
                                      ctypes.byref(r), _stream(stream)), "irls_best_shift_error")
    return E, a.value, r.value


def apply_A(plan, U, Vv, Vh, Dv, Dh, stream=None):
    """(q_U, q_Vv, q_Vh) = A (U, Vv, Vh) with the matrix A of Sec. 3.2, on device."""
    torch = _torch()
    qU = torch.empty_like(U)
    qVv = torch.empty_like(Vv)
    qVh = torch.empty_like(Vh)
    nz = lambda t: _ptr(t) if t.numel() else None  # noqa: E731
    check(lib().irls_apply_A(plan.handle, _ptr(U), nz(Vv), nz(Vh), nz(Dv), nz(Dh), _ptr(qU),
                             nz(qVv), nz(qVh), _stream(stream)), "irls_apply_A")
    return qU, qVv, qVh
