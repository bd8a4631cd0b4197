"""ctypes binding of libirls (include/irls.h): argument marshalling only.

Every step of the unwrapping path runs in the library's CUDA kernels; this module converts
Python arguments into the C ABI's plain pointers and sizes.  There is no CPU fallback: if the
library is missing the import of the functions below raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libirls.so")

IRLS_MAX_OUTER = 256
DCT_FORMS = {"auto": 0, "direct": 1, "folded": 2, "fft": 3}
CG_SCHEDULES = {"fixed": 0, "paper": 1}
SYSTEMS = {"full": 0, "schur": 1}
PRECISIONS = {"fp32": 0, "bf16": 1, "bf16x3": 2, "fp16": 3}

STATUS = {
    0: "IRLS_OK", 1: "IRLS_WARN_CG_MAX", -1: "IRLS_ERR_ARG", -2: "IRLS_ERR_SHAPE",
    -3: "IRLS_ERR_NONFINITE", -4: "IRLS_ERR_OOM", -5: "IRLS_ERR_BREAKDOWN",
    -6: "IRLS_ERR_TIMEOUT", -7: "IRLS_ERR_CUDA", -8: "IRLS_ERR_UNSUPPORTED",
}


class Opts(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_float),
        ("delta", ctypes.c_float),
        ("outer_iters", ctypes.c_int),
        ("cg_tol", ctypes.c_float),
        ("cg_max_iter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("flexible_cg", ctypes.c_int),
        ("warm_start", ctypes.c_int),
        ("dct_form", ctypes.c_int),
        ("cg_schedule", ctypes.c_int),
        ("cg_m0", ctypes.c_int),
        ("cg_eps_tol", ctypes.c_float),
        ("cg_alpha", ctypes.c_float),
        ("system", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("outer_done", ctypes.c_int),
        ("cg_total", ctypes.c_int),
        ("status", ctypes.c_int),
        ("cg_iters", ctypes.c_int * IRLS_MAX_OUTER),
        ("rel_res", ctypes.c_double * IRLS_MAX_OUTER),
        ("l1_obj", ctypes.c_double * IRLS_MAX_OUTER),
        ("h_delta", ctypes.c_double * IRLS_MAX_OUTER),
        ("f_delta", ctypes.c_double * IRLS_MAX_OUTER),
        ("cg_cap", ctypes.c_int * IRLS_MAX_OUTER),
        ("schedule_stop", ctypes.c_int),
    ]

    def to_dict(self):
        n = self.outer_done
        return {
            "outer_done": n,
            "cg_total": self.cg_total,
            "status": self.status,
            "cg_iters": list(self.cg_iters[:n]),
            "rel_res": list(self.rel_res[:n]),
            "l1_obj": list(self.l1_obj[:n]),
            "h_delta": list(self.h_delta[:n]),
            "f_delta": list(self.f_delta[:n]),
            "cg_cap": list(self.cg_cap[:n]),
            "schedule_stop": bool(self.schedule_stop),
            "f_delta_stop": (self.f_delta[n] if self.schedule_stop and n < IRLS_MAX_OUTER
                             else None),
        }


_P = ctypes.c_void_p
_F = ctypes.c_float
_I = ctypes.c_int

# name -> (restype, argtypes); mirrors include/irls.h
SIGNATURES = {
    "irls_opts_default": (_I, [ctypes.POINTER(Opts)]),
    "irls_workspace_bytes": (ctypes.c_size_t, [_I, _I, ctypes.POINTER(Opts)]),
    "irls_plan_create": (_I, [_I, _I, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "irls_plan_destroy": (_I, [_P]),
    "irls_plan_set_opts": (_I, [_P, ctypes.POINTER(Opts)]),
    "irls_plan_dct_form": (_I, [_P]),
    "irls_plan_set_tiles": (_I, [_P, _I, _I]),
    "irls_debug_stall_fold": (_I, [_P, _I]),
    "irls_debug_fold_schedule": (_I, [_I, _P, _P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                      ctypes.POINTER(_I), _P, _I]),
    "irls_plan_get_tiles": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "irls_plan_autotune": (_I, [_P, ctypes.POINTER(ctypes.c_float), _P]),
    "irls_round_congruent": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "irls_best_shift_error": (_I, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), _P]),
    "irls_unwrap": (_I, [_P, _P, _I, _I, _F, _I, _F, _P, _P]),
    "irls_unwrap_ex": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Stats), _P]),
    "irls_unwrap_forward_record": (_I, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(_P),
                                        ctypes.POINTER(Stats), _P]),
    "irls_unwrap_backward": (_I, [_P, _P, _P, _P, ctypes.POINTER(Stats), _P]),
    "irls_tape_free": (_I, [_P]),
    "irls_batch_create": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(Opts),
                               ctypes.POINTER(_P)]),
    "irls_batch_destroy": (_I, [_P]),
    "irls_unwrap_batched_ex": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                    ctypes.POINTER(_P), ctypes.POINTER(Stats), _P]),
    "irls_unwrap_batched": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_P),
                                 ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(Opts),
                                 ctypes.POINTER(Stats), _P]),
    "irls_batch_uses_graphs": (_I, [_P]),
    "irls_batch_dct_form": (_I, [_P]),
    "irls_batch_set_tiles": (_I, [_P, _I, _I]),
    "irls_batch_get_tiles": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "irls_batch_autotune": (_I, [_P, ctypes.POINTER(ctypes.c_float), _P]),
    "irls_tiled_create": (_I, [_I, _I, _I, _I, ctypes.POINTER(Opts), ctypes.POINTER(_P)]),
    "irls_tiled_destroy": (_I, [_P]),
    "irls_tiled_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                             ctypes.POINTER(_I)]),
    "irls_tiled_batch": (_I, [_P, ctypes.POINTER(_P)]),
    "irls_unwrap_tiled": (_I, [_P, _P, _P, _P, ctypes.POINTER(Stats),
                               ctypes.POINTER(ctypes.c_double), _P]),
    "irls_precond_laplacian": (_I, [_P, _P, _P, _P]),
    "irls_apply_A": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "irls_precond_laplacian_noalloc": (_I, [_P, _P, _I, _I, _F, _P]),
    "irls_plan_set_profiling": (_I, [_P, _I]),
    "irls_plan_profile": (_I, [_P, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_longlong), _I]),
    "irls_status_string": (ctypes.c_char_p, [_I]),
    "irls_last_cuda_error": (_I, []),
}

_lib = None


def lib():
    """Load libirls.so (built in-tree by ``paper_2401_09961_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libirls.so not found at {LIB_PATH}; build it with "
                "`python -m paper_2401_09961_gb300.build` (the CUDA path has no fallback)")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


class IrlsError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().irls_status_string(code).decode()
        extra = ""
        if code == -7:
            extra = f" (cudaError {lib().irls_last_cuda_error()})"
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}{extra}")


def check(code, where=""):
    if code < 0:
        raise IrlsError(code, where)
    return code


def default_opts(**kw):
    o = Opts()
    check(lib().irls_opts_default(ctypes.byref(o)), "irls_opts_default")
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
    return o


FOLD_SCHED_INTS = 33
FOLD_SCHED_FIELDS = (["stage", "image", "local", "m0", "n0", "width", "nkb", "dual", "half",
                      "sig", "ndep"] + [f"dep{d}" for d in range(8)] +
                     [f"need{d}" for d in range(8)] + ["rho_end", "rho_nslot", "M", "N", "K", "prob"])


def fold_schedule(shapes, pairs):
    """The folded preconditioner launch's work list for images of the given (H, W) shapes run
    by `pairs` CTA pairs (host only, no device work): an int32 array with one row of
    FOLD_SCHED_FIELDS per item in list order, the panel counter count and the item capacity."""
    import numpy as np
    T = len(shapes)
    H = (ctypes.c_int * max(T, 1))(*[int(h) for h, _ in shapes])
    W = (ctypes.c_int * max(T, 1))(*[int(w) for _, w in shapes])
    ni, nc, cap = _I(), _I(), _I()
    check(lib().irls_debug_fold_schedule(T, H, W, int(pairs), ctypes.byref(ni), ctypes.byref(nc),
                                         ctypes.byref(cap), None, 0), "irls_debug_fold_schedule")
    rec = np.zeros((ni.value, FOLD_SCHED_INTS), dtype=np.int32)
    check(lib().irls_debug_fold_schedule(T, H, W, int(pairs), ctypes.byref(ni), ctypes.byref(nc),
                                         ctypes.byref(cap), rec.ctypes.data, ni.value),
          "irls_debug_fold_schedule")
    return rec, nc.value, cap.value
