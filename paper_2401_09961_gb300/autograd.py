"""Differentiable unwrapping: torch.autograd.Function over the library's recorded forward solve
and its adjoint sweep (irls_unwrap_forward_record / irls_unwrap_backward).

The backward pass treats each IRLS step as its converged inner solve: one adjoint PCG solve per
outer step with the same symmetric operator, plus the reweighting chain (Sec. 3.1-3.2).  The
checkpoints are the slack variables V^k of every outer step, not CG states.
"""
from __future__ import annotations

import ctypes

import torch

from ._binding import Stats, check, lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Tape:
    """Owns an irls_tape (device checkpoints of one recorded forward solve)."""

    def __init__(self, handle, has_coherence):
        self._h = handle
        self.has_coherence = has_coherence

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("tape already freed")
        return self._h

    def free(self):
        if getattr(self, "_h", None) is not None:
            lib().irls_tape_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def unwrap_record(plan, X, coherence=None, Cv=None, Ch=None):
    """Forward solve on `plan` that keeps the checkpoints for the adjoint; returns (U, tape, stats)."""
    U = torch.empty_like(X)
    h = ctypes.c_void_p()
    st = Stats()
    check(lib().irls_unwrap_forward_record(plan.handle, _ptr(X), _ptr(coherence), _ptr(Cv),
                                           _ptr(Ch), _ptr(U), ctypes.byref(h), ctypes.byref(st),
                                           _stream()), "irls_unwrap_forward_record")
    return U, Tape(h, coherence is not None and Cv is None), st.to_dict()


def unwrap_backward(tape, dL_dU, want_coherence=True):
    """Adjoint sweep: returns (dL/dX, dL/dcoherence or None, stats of the adjoint solves)."""
    dX = torch.empty_like(dL_dU)
    dc = torch.empty_like(dL_dU) if (want_coherence and tape.has_coherence) else None
    st = Stats()
    check(lib().irls_unwrap_backward(tape.handle, _ptr(dL_dU), _ptr(dX), _ptr(dc),
                                     ctypes.byref(st), _stream()), "irls_unwrap_backward")
    return dX, dc, st.to_dict()


class UnwrapFn(torch.autograd.Function):
    """U = UnwrapFn.apply(X, coherence, plan): gradients with respect to X and coherence."""

    @staticmethod
    def forward(ctx, X, coherence, plan):
        X = X.contiguous()
        coherence = coherence.contiguous() if coherence is not None else None
        U, tape, _ = unwrap_record(plan, X, coherence)
        ctx.tape = tape
        return U

    @staticmethod
    def backward(ctx, gU):
        want_c = ctx.needs_input_grad[1]
        dX, dc, _ = unwrap_backward(ctx.tape, gU.contiguous(), want_coherence=want_c)
        ctx.tape.free()
        return dX, dc, None
