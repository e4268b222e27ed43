"""Differentiable hybrid step: the CUDA engine's forward and hand-written adjoint (include/genga.h,
genga_adj_*) behind a torch.autograd.Function.

Argument marshalling only: every step of the forward and of the backward runs in the library's
kernels on the tensors' device memory, on torch's current CUDA stream.

    eng = AdjointEngine(m0, G, dt, order=2, ckpt_every=50)      # m0: central masses [B]
    x1, v1 = hybrid_steps(x0, v0, m, eng, n_steps)              # x0, v0 [B, N, 3], m [B, N]
    loss(x1, v1).backward()                                     # gradients on x0, v0, m

Inputs are heliocentric positions and velocities (float64, CUDA); merging is off (the engine
integrates through close passes), and every discrete decision of the step is frozen from the
forward pass (see genga_adj_init).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import genga


def _ptr(t: torch.Tensor):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise genga.GengaError("adjoint engine tensors must be contiguous float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


class AdjointEngine:
    """One engine for B systems of N bodies (created on first use, sized by the first inputs)."""

    def __init__(self, m0, G, dt, order=2, ckpt_every=50):
        self.m0 = np.ascontiguousarray(np.atleast_1d(m0), dtype=np.float64)
        self.G, self.dt, self.order, self.ckpt_every = float(G), float(dt), int(order), int(ckpt_every)
        self._h = None
        self._shape = None
        self.generation = 0

    def _ensure(self, B, N):
        if self._h is not None and self._shape == (B, N):
            return
        if len(self.m0) != B:
            raise genga.GengaError(f"m0 has {len(self.m0)} entries for {B} systems")
        self.close()
        h = C.c_void_p()
        genga._check(genga.lib().genga_adj_init(C.byref(h), B, N, self.m0.ctypes.data_as(genga._D), self.G,
                                                self.dt, self.order, self.ckpt_every), "genga_adj_init")
        self._h, self._shape = h, (B, N)

    def close(self):
        if self._h is not None:
            genga.lib().genga_adj_free(self._h)
            self._h = None

    __del__ = close

    def _stream(self):
        genga._check(genga.lib().genga_adj_set_stream(self._h, C.c_void_p(torch.cuda.current_stream().cuda_stream)),
                     "genga_adj_set_stream")

    def forward(self, x, v, m, n_steps):
        B, N, _ = x.shape
        self._ensure(B, N)
        self._stream()
        xo, vo = torch.empty_like(x), torch.empty_like(v)
        genga._check(genga.lib().genga_adj_forward(self._h, int(n_steps), _ptr(x), _ptr(v), _ptr(m), _ptr(xo),
                                                   _ptr(vo)), "genga_adj_forward")
        self.generation += 1
        return xo, vo

    def backward(self, xbar, vbar):
        self._stream()
        B, N = self._shape
        dev = xbar.device
        gx = torch.empty((B, N, 3), dtype=torch.float64, device=dev)
        gv = torch.empty((B, N, 3), dtype=torch.float64, device=dev)
        gm = torch.empty((B, N), dtype=torch.float64, device=dev)
        genga._check(genga.lib().genga_adj_backward(self._h, _ptr(xbar), _ptr(vbar), _ptr(gx), _ptr(gv), _ptr(gm)),
                     "genga_adj_backward")
        return gx, gv, gm

    def status(self):
        code = C.c_int(0)
        genga._check(genga.lib().genga_adj_status(self._h, C.byref(code)), "genga_adj_status")
        return code.value


class HybridSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, v, m, engine: AdjointEngine, n_steps: int):
        x, v, m = x.contiguous(), v.contiguous(), m.contiguous()
        xo, vo = engine.forward(x, v, m, n_steps)
        ctx.engine = engine
        ctx.generation = engine.generation
        return xo, vo

    @staticmethod
    def backward(ctx, gxo, gvo):
        eng = ctx.engine
        if eng.generation != ctx.generation:
            raise genga.GengaError("the adjoint engine ran another forward pass before this backward pass")
        if gxo is None:
            gxo = torch.zeros(eng._shape + (3,), dtype=torch.float64, device=gvo.device)
        if gvo is None:
            gvo = torch.zeros(eng._shape + (3,), dtype=torch.float64, device=gxo.device)
        gx, gv, gm = eng.backward(gxo.contiguous(), gvo.contiguous())
        return gx, gv, gm, None, None


def hybrid_steps(x, v, m, engine: AdjointEngine, n_steps: int):
    """n_steps hybrid steps of every system; differentiable with respect to x, v and m."""
    return HybridSteps.apply(x, v, m, engine, n_steps)
