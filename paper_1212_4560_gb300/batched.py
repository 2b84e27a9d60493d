"""Batched randomized GENP and its autograd binding.

``BatchedPlan`` wraps the genp_batched_* entry points: many independent
small systems solved in one persistent launch (graph-capturable run).
``GenpSolve`` is a ``torch.autograd.Function`` for X = A^{-1} B whose
backward is the library's adjoint through the GENP factors:
Lambda = L^{-T} U^{-T} G^T gX, dA = -Lambda X^T, dB = Lambda.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import CIRCULANT, FP32, FP64, GAUSSIAN, check
from .api import _ptr, _stream


class BatchedPlan:
    """genp_batched_plan for systems of orders ``sizes`` (each 1..1024)."""

    AUTOTUNE, FP64_ESCALATION = 1, 2

    def __init__(self, sizes, nrhs: int, kind: int = GAUSSIAN, a_dtype=torch.float64, max_iter: int = 10,
                 tol: float = 1e-14, autotune: bool = False, escalate: bool = False, stream=None):
        self.sizes = np.asarray(sizes, dtype=np.int64)
        self.count, self.nrhs, self.kind, self.a_dtype = len(self.sizes), int(nrhs), kind, a_dtype
        a_prec = FP64 if a_dtype == torch.float64 else FP32
        flags = (self.AUTOTUNE if autotune else 0) | (self.FP64_ESCALATION if escalate else 0)
        h = ctypes.c_void_p()
        arr = np.ascontiguousarray(self.sizes)
        check(_lib.load().genp_batched_plan_create(self.count, arr.ctypes.data_as(ctypes.c_void_p), self.nrhs, kind,
                                                   a_prec, int(max_iter), float(tol), flags, _stream(stream),
                                                   ctypes.byref(h)), "genp_batched_plan_create")
        self.handle = h
        self.mat_off = np.zeros(self.count + 1, dtype=np.int64)
        self.vec_off = np.zeros(self.count + 1, dtype=np.int64)
        check(_lib.load().genp_batched_layout(h, self.mat_off.ctypes.data_as(ctypes.c_void_p),
                                              self.vec_off.ctypes.data_as(ctypes.c_void_p)), "genp_batched_layout")

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.load().genp_batched_plan_destroy(self.handle)
            self.handle = None

    @property
    def mat_size(self) -> int:
        return int(self.mat_off[-1])

    @property
    def vec_size(self) -> int:
        return int(self.vec_off[-1])

    def block_size(self, n: int) -> int:
        return int(_lib.load().genp_batched_block_size(self.handle, int(n)))

    def pack(self, mats, vecs, device="cuda"):
        """Pools from lists of per-system (n, n) and (n, nrhs) tensors."""
        A = torch.cat([m.reshape(-1) for m in mats]).to(device=device, dtype=self.a_dtype)
        B = torch.cat([v.reshape(-1) for v in vecs]).to(device=device, dtype=torch.float64)
        return A.contiguous(), B.contiguous()

    def unpack_vec(self, pool, i):
        n = int(self.sizes[i])
        return pool[self.vec_off[i]:self.vec_off[i + 1]].view(n, self.nrhs)

    def run(self, seed: int, A_pool, B_pool, X_pool, stream=None) -> None:
        check(_lib.load().genp_batched_run(self.handle, int(seed), _ptr(A_pool), _ptr(B_pool), _ptr(X_pool),
                                           _stream(stream)), "genp_batched_run")

    def adjoint(self, A_pool, gX_pool, X_pool, dA_pool=None, dB_pool=None, stream=None) -> None:
        check(_lib.load().genp_batched_adjoint(self.handle, _ptr(A_pool), _ptr(gX_pool), _ptr(X_pool),
                                               _ptr(dA_pool), _ptr(dB_pool), _stream(stream)), "genp_batched_adjoint")

    def multipliers(self, G_pool=None, g_pool=None, stream=None) -> None:
        check(_lib.load().genp_batched_multipliers(self.handle, _ptr(G_pool), _ptr(g_pool), _stream(stream)),
              "genp_batched_multipliers")

    def status(self, stream=None) -> dict:
        c = self.count
        out = {"status": np.zeros(c, np.int32), "iters": np.zeros(c, np.int32), "eta0": np.zeros(c),
               "eta": np.zeros(c), "growth": np.zeros(c), "escalated": np.zeros(c, np.int32),
               "krylov": np.zeros(c, np.int32)}
        p = {k: v.ctypes.data_as(ctypes.c_void_p) for k, v in out.items()}
        check(_lib.load().genp_batched_status(self.handle, p["status"], p["iters"], p["eta0"], p["eta"],
                                              p["growth"], p["escalated"], p["krylov"], _stream(stream)),
              "genp_batched_status")
        return out


    PHASES = ("precondition", "factor", "invert", "solve", "residual", "gmres", "update")

    def profile(self, enable: bool = True) -> None:
        """Record per-phase SM cycles in later runs (genp_batched_profile)."""
        check(_lib.load().genp_batched_profile(self.handle, 1 if enable else 0), "genp_batched_profile")

    def profile_read(self, stream=None) -> dict:
        """SM cycles of the last run by phase, summed over the persistent CTAs."""
        cyc = np.zeros(len(self.PHASES))
        check(_lib.load().genp_batched_profile_read(self.handle, cyc.ctypes.data_as(ctypes.c_void_p),
                                                    _stream(stream)), "genp_batched_profile_read")
        return dict(zip(self.PHASES, cyc.tolist()))


_plans: dict = {}


def _plan_for(batch, n, nrhs, kind, dtype, max_iter, tol):
    key = (batch, n, nrhs, kind, dtype, max_iter, tol, torch.cuda.current_device())
    if key not in _plans:
        _plans[key] = BatchedPlan([n] * batch, nrhs, kind=kind, a_dtype=dtype, max_iter=max_iter, tol=tol)
    return _plans[key]


class GenpSolve(torch.autograd.Function):
    """X = A^{-1} B for a batch of systems (A: (batch, n, n), B: (batch, n, nrhs)),
    float32 A through the batched FP32 path; backward by the library's adjoint.
    ``kind``: GAUSSIAN or CIRCULANT multiplier; ``refine``: FP64 refinement steps."""

    @staticmethod
    def forward(ctx, A, B, kind=CIRCULANT, seed=0, refine=0, tol=1e-14):
        if A.dtype != torch.float32:
            raise TypeError("GenpSolve takes float32 A; use GenpSolve64 for float64")
        batch, n, _ = A.shape
        nrhs = B.shape[2]
        plan = _plan_for(batch, n, nrhs, kind, torch.float32, int(refine), float(tol))
        Ap = A.detach().contiguous().reshape(-1)
        Bp = B.detach().to(torch.float64).contiguous().reshape(-1)
        Xp = torch.empty_like(Bp)
        plan.run(seed, Ap, Bp, Xp)
        ctx.plan, ctx.shape, ctx.Bdtype = plan, (batch, n, nrhs), B.dtype
        ctx.save_for_backward(Ap, Xp)
        return Xp.view(batch, n, nrhs).to(B.dtype)

    @staticmethod
    def backward(ctx, gX):
        Ap, Xp = ctx.saved_tensors
        batch, n, nrhs = ctx.shape
        gXp = gX.detach().to(torch.float64).contiguous().reshape(-1)
        dA = torch.empty(batch * n * n, dtype=torch.float32, device=gX.device) if ctx.needs_input_grad[0] else None
        dB = torch.empty_like(gXp) if ctx.needs_input_grad[1] else None
        ctx.plan.adjoint(Ap, gXp, Xp, dA, dB)
        return (dA.view(batch, n, n) if dA is not None else None,
                dB.view(batch, n, nrhs).to(ctx.Bdtype) if dB is not None else None, None, None, None, None)


class GenpSolve64(torch.autograd.Function):
    """Float64 variant (one system at a time through genp_factor / genp_solve /
    genp_refine / genp_adjoint), used for exact gradient checks."""

    @staticmethod
    def forward(ctx, A, B, kind=CIRCULANT, seed=0, refine=8, tol=1e-16):
        from . import api
        batch = A.shape[0]
        X = torch.empty_like(B)
        saved = []
        for b in range(batch):
            x, info, G, F = api.solve_system(A[b].detach(), B[b].detach(), kind=kind, seed=seed + b,
                                             refine_steps=int(refine), tol=tol)
            X[b] = x
            saved.append((G, F))
        ctx.saved = saved
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, gX):
        from . import api
        (X,) = ctx.saved_tensors
        batch, n, nrhs = X.shape
        dA = torch.empty((batch, n, n), dtype=torch.float64, device=X.device)
        dB = torch.empty_like(X)
        for b, (G, F) in enumerate(ctx.saved):
            api.adjoint(F, G, gX[b].contiguous(), X[b].contiguous(), dA[b], dB[b])
        return dA, dB, None, None, None, None


def genp_solve(A, B, kind=CIRCULANT, seed=0, refine=None):
    """Differentiable randomized-GENP solve: float32 batches go through the
    batched kernel (FP32 factors; forward and adjoint refined in FP64 unless
    refine=0), float64 through the single-system path."""
    if A.dtype == torch.float64:
        return GenpSolve64.apply(A, B, kind, seed, 8 if refine is None else refine)
    return GenpSolve.apply(A, B, kind, seed, 10 if refine is None else refine)
