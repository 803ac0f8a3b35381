"""torch.autograd integration of the multigrid solver.

``DMGSolve.apply(q, D, mu, solver, recompute)`` returns u = A(D, mu)^{-1} q
computed by the C ABI (``dmg_solve``). Its backward is the analytically
derived pull-back of arXiv 2608.00760 Sec. 2.4 (the transposed V-cycle,
``dmg_vjp``), which also returns the gradients w.r.t. D and mu through the
adjoint state; its forward-mode rule is the push-forward of Sec. 2.3
(``dmg_jvp``). With ``recompute=True`` the solution is not kept for backward:
it is solved again from q when a derivative needs it, trading one solve for
one field of memory per call.

``solve(q, D, mu, h, **params)`` is the user-facing function: it keeps a small
cache of solver contexts (keyed by the identity and version of D and mu, the
shape and the parameters) so that repeated calls with the same coefficients
reuse the coefficient hierarchy.
"""
from __future__ import annotations

import weakref

import torch

from . import dmg


def _c(x):
    return None if x is None else x.contiguous()


class DMGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, D, mu, solver, recompute=False):
        q = q.contiguous()
        u = solver.solve(q)
        ctx.solver = solver
        ctx.recompute = bool(recompute)
        ctx.save_for_backward(q if recompute else u)
        # forward mode (jvp) runs right after forward and needs u
        ctx.fwd = q if recompute else u
        return u

    @staticmethod
    def backward(ctx, w):
        (saved,) = ctx.saved_tensors
        need = tuple(bool(x) for x in ctx.needs_input_grad[:3])
        if not any(need):
            return None, None, None, None, None
        u = ctx.solver.solve(saved) if ctx.recompute else saved
        qb, Db, mb = ctx.solver.vjp(u, w.contiguous(), need=need)
        return qb, Db, mb, None, None

    @staticmethod
    def jvp(ctx, dq, dD, dmu, _solver=None, _recompute=None):
        u = ctx.solver.solve(ctx.fwd) if ctx.recompute else ctx.fwd
        ctx.fwd = None
        if dD is None and dmu is None:
            if dq is None:
                return torch.zeros_like(u)
            return ctx.solver.jvp(None, dq=_c(dq))
        return ctx.solver.jvp(u, dq=_c(dq), dD=_c(dD), dmu=_c(dmu))


class DMGSolveUnrolled(torch.autograd.Function):
    """u = S_m(q; D, mu), m fixed FP64 V-cycles from u = 0 (the solver must be
    set up with fixed_cycles = m), whose backward is the exact derivative of
    the m-cycle iteration through every iterate and the coarsened coefficients
    (dmg_vjp_unrolled). Only q is kept for backward: the iterates are recomputed
    there from checkpoints every `stride` cycles (0: about sqrt(m))."""

    @staticmethod
    def forward(ctx, q, D, mu, solver, m, stride=0):
        q = q.contiguous()
        u = solver.solve(q)
        ctx.solver, ctx.m, ctx.stride = solver, int(m), int(stride)
        ctx.save_for_backward(q)
        return u

    @staticmethod
    def backward(ctx, w):
        (q,) = ctx.saved_tensors
        _, qb, Db, mb = ctx.solver.vjp_unrolled(q, w.contiguous(), ctx.m, ctx.stride)
        need = ctx.needs_input_grad
        return (qb if need[0] else None, Db if need[1] else None, mb if need[2] else None, None, None, None)


class DMGResponse(torch.autograd.Function):
    """L_e = M(mu S(q)), the application's forward model (Sec. 2.5.3, Eq.
    response), with its pull-back (dmg_response_vjp) and push-forward
    (dmg_response_jvp)."""

    @staticmethod
    def forward(ctx, q, D, mu, solver, edge):
        Le, u = solver.response(q.contiguous(), edge)
        ctx.solver, ctx.edge = solver, float(edge)
        ctx.save_for_backward(u)
        ctx.fwd = u
        return Le

    @staticmethod
    def backward(ctx, rbar):
        (u,) = ctx.saved_tensors
        qb, Db, mb = ctx.solver.response_vjp(u, rbar.contiguous(), ctx.edge)
        need = ctx.needs_input_grad
        return (qb if need[0] else None, Db if need[1] else None, mb if need[2] else None, None, None)

    @staticmethod
    def jvp(ctx, dq, dD, dmu, _solver=None, _edge=None):
        u = ctx.fwd
        ctx.fwd = None
        return ctx.solver.response_jvp(u, ctx.edge, dq=_c(dq), dD=_c(dD), dmu=_c(dmu))


class _Cache:
    """Solver contexts for recently used coefficient fields.

    An entry holds weak references to the D and mu tensors it was built from and
    their versions; it matches only the same live tensor objects, unchanged (a
    new tensor that happens to reuse a freed address never matches).

    Dropping an entry (eviction, dead tensors, clear) only drops the cache's
    reference: an autograd graph that still needs the solver for its backward
    or forward-mode rule keeps it alive, and the solver's context is destroyed
    when the last reference goes (Solver.__del__).
    """

    def __init__(self, size=8):
        self.size = size
        self.items = []   # (Dref, muref, Dver, muver, key, solver), most recent last

    def get(self, D, mu, h, params):
        key = (tuple(D.shape), float(h), tuple(sorted(params.items())), str(D.device))
        for n, (dr, mr, dv, mv, k, s) in enumerate(self.items):
            if dr() is D and mr() is mu and dv == D._version and mv == mu._version and k == key:
                self.items.append(self.items.pop(n))
                return s
        s = dmg.Solver(D.detach(), mu.detach(), h, **params)
        self.items.append((weakref.ref(D), weakref.ref(mu), D._version, mu._version, key, s))
        self.items = [e for e in self.items if e[0]() is not None and e[1]() is not None or e[5] is s]
        while len(self.items) > self.size:
            self.items.pop(0)
        return s

    def clear(self):
        self.items = []


_cache = _Cache()


def solve(q, D, mu, h, recompute=False, unrolled=False, stride=0, **params):
    """u = A(D, mu)^{-1} q, differentiable w.r.t. q, D and mu (reverse and forward mode).

    q, D, mu: float64 CUDA tensors of shape (nz, ny, nx) over all vertices (or
    (B, nz, ny, nx) for a batch).
    params: dmg_params fields (rtol, precision, nu1, nu2, face_mean, ...).
    unrolled=True (with fixed_cycles=m in params): u = S_m(q), the m-cycle
    iterate, and its backward is the exact derivative of the m-cycle solver
    (dmg_vjp_unrolled) instead of the converged-solution gradient.
    """
    if unrolled:
        m = int(params.get("fixed_cycles", 0))
        if m < 1:
            raise ValueError("unrolled=True needs fixed_cycles = m >= 1")
        s = _cache.get(D, mu, h, params)
        return DMGSolveUnrolled.apply(q, D, mu, s, m, stride)
    s = _cache.get(D, mu, h, params)
    return DMGSolve.apply(q, D, mu, s, recompute)


def response(q, D, mu, h, edge, **params):
    """L_e = M(mu S(q)) with the edge mask of depth `edge` (Eq. response),
    differentiable w.r.t. q, D and mu (reverse and forward mode)."""
    s = _cache.get(D, mu, h, params)
    return DMGResponse.apply(q, D, mu, s, edge)


def clear_cache():
    _cache.clear()
