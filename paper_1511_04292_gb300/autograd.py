"""Differentiable SRJ solve: torch.autograd.Function over the C ABI.

u = S(f, g) solves A_h u = h^2 f + B g (5-/7-point Dirichlet Laplacian, ghost
layer = boundary data g).  The backward pass is the library's srj_gradient:
one adjoint SRJ solve (A_h is symmetric) and one kernel that forms dL/df and
dL/dg; no iterate of the forward solve is stored (implicit differentiation of
the converged solve).  Both passes run in the native library; this module only
marshals tensors.
"""
from __future__ import annotations

import ctypes

import torch

from . import Plan, _dev_ptr, _stream_ptr
from ._native import Stats, check


class SRJSolve(torch.autograd.Function):
    """u = SRJSolve.apply(f, g, plan, tol, max_cycles[, adjoint_tol]).

    f, g: float64 CUDA tensors in the plan's padded shape; the ghost layer of g
    is the Dirichlet data (its interior is ignored), the ghost layer of f is
    ignored.  Returns u (padded; its ghost layer equals g's).  Gradients flow to
    f (interior) and g (ghost layer).  The adjoint solve of the backward pass
    runs to adjoint_tol (default: tol).  A solve that stops at its
    floating-point floor above its tolerance (stats["stagnated"]) is accepted;
    other failures raise.  The adjoint's right-hand side dL/du is smooth when u
    is, and then its FP64 floor, relative to that right-hand side, is about
    the unit roundoff times cond(A) ~ 2 / kappa_min (2e-10 at 2048^2), well
    above the forward solve's: an adjoint_tol near that floor stops the
    backward pass where further cycles no longer change the gradient.
    """

    @staticmethod
    def forward(ctx, f, g, plan, tol, max_cycles, adjoint_tol=None):
        u = g.detach().clone().contiguous()
        inner = tuple(slice(1, -1) for _ in range(u.dim()))
        u[inner] = 0.0
        ctx.stats = plan.solve(f.detach().contiguous(), u, tol, max_cycles, raise_on_fail=False)
        if ctx.stats["status"] != 0 and not ctx.stats["stagnated"]:
            check(ctx.stats["status"])
        ctx.plan, ctx.tol, ctx.max_cycles = plan, tol, max_cycles
        ctx.adjoint_tol = tol if adjoint_tol is None else adjoint_tol
        return u

    @staticmethod
    def backward(ctx, grad_u):
        plan = ctx.plan
        gu = grad_u.detach().contiguous()
        lam = torch.zeros_like(gu)
        gf = torch.empty_like(gu)
        gg = torch.empty_like(gu)
        st = Stats()
        rc = plan._lib.srj_gradient(plan._h, _dev_ptr(gu, plan.shape, "grad_u"), _dev_ptr(lam, plan.shape, "lambda"),
                                    _dev_ptr(gf, plan.shape, "grad_f"), _dev_ptr(gg, plan.shape, "grad_g"),
                                    float(ctx.adjoint_tol), int(ctx.max_cycles), _stream_ptr(None), ctypes.byref(st))
        ctx.adjoint_stats = st.as_dict()
        if rc != 0 and not st.stagnated:
            check(rc)
        return gf, gg, None, None, None, None


def srj_solve(f, g, plan: Plan, tol=1e-12, max_cycles=100000, adjoint_tol=None):
    """Functional form of SRJSolve."""
    return SRJSolve.apply(f, g, plan, tol, max_cycles, adjoint_tol)
