"""torch.autograd wrappers: S(eps) and S(ridge edges) with the adjoint contraction as backward.

``scattering(eps, solver)`` returns the complex transmission matrix S for the
slab permittivity ``eps`` (float64, shape (h, nx), CPU or CUDA).  Any real
objective f written in torch on S then back-propagates to eps through the
library's single-elimination gradient (paper Eq. 1 with Eq. 3): the backward
receives torch's gradient g = dL/dS (torch's complex convention, which is
2 * conj of the Wirtinger derivative used in the paper, Gamma = df/dS), turns
it into Gamma = conj(g) / 2 and calls ``apf_grad_from_gamma`` with the fields
kept from the forward solve (the solve is repeated only if another solve on
the same solver replaced those fields in between).

This module only marshals tensors; every numerical step runs in libapf.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np
import torch

from . import apf as _apf


class _Scattering(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps: torch.Tensor, solver: "_apf.Solver", eps_sub: float, eps_clad: float, j0: int):
        eps_c = eps.detach().to(torch.float64).contiguous()
        solver.set_eps(eps_c, eps_sub, eps_clad, j0=j0)
        mi, mo = solver.channels()
        S = torch.empty((len(mo), len(mi)), dtype=torch.complex128, device=eps.device)
        solver.solve_S(out=S)
        ctx.version = solver.version
        ctx.save_for_backward(eps_c)
        ctx.bg = (eps_sub, eps_clad, j0)
        ctx.solver = solver
        ctx.eps_shape = eps_c.shape
        ctx.eps_device = eps.device
        ctx.eps_dtype = eps.dtype
        return S

    @staticmethod
    def backward(ctx, grad_S: torch.Tensor):
        gamma = (grad_S.conj() * 0.5).to(torch.complex128).contiguous()
        g = torch.empty(ctx.eps_shape, dtype=torch.float64, device=ctx.eps_device)
        solver = ctx.solver
        if solver.version != ctx.version:
            # another solve replaced the stored fields: redo this forward first
            (eps_c,) = ctx.saved_tensors
            solver.set_eps(eps_c, *ctx.bg[:2], j0=ctx.bg[2])
            mi, mo = solver.channels()
            solver.solve_S(out=torch.empty((len(mo), len(mi)), dtype=torch.complex128, device=eps_c.device))
        solver.grad_from_gamma(gamma, out=g)
        return g.to(ctx.eps_dtype), None, None, None, None


def scattering(eps: torch.Tensor, solver: "_apf.Solver", eps_sub: float, eps_clad: float,
               j0: int = -1) -> torch.Tensor:
    """S(eps) as a differentiable torch op (the solver keeps its grid and
    channel set; eps must have the solver's slab shape)."""
    return _Scattering.apply(eps, solver, eps_sub, eps_clad, j0)


class _RidgeScattering(torch.autograd.Function):
    @staticmethod
    def forward(ctx, edges: torch.Tensor, solver: "_apf.Solver", geom: tuple):
        e = edges.detach().to(torch.float64).contiguous()
        solver.set_ridges(e, *geom, eps_out=False)
        mi, mo = solver.channels()
        S = torch.empty((len(mo), len(mi)), dtype=torch.complex128, device=edges.device)
        solver.solve_S(out=S)
        ctx.version = solver.version
        ctx.save_for_backward(e)
        ctx.solver, ctx.geom = solver, geom
        ctx.edges_dtype = edges.dtype
        return S

    @staticmethod
    def backward(ctx, grad_S: torch.Tensor):
        (e,) = ctx.saved_tensors
        solver = ctx.solver
        if solver.version != ctx.version:
            solver.set_ridges(e, *ctx.geom, eps_out=False)
            mi, mo = solver.channels()
            solver.solve_S(out=torch.empty((len(mo), len(mi)), dtype=torch.complex128, device=e.device))
        gamma = (grad_S.conj() * 0.5).to(torch.complex128).contiguous()
        g_eps = torch.empty((solver.h, solver.nx), dtype=torch.float64, device=e.device)
        solver.grad_from_gamma(gamma, out=g_eps)
        g_e = torch.empty(e.shape[0], dtype=torch.float64, device=e.device)
        solver.ridge_grad(g_eps, out=g_e)
        return g_e.to(ctx.edges_dtype), None, None


def ridge_scattering(edges: torch.Tensor, solver: "_apf.Solver", h: int, eps_ridge: float, eps_bg: float,
                     eps_sub: float, eps_clad: float, mirror: bool = True, j0: int = -1) -> torch.Tensor:
    """S as a differentiable function of the ridge edge positions (paper
    Sec. 3, Eq. 5's design variables): forward = apf_set_ridges + solve_S,
    backward = the pixel adjoint contraction followed by apf_ridge_grad.  The
    solver keeps its grid and channel set."""
    return _RidgeScattering.apply(edges, solver, (h, eps_ridge, eps_bg, eps_sub, eps_clad, mirror, j0))


def relative_order_mask(m_in: Sequence[int], m_out: Sequence[int], orders: Sequence[int],
                        device=None) -> torch.Tensor:
    """Boolean (n_out, n_in) mask of the pairs with m_out - m_in in `orders`."""
    mi = np.asarray(m_in)[None, :]
    mo = np.asarray(m_out)[:, None]
    mask = np.zeros((mo.shape[0], mi.shape[1]), dtype=bool)
    for d in orders:
        mask |= (mo - mi) == d
    return torch.as_tensor(mask, device=device)


def splitter_loss(S: torch.Tensor, mask: torch.Tensor, target: float) -> torch.Tensor:
    """Eq. (5): sum over the masked pairs of (|S|^2 - t)^2."""
    p = (S.real ** 2 + S.imag ** 2)[mask]
    return ((p - target) ** 2).sum()
