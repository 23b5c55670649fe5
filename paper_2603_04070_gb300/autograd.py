"""Differentiable forward model: the simulator behind ``torch.autograd.Function``.

The forward pass is ``dufwi_forward_save``: the channel data M = F(C) of every shot (Eqs. 2-4),
with the checkpoint snapshots (or the whole history) kept in a workspace. The backward pass is
``dufwi_backward``, the hand-written discrete adjoint: for any upstream cotangent dL/dM it
returns dL/dC = (dM/dC)^T dL/dM. The same kernels compute the misfit gradient of Eq. 6; this
wrapper exposes them to any loss built on the channel data. An example is the block-wise
DUFWI training of Sec. III-B, where g_k feeds N_theta_k.

Gradients flow to the SoS maps only. The pulse, the density and the geometry are constants.
Calling ``backward`` twice needs ``retain_graph=True``; the saved workspace is reused.
Forward-mode AD (``torch.autograd.forward_ad``) uses the linearised Born simulation
(``dufwi_jvp``). ``hvp_gauss_newton`` combines it with the adjoint into Gauss-Newton
Hessian-vector products of the misfit.

Double backward: with ``create_graph=True`` the vector-Jacobian product is itself a node,
G(C, w) = (dM/dC)^T w, whose backward is ``dufwi_second_order``. For a cotangent v of G it
returns the Born data (dM/dC) v for w and the second-order term d/dC[(dM/dC)^T w] . v for C, so
``torch.autograd.grad`` of a gradient gives exact Hessian-vector products of any loss built on
the channel data (``hvp`` does this for the misfit). Third derivatives are not provided: a
second backward with ``create_graph=True`` raises.
"""
from __future__ import annotations

import torch

from . import dufwi


class _Simulate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sos, wavelet, problem, geom):
        cd, ws = dufwi.forward_save(problem, sos.detach().contiguous(), wavelet.detach().contiguous(), geom)
        ctx.save_for_backward(sos, wavelet)
        ctx.save_for_forward(sos, wavelet)
        ctx.workspace = ws
        ctx.problem = problem
        ctx.geom = geom
        return cd

    @staticmethod
    def jvp(ctx, sos_t, wavelet_t, problem_t, geom_t):
        sos, wavelet = ctx.saved_tensors
        if sos_t is None:
            return None
        return dufwi.jvp(ctx.problem, sos.detach().contiguous(), wavelet.detach().contiguous(), ctx.geom,
                         sos_t.contiguous())

    @staticmethod
    def backward(ctx, cd_grad):
        sos, wavelet = ctx.saved_tensors
        grad = None
        if ctx.needs_input_grad[0]:
            if torch.is_grad_enabled():   # create_graph: the product must be differentiable in (C, w)
                grad = _VJP.apply(sos, cd_grad, wavelet, ctx.problem, ctx.geom, ctx.workspace)
            else:
                grad = dufwi.backward(ctx.problem, sos.detach().contiguous(), wavelet.detach().contiguous(),
                                      ctx.geom, cd_grad.contiguous(), ctx.workspace)
        return grad, None, None, None


class _VJP(torch.autograd.Function):
    """G = (dM/dC)^T w as a function of C and w (the differentiable form of the backward pass)."""

    @staticmethod
    def forward(ctx, sos, cd_grad, wavelet, problem, geom, workspace):
        sos_d = sos.detach().contiguous()
        w_d = cd_grad.detach().contiguous()
        grad = dufwi.backward(problem, sos_d, wavelet.detach().contiguous(), geom, w_d, workspace)
        ctx.save_for_backward(sos, cd_grad, wavelet)
        ctx.problem = problem
        ctx.geom = geom
        return grad

    @staticmethod
    def backward(ctx, v):
        if torch.is_grad_enabled():
            raise RuntimeError("dufwi autograd: third derivatives are not provided (the second backward must not "
                               "use create_graph=True)")
        sos, cd_grad, wavelet = ctx.saved_tensors
        so, dcd = dufwi.second_order(ctx.problem, sos.detach().contiguous(), wavelet.detach().contiguous(), ctx.geom,
                                     cd_grad.detach().contiguous(), v.contiguous())
        return (so if ctx.needs_input_grad[0] else None), (dcd if ctx.needs_input_grad[1] else None), \
            None, None, None, None


def simulate(problem: dufwi.Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: dufwi.Geometry) -> torch.Tensor:
    """Channel data ``[n_maps][n_tx][nt][n_rx]``, differentiable with respect to ``sos``."""
    return _Simulate.apply(sos, wavelet, problem, geom)


def misfit(problem: dufwi.Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: dufwi.Geometry,
           cd_obs: torch.Tensor) -> torch.Tensor:
    """Per-map data misfit J = sum (M - M_obs)^2 (Eq. 5 with lambda = 0), differentiable in sos."""
    r = simulate(problem, sos, wavelet, geom) - cd_obs
    return (r * r).sum(dim=(1, 2, 3), dtype=torch.float64)


def hvp_gauss_newton(problem: dufwi.Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: dufwi.Geometry,
                     v: torch.Tensor) -> torch.Tensor:
    """Gauss-Newton Hessian-vector product of the misfit J = sum (M - M_obs)^2: H v = 2 J^T (J v),
    with J = dM/dC (Born forward, then the adjoint)."""
    sos = sos.detach().contiguous()
    wavelet = wavelet.detach().contiguous()
    _, ws = dufwi.forward_save(problem, sos, wavelet, geom)
    dcd = dufwi.jvp(problem, sos, wavelet, geom, v.contiguous())
    return dufwi.backward(problem, sos, wavelet, geom, 2.0 * dcd, ws)


def hvp(problem: dufwi.Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: dufwi.Geometry, cd_obs: torch.Tensor,
        v: torch.Tensor) -> torch.Tensor:
    """Exact Hessian-vector product of the misfit J = sum (M - M_obs)^2 per map, by double
    backward through the autograd wrapper: H v = 2 J^T (J v) + d/dC[J^T 2 (M - M_obs)] . v."""
    c = sos.detach().clone().requires_grad_(True)
    with torch.enable_grad():
        J = misfit(problem, c, wavelet, geom, cd_obs).sum()
        (g,) = torch.autograd.grad(J, c, create_graph=True)
        (Hv,) = torch.autograd.grad(g, c, grad_outputs=v)
    return Hv
