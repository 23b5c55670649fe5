"""Deep-unfolded FWI (DUFWI) around the GPU misfit gradient (Sec. III, Eqs. 9-10).

Each iteration k computes the data-fidelity gradient g_k = dJ/dC at the current estimate C_k
(Eq. 6) with the library's adjoint kernels. A per-iteration network N_k turns (C_k, g_k) into
an update H_k, and C_{k+1} = C_k + H_k (Eq. 9). Training is block-wise (Sec. III-B, Eq. 10).
Iteration k's gradients are computed once for the whole training set, N_k is fitted alone to
the SoS-map MSE, and its outputs become the inputs of iteration k+1. No gradient flows back
through the physics or through earlier blocks.

End-to-end training (``train_end_to_end``), which the paper avoids, backpropagates the loss
through every iteration, the physics included. Then dL/dC_k picks up the term H_k gbar_k, where
gbar_k = dL/dg_k and H_k is the Hessian of the misfit at C_k. ``data_gradient_differentiable``
supplies it: g_k = dJ/dC is an autograd node whose backward is the exact Hessian-vector product
of ``dufwi_hvp`` (the Hessian is symmetric, so the VJP of g is H gbar).

N_k is a small convolutional net: three 3 x 3 layers with 32 channels and ReLU in between. Its
inputs are the SoS offset by 1400 m/s and scaled (Sec. V), and the gradient normalised by its
max |.| per map. Its output is rescaled to m/s. The convolutions run in torch (cuDNN); they are
library dense contractions, not part of the hot path.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import torch
import torch.nn as nn

from . import dufwi

SOS_OFFSET = 1400.0    # m/s, subtracted from the SoS input (Sec. V)
SOS_SCALE = 200.0      # m/s per unit of the normalised SoS input and of the network output


class UpdateNet(nn.Module):
    """N_k: (C_k, g_k) -> H_k, three 3 x 3 convolutions (2 -> 32 -> 32 -> 1), ReLU in between."""

    def __init__(self, channels: int = 32):
        super().__init__()
        self.body = nn.Sequential(
            nn.Conv2d(2, channels, 3, padding=1), nn.ReLU(),
            nn.Conv2d(channels, channels, 3, padding=1), nn.ReLU(),
            nn.Conv2d(channels, 1, 3, padding=1))
        nn.init.zeros_(self.body[-1].weight)
        nn.init.zeros_(self.body[-1].bias)

    def forward(self, sos: torch.Tensor, grad: torch.Tensor) -> torch.Tensor:
        """H_k in the dtype of sos; the net itself runs in the dtype of its parameters."""
        g = grad / grad.abs().amax(dim=(-2, -1), keepdim=True).clamp_min(1e-30)
        x = torch.stack([(sos - SOS_OFFSET) / SOS_SCALE, g], dim=1).to(self.body[0].weight.dtype)
        return (SOS_SCALE * self.body(x)[:, 0]).to(sos.dtype)


@dataclass
class Physics:
    """Everything the gradient needs besides the maps: grid, pulse, array, observed data."""
    problem: dufwi.Problem
    wavelet: torch.Tensor
    geom: dufwi.Geometry


def data_gradient(phys: Physics, sos: torch.Tensor, cd_obs: torch.Tensor, chunk: int = 8):
    """g_k = dJ/dC for a batch of maps (Eq. 6), in chunks of `chunk` maps per library call."""
    J, g = [], []
    for i in range(0, sos.shape[0], chunk):
        Ji, gi = dufwi.misfit_gradient(phys.problem, sos[i:i + chunk].contiguous(), phys.wavelet, phys.geom,
                                       cd_obs[i:i + chunk].contiguous())
        J.append(Ji)
        g.append(gi)
    return torch.cat(J), torch.cat(g)


class _DataGradient(torch.autograd.Function):
    """g = dJ/dC (Eq. 6) as a function of C; backward: H gbar by dufwi_hvp."""

    @staticmethod
    def forward(ctx, sos, cd_obs, phys, chunk):
        _, g = data_gradient(phys, sos.detach(), cd_obs.detach(), chunk)
        ctx.save_for_backward(sos, cd_obs)
        ctx.phys = phys
        ctx.chunk = chunk
        return g

    @staticmethod
    def backward(ctx, gbar):
        if not ctx.needs_input_grad[0]:
            return None, None, None, None
        sos, cd_obs = ctx.saved_tensors
        phys = ctx.phys
        # H gbar = s H (gbar / s), s = max |gbar| per map: a unit-scale direction keeps the FP32
        # sweeps in range whatever the scale of the cotangent
        s = gbar.abs().amax(dim=(-2, -1), keepdim=True).clamp_min(1e-30)
        v = (gbar / s).contiguous()
        out = []
        for i in range(0, sos.shape[0], ctx.chunk):
            out.append(dufwi.hvp(phys.problem, sos[i:i + ctx.chunk].detach().contiguous(), phys.wavelet, phys.geom,
                                 cd_obs[i:i + ctx.chunk].detach().contiguous(), v[i:i + ctx.chunk]))
        return torch.cat(out) * s, None, None, None


def data_gradient_differentiable(phys: Physics, sos: torch.Tensor, cd_obs: torch.Tensor, chunk: int = 8):
    """g_k = dJ/dC as an autograd node: backpropagating through it applies the exact Hessian."""
    return _DataGradient.apply(sos, cd_obs, phys, chunk)


class UnfoldedFWI(nn.Module):
    """K unfolded iterations C_{k+1} = C_k + N_k(C_k, g_k) (Eq. 9)."""

    def __init__(self, K: int = 5, channels: int = 32):
        super().__init__()
        self.nets = nn.ModuleList(UpdateNet(channels) for _ in range(K))

    @torch.no_grad()
    def infer(self, phys: Physics, sos0: torch.Tensor, cd_obs: torch.Tensor, timings: list | None = None):
        """Inference from C_0 (a homogeneous map, Sec. III-A); returns all estimates C_0..C_K."""
        out = [sos0]
        c = sos0
        for k, net in enumerate(self.nets):
            if timings is not None:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            _, g = data_gradient(phys, c, cd_obs)
            c = c + net(c, g)
            if timings is not None:
                torch.cuda.synchronize()
                timings.append(time.perf_counter() - t0)
            out.append(c)
        return out

    def train_blockwise(self, phys: Physics, sos0: torch.Tensor, cd_obs: torch.Tensor, sos_gt: torch.Tensor,
                        epochs: int = 40, batch: int = 32, lrs=(1e-4, 1e-4, 5e-5, 1e-5, 1e-5), log=None):
        """Block-wise training (Sec. III-B). For each k: compute g_k for the whole set once, fit
        N_k with Adam on the SoS MSE of C_k + N_k(C_k, g_k) (Eq. 10), then advance the set to
        C_{k+1} with N_k in inference mode. Returns the training losses per block and epoch."""
        c = sos0
        history = []
        for k, net in enumerate(self.nets):
            with torch.no_grad():
                _, g = data_gradient(phys, c, cd_obs)
            opt = torch.optim.Adam(net.parameters(), lr=lrs[min(k, len(lrs) - 1)])
            losses = []
            for _ in range(epochs):
                perm = torch.randperm(c.shape[0], device=c.device)
                tot = 0.0
                for i in range(0, c.shape[0], batch):
                    idx = perm[i:i + batch]
                    pred = c[idx] + net(c[idx], g[idx])
                    loss = ((pred - sos_gt[idx]) ** 2).mean()
                    opt.zero_grad()
                    loss.backward()
                    opt.step()
                    tot += float(loss.detach()) * idx.numel()
                losses.append(tot / c.shape[0])
            history.append(losses)
            if log:
                log("block %d: mse %.4g -> %.4g" % (k, losses[0], losses[-1]))
            with torch.no_grad():
                c = c + net(c, g)
        return history

    def train_end_to_end(self, phys: Physics, sos0: torch.Tensor, cd_obs: torch.Tensor, sos_gt: torch.Tensor,
                         epochs: int = 20, batch: int = 8, lr: float = 1e-4, log=None):
        """End-to-end training: every N_k at once, on the SoS MSE of C_K (Eq. 10 at the last
        iteration), with gradients through the K data gradients (exact Hessian-vector products)
        as well as through the nets. Returns the training loss per epoch."""
        opt = torch.optim.Adam(self.parameters(), lr=lr)
        losses = []
        for _ in range(epochs):
            perm = torch.randperm(sos0.shape[0], device=sos0.device)
            tot = 0.0
            for i in range(0, sos0.shape[0], batch):
                idx = perm[i:i + batch]
                c = sos0[idx]
                obs = cd_obs[idx]
                for net in self.nets:
                    g = data_gradient_differentiable(phys, c, obs)
                    c = c + net(c, g)
                loss = ((c - sos_gt[idx]) ** 2).mean()
                opt.zero_grad()
                loss.backward()
                opt.step()
                tot += float(loss.detach()) * idx.numel()
            losses.append(tot / sos0.shape[0])
            if log:
                log("end-to-end epoch %d: mse %.4g" % (len(losses), losses[-1]))
        return losses
