"""Multi-GPU data parallelism over shots (one process per GPU).

Shots, i.e. (map, transmit) pairs, are independent (Sec. II-A; Eq. 4), so the path shards
without communication:

* ``shard_maps``: each rank takes a contiguous block of maps and computes their misfits and
  gradients alone. This is weak scaling with no collective on the data path; the benchmark
  runs this way.
* ``sharded_misfit_gradient``: the transmits of the same maps are split across ranks. The one
  exchange is then a sum of the per-rank partial misfits and gradients, reduced in FP64
  (``gradient_allreduce``). The misfit and gradient are sums over transmits (Eqs. 5-6), so the
  reduced result equals the single-rank one up to FP64 summation order.
* ``sharded_hvp``: the same split for exact Hessian-vector products (``dufwi_hvp``): H v, the
  misfit and the gradient are all sums over transmits, reduced together.

The compute callback defaults to the CUDA library on the rank's device. Tests substitute the CPU
oracle and run the collective on ``gloo`` ranks.
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import torch
import torch.distributed as dist


def block_range(n: int, world: int, rank: int) -> range:
    """Contiguous block of [0, n) owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %d of %d" % (rank, world))
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def shard_maps(n_maps: int, world: int, rank: int) -> range:
    return block_range(n_maps, world, rank)


def shard_transmits(n_tx: int, world: int, rank: int) -> range:
    return block_range(n_tx, world, rank)


def gradient_allreduce(misfit: torch.Tensor, grad: torch.Tensor, group=None):
    """Sum per-rank partial misfits [B] and gradients [B, nz, nx] over ranks in FP64 (the one
    collective of transmit sharding). Partial gradients may come in FP64 (the library's FP64
    output) or FP32; the sum is FP64 and is rounded to FP32 once, at the end. Returns (misfit FP64,
    gradient FP32) on the inputs' device."""
    if not dist.is_available() or not dist.is_initialized():
        return misfit.to(torch.float64), grad.to(torch.float32)
    m = misfit.to(torch.float64).contiguous()
    g = grad.to(torch.float64).contiguous()
    dist.all_reduce(m, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return m, g.to(torch.float32)


def _cuda_compute(problem, sos, wavelet, geom, cd_obs):
    """The rank's partial misfit and gradient, the gradient left in FP64 (dufwi_misfit_gradient_fp64),
    so that the sum over ranks is FP64 from the library's cross-transmit sum to the final rounding."""
    from . import dufwi
    grad = torch.empty(sos.shape, dtype=torch.float64, device=sos.device)
    return dufwi.misfit_gradient(problem, sos, wavelet, geom, cd_obs, grad=grad)


def _transmit_shard(geom, wavelet, cd_obs, group):
    """This rank's block of transmits: (index array, sub-geometry, pulse, observed data)."""
    from .dufwi import Geometry
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    sel = shard_transmits(geom.n_tx, world, rank)
    idx = np.arange(sel.start, sel.stop)
    sub = Geometry(geom.elem_ix, geom.elem_iz, geom.tx_elem[idx], geom.rx_elem[idx], geom.wavelet_per_tx)
    w = wavelet[sel.start:sel.stop] if geom.wavelet_per_tx else wavelet
    return idx, sub, w, cd_obs[:, sel.start:sel.stop].contiguous()


def _cuda_hvp(problem, sos, wavelet, geom, cd_obs, v):
    from . import dufwi
    return dufwi.hvp(problem, sos, wavelet, geom, cd_obs, v, return_all=True)


def sharded_hvp(problem, sos: torch.Tensor, wavelet: torch.Tensor, geom, cd_obs: torch.Tensor, v: torch.Tensor, *,
                group=None, compute: Callable | None = None):
    """Exact Hessian-vector product H v of the misfit, with the misfit and gradient, for every map,
    the transmits split over the ranks of ``group`` as in ``sharded_misfit_gradient``.
    ``compute(problem, sos, wavelet, sub_geom, sub_cd_obs, v) -> (Hv, J, g)`` runs on the rank.
    Returns (Hv FP32, J FP64, g FP32), each summed over ranks in FP64."""
    idx, sub, w, obs = _transmit_shard(geom, wavelet, cd_obs, group)
    compute = compute or _cuda_hvp
    if len(idx) == 0:   # more ranks than transmits: contribute zeros
        hv = torch.zeros_like(sos)
        J = torch.zeros(sos.shape[0], dtype=torch.float64, device=sos.device)
        g = torch.zeros_like(sos)
    else:
        hv, J, g = compute(problem, sos, w, sub, obs, v)
    J, g = gradient_allreduce(J, g, group)
    if dist.is_available() and dist.is_initialized():
        h = hv.to(torch.float64).contiguous()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        hv = h
    return hv.to(torch.float32), J, g


def sharded_misfit_gradient(problem, sos: torch.Tensor, wavelet: torch.Tensor, geom, cd_obs: torch.Tensor, *,
                            group=None, compute: Callable | None = None):
    """Misfit and gradient of every map with the transmits split over the ranks of `group`.

    ``geom`` is the full geometry; each rank keeps the transmits of its block, the matching
    rows of the receive table and of ``cd_obs [maps][n_tx][nt][n_rx]`` (and of a per-transmit
    pulse). ``compute(problem, sos, wavelet, sub_geom, sub_cd_obs) -> (J, g)`` runs on the rank.
    """
    idx, sub, w, obs = _transmit_shard(geom, wavelet, cd_obs, group)
    compute = compute or _cuda_compute
    if len(idx) == 0:   # more ranks than transmits: contribute zeros
        J = torch.zeros(sos.shape[0], dtype=torch.float64, device=sos.device)
        g = torch.zeros_like(sos)
    else:
        J, g = compute(problem, sos, w, sub, obs)
    return gradient_allreduce(J, g, group)
