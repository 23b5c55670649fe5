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
    collective of transmit sharding). Returns (misfit FP64, gradient FP32) on the inputs' device."""
    if not dist.is_available() or not dist.is_initialized():
        return misfit.to(torch.float64), grad.to(torch.float32)
    m = misfit.to(torch.float64).contiguous()
    g = grad.to(torch.float64).contiguous()
    dist.all_reduce(m, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return m, g.to(torch.float32)


def _cuda_compute(problem, sos, wavelet, geom, cd_obs):
    from . import dufwi
    return dufwi.misfit_gradient(problem, sos, wavelet, geom, cd_obs)


def sharded_misfit_gradient(problem, sos: torch.Tensor, wavelet: torch.Tensor, geom, cd_obs: torch.Tensor, *,
                            group=None, compute: Callable | None = None):
    """Misfit and gradient of every map with the transmits split over the ranks of `group`.

    ``geom`` is the full geometry; each rank keeps the transmits of its block, the matching
    rows of the receive table and of ``cd_obs [maps][n_tx][nt][n_rx]`` (and of a per-transmit
    pulse). ``compute(problem, sos, wavelet, sub_geom, sub_cd_obs) -> (J, g)`` runs on the rank.
    """
    from .dufwi import Geometry
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    sel = shard_transmits(geom.n_tx, world, rank)
    idx = np.arange(sel.start, sel.stop)
    sub = Geometry(geom.elem_ix, geom.elem_iz, geom.tx_elem[idx], geom.rx_elem[idx], geom.wavelet_per_tx)
    w = wavelet[sel.start:sel.stop] if geom.wavelet_per_tx else wavelet
    compute = compute or _cuda_compute
    if len(idx) == 0:   # more ranks than transmits: contribute zeros
        J = torch.zeros(sos.shape[0], dtype=torch.float64, device=sos.device)
        g = torch.zeros_like(sos)
    else:
        J, g = compute(problem, sos, w, sub, cd_obs[:, sel.start:sel.stop].contiguous())
    return gradient_allreduce(J, g, group)
