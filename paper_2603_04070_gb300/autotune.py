"""Autotuner for the step-kernel launch options and for the history split of gradients.

Launch options: the tile height of the one-step kernel (64 x 32 or 64 x 64), its multi-tile form
(co-resident CTAs walking the tiles with two-stage TMA loads), early requests of the operands the
previous two launches did not write (on or off), the number of shot groups stepped on concurrent
streams (1, 2 or 4), the register-cap variant of the one-step kernel (compiled for 4, 5 or 6
resident CTAs per SM), two steps per launch, one persistent launch per sweep segment, and, for
grids that fit, one launch of a thread-block cluster per shot and sweep segment. For a given
problem shape the tuner times a short forward simulation (or, for callers whose work is
gradients, a short misfit gradient) with each candidate, on the caller's device, and keeps the
fastest. Results are cached per (GPU name, grid, shots, stencil order): in
memory, and optionally in a JSON file. The options change speed only: every candidate produces
bit-identical results (tests check each pair against the default).

History split: ``kept_segments_for_budget`` picks how many checkpoint segments keep their
history from the forward sweep (each one saves the recompute of a segment) so that the gradient's
workspace stays within a memory budget; more kept segments never cost time, so the largest count
that fits is the fastest.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import dufwi

_BASE = {"tile_z": 32, "two_step": 0, "persistent": 0, "multi_tile": 0, "early": 1, "groups": 2, "min_ctas": 5,
         "cluster": 0}
CANDIDATES = (
    dict(_BASE),
    {**_BASE, "groups": 1},
    {**_BASE, "groups": 4},
    {**_BASE, "min_ctas": 4},
    {**_BASE, "min_ctas": 6},
    {**_BASE, "cluster": 1},
    {**_BASE, "early": 0},
    {**_BASE, "tile_z": 64},
    {**_BASE, "tile_z": 64, "groups": 1},
    {**_BASE, "multi_tile": 1, "groups": 1},
    {**_BASE, "multi_tile": 1, "early": 0, "groups": 1},
    {**_BASE, "two_step": 1, "groups": 1},
    {**_BASE, "persistent": 1, "groups": 1},
)
KNOBS = tuple(_BASE)

_lock = threading.Lock()
_cache: dict[str, dict] = {}


def _key(problem: dufwi.Problem, geom: dufwi.Geometry, n_maps: int) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "%s|%dx%d|P%d|o%d|shots%d|rx%d" % (name, problem.nx, problem.nz, problem.pml_cells, problem.fd_order,
                                             n_maps * geom.n_tx, geom.n_rx)


def cluster_fits(problem: dufwi.Problem) -> bool:
    """Whether the cluster-resident sweep applies to this grid: one shot's three fields (with 4
    halo rows per CTA), kappa' and the imaging sum fit 220 KB of shared memory in each of the 8
    CTAs of a cluster (the library makes the same test; elsewhere the option has no effect)."""
    nxp, nzp = problem.nx + 2 * problem.pml_cells, problem.nz + 2 * problem.pml_cells
    h = ((nzp + 7) // 8 + 3) // 4 * 4
    lp = (nxp + 3) // 4 * 4 + 8
    return (3 * (h + 8) + 2 * h) * lp * 4 <= 220 * 1024


def applicable(options: dict, problem: dufwi.Problem, sizes=None) -> bool:
    """False for a candidate whose option does nothing for this problem (it would only time the
    default again): the cluster form on a grid that does not fit or with maps of different sizes,
    the register-cap variants outside the 8th-order 64 x 32 form."""
    if options.get("cluster", 0) and (sizes is not None or not cluster_fits(problem)):
        return False
    if options.get("min_ctas", 5) != 5 and (problem.fd_order != 8 or options.get("tile_z", 32) != 32):
        return False
    return True


def apply(options: dict):
    dufwi.set_option(dufwi.OPT_TILE_Z, int(options.get("tile_z", 32)))
    dufwi.set_option(dufwi.OPT_TWO_STEP, int(options.get("two_step", 0)))
    dufwi.set_option(dufwi.OPT_PERSISTENT, int(options.get("persistent", 0)))
    dufwi.set_option(dufwi.OPT_MULTI_TILE, int(options.get("multi_tile", 0)))
    dufwi.set_option(dufwi.OPT_EARLY_LOADS, int(options.get("early", 1)))
    dufwi.set_option(dufwi.OPT_SHOT_GROUPS, int(options.get("groups", 2)))
    dufwi.set_option(dufwi.OPT_MIN_CTAS, int(options.get("min_ctas", 5)))
    dufwi.set_option(dufwi.OPT_CLUSTER, int(options.get("cluster", 0)))


def kept_segments_for_budget(problem: dufwi.Problem, geom: dufwi.Geometry, n_maps: int, budget_bytes: int) -> int:
    """Largest kept_segments whose gradient workspace fits budget_bytes (0 if none beyond the plain
    checkpointed layout fits; the plain layout's own size is not checked here)."""
    steps = problem.nt - 1
    K = problem.ckpt_interval
    if K <= 0 or K >= steps:
        return 0
    n_seg = (steps + K - 1) // K

    def size(k):
        return dufwi.workspace_size(dufwi.Problem(**{**problem.__dict__, "kept_segments": k}), geom, n_maps)

    lo, hi = 0, n_seg
    if size(1) > budget_bytes:
        return 0
    lo = 1
    while lo < hi:                      # the size grows with k: largest k with size(k) <= budget
        mid = (lo + hi + 1) // 2
        if size(mid) <= budget_bytes:
            lo = mid
        else:
            hi = mid - 1
    return lo


def tune(problem: dufwi.Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: dufwi.Geometry, *,
         steps: int = 200, repeats: int = 3, cache_file: str | None = None, sizes=None,
         gradient: bool = False, cd_obs: torch.Tensor | None = None) -> dict:
    """Pick and apply the fastest option set for this problem shape; returns it with timings.

    The probe is a short forward simulation, or with ``gradient`` a short misfit gradient (the
    forward, recompute and adjoint sweeps in the proportions of the call), keeping the problem's
    checkpoint interval relative to the probe length."""
    key = _key(problem, geom, sos.shape[0]) + ("|grad" if gradient else "")
    with _lock:
        if key not in _cache and cache_file and os.path.exists(cache_file):
            try:
                with open(cache_file) as f:
                    _cache.update(json.load(f))
            except (OSError, ValueError):
                pass
        if key in _cache:
            apply(_cache[key])
            return dict(_cache[key])
    nt = min(problem.nt, steps)
    fields = {**problem.__dict__, "nt": nt}
    if gradient and problem.ckpt_interval:
        fields["ckpt_interval"] = max(1, min(problem.ckpt_interval, nt // 4))
    short = dufwi.Problem(**fields)
    w = wavelet[..., :nt].contiguous()
    cd = torch.empty((sos.shape[0], geom.n_tx, nt, geom.n_rx), dtype=torch.float32, device=sos.device)
    if gradient:
        ws = torch.empty(dufwi.workspace_size(short, geom, sos.shape[0], gradient=True), dtype=torch.uint8,
                         device=sos.device)
        obs = cd_obs[:, :, :nt].contiguous() if cd_obs is not None else torch.zeros_like(cd)

        def run():
            dufwi.misfit_gradient(short, sos, w, geom, obs, workspace=ws, sizes=sizes)
    else:
        ws = torch.empty(dufwi.workspace_size(short, geom, sos.shape[0], gradient=False), dtype=torch.uint8,
                         device=sos.device)

        def run():
            dufwi.simulate(short, sos, w, geom, cd=cd, workspace=ws, sizes=sizes)
    timings = []
    for cand in CANDIDATES:
        if not applicable(cand, problem, sizes):
            timings.append(float("inf"))
            continue
        apply(cand)
        run()                                                                # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(repeats):
            run()
        ev[1].record()
        torch.cuda.synchronize()
        timings.append(ev[0].elapsed_time(ev[1]) / repeats)
    best = dict(CANDIDATES[min(range(len(CANDIDATES)), key=lambda i: timings[i])])
    best["ms_per_step"] = min(timings) / nt
    best["candidates_ms_per_step"] = [t / nt if t != float("inf") else None for t in timings]
    best["candidates"] = [dict(c) for c in CANDIDATES]
    apply(best)
    with _lock:
        _cache[key] = best
        if cache_file:
            try:
                with open(cache_file, "w") as f:
                    json.dump(_cache, f, indent=1)
            except OSError:
                pass
    return dict(best)
