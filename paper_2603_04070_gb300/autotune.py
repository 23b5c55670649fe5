"""Autotuner for the step-kernel launch options (tile height, one or two steps per launch, one
launch per step or one persistent launch per sweep segment).

For a given problem shape the tuner times a short forward simulation (or, for callers whose
work is gradients, a short misfit gradient) with each candidate option set, on the caller's
device, and keeps the fastest. Results are cached per (GPU name,
grid, shots, stencil order): in memory, and optionally in a JSON file. The options change
speed only: every candidate produces bit-identical results, which the tests check for the
one/two-step pair and the per-step/persistent pair.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import dufwi

CANDIDATES = (
    {"tile_z": 32, "two_step": 0, "persistent": 0},
    {"tile_z": 64, "two_step": 0, "persistent": 0},
    {"tile_z": 32, "two_step": 1, "persistent": 0},
    {"tile_z": 32, "two_step": 0, "persistent": 1},
)

_lock = threading.Lock()
_cache: dict[str, dict] = {}


def _key(problem: dufwi.Problem, geom: dufwi.Geometry, n_maps: int) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "%s|%dx%d|P%d|o%d|shots%d|rx%d" % (name, problem.nx, problem.nz, problem.pml_cells, problem.fd_order,
                                             n_maps * geom.n_tx, geom.n_rx)


def apply(options: dict):
    dufwi.set_option(dufwi.OPT_TILE_Z, int(options["tile_z"]))
    dufwi.set_option(dufwi.OPT_TWO_STEP, int(options["two_step"]))
    dufwi.set_option(dufwi.OPT_PERSISTENT, int(options.get("persistent", 0)))


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
    best["candidates_ms_per_step"] = [t / nt for t in timings]
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
