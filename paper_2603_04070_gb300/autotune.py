"""Autotuner for the step-kernel launch options (tile height, one or two steps per launch, one
launch per step or one persistent launch per sweep segment).

For a given problem shape the tuner times a short forward simulation with each candidate
option set, on the caller's device, and keeps the fastest. Results are cached per (GPU name,
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
         steps: int = 200, repeats: int = 3, cache_file: str | None = None, sizes=None) -> dict:
    """Pick and apply the fastest option set for this problem shape; returns it with timings."""
    key = _key(problem, geom, sos.shape[0])
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
    short = dufwi.Problem(**{**problem.__dict__, "nt": nt})
    w = wavelet[..., :nt].contiguous()
    ws = torch.empty(dufwi.workspace_size(short, geom, sos.shape[0], gradient=False), dtype=torch.uint8,
                     device=sos.device)
    cd = torch.empty((sos.shape[0], geom.n_tx, nt, geom.n_rx), dtype=torch.float32, device=sos.device)
    timings = []
    for cand in CANDIDATES:
        apply(cand)
        dufwi.simulate(short, sos, w, geom, cd=cd, workspace=ws, sizes=sizes)      # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(repeats):
            dufwi.simulate(short, sos, w, geom, cd=cd, workspace=ws, sizes=sizes)
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
