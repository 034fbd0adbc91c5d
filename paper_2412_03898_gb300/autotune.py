"""Tile autotuner for the forward projection.

Times candidate tile plans (sensors per CTA, samples per CTA, balls per TMA
stage, ball splits, pairs per sweep) on the caller's actual data with CUDA
events and keeps the fastest per shape class.  The shape class is (sensors,
samples, frames, log2 of the ball count); results are cached in memory and,
when PA_TILE_CACHE names a file, in that JSON file.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional, Sequence

import torch

from . import Geometry, forward, forward_batched, forward_plan, forward_workspace_size

# (s_tile, t_tile, nb_tile, splits, group); splits 0 = the planner's choice
DEFAULT_CANDIDATES = [
    (16, 1536, 512, 0, 8), (16, 1536, 512, 0, 16), (12, 2048, 512, 0, 8), (12, 2048, 512, 0, 16),
    (16, 1536, 256, 0, 8), (16, 1024, 512, 0, 8), (8, 2048, 512, 0, 8), (16, 1536, 512, 0, 4),
]

_cache: dict = {}


def _cache_file() -> Optional[str]:
    return os.environ.get("PA_TILE_CACHE")


def _load_file():
    path = _cache_file()
    if path and os.path.exists(path):
        try:
            with open(path) as fh:
                for k, v in json.load(fh).items():
                    _cache.setdefault(k, tuple(v))
        except (OSError, ValueError):
            pass


def _store_file():
    path = _cache_file()
    if path:
        try:
            with open(path, "w") as fh:
                json.dump({k: list(v) for k, v in _cache.items()}, fh)
        except OSError:
            pass


def shape_key(geom: Geometry, state: torch.Tensor, n: int) -> str:
    F = int(state.shape[0]) if state.dim() == 3 else 1
    return f"fwd:S{geom.n_sensors}:T{geom.n_samples}:F{F}:N2^{int(round(math.log2(max(n, 1))))}"


def _time(fn, reps: int, flush: torch.Tensor) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_forward(geom: Geometry, state: torch.Tensor, n: Optional[int] = None,
                 candidates: Optional[Sequence[tuple]] = None, reps: int = 3, verbose: bool = False) -> tuple:
    """Fastest tile plan for pa_forward on this data (cached per shape class)."""
    n = int(state.shape[-1]) if n is None else int(n)
    _load_file()
    key = shape_key(geom, state, n)
    if key in _cache:
        return _cache[key]
    cands = []
    smem_max = torch.cuda.get_device_properties(state.device).shared_memory_per_block_optin
    for c in (candidates or DEFAULT_CANDIDATES):
        plan = forward_plan(geom, state, n, tiles=c)
        if plan["smem"] <= smem_max:
            cands.append(c)
    out = torch.empty(state.shape[0] if state.dim() == 3 else 1, geom.n_sensors, geom.n_samples,
                      dtype=torch.float32, device=state.device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=state.device)
    best, best_ms = None, float("inf")
    for c in cands:
        need = forward_workspace_size(geom, state, n, tiles=c)
        ws = torch.empty(max(need, 16), dtype=torch.uint8, device=state.device)
        ms = _time(lambda: forward(geom, state, n, out=out, tiles=c, workspace=ws), reps, flush)
        if verbose:
            print(f"autotune {key} {c}: {ms:.3f} ms")
        if ms < best_ms:
            best, best_ms = c, ms
    _cache[key] = tuple(best)
    _store_file()
    return _cache[key]


def tune_batched(scenes, candidates: Optional[Sequence[tuple]] = None, reps: int = 2,
                 verbose: bool = False) -> tuple:
    """Fastest tile plan for one persistent batched forward over `scenes`."""
    key = "batched:" + ";".join(f"{sc.geom.n_sensors}x{sc.geom.n_samples}x{sc.F}x{sc.n}" for sc in scenes)
    if key in _cache:
        return _cache[key]
    dev = scenes[0].state.device
    smem_max = torch.cuda.get_device_properties(dev).shared_memory_per_block_optin
    cands = []
    for c in (candidates or DEFAULT_CANDIDATES):
        if forward_plan(scenes[0].geom, scenes[0].state, scenes[0].n, tiles=c)["smem"] <= smem_max:
            cands.append(c)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    best, best_ms = None, float("inf")
    for c in cands:
        ms = _time(lambda: forward_batched(scenes, tiles=c), reps, flush)
        if verbose:
            print(f"autotune batched {c}: {ms:.3f} ms")
        if ms < best_ms:
            best, best_ms = c, ms
    _cache[key] = tuple(best)
    return _cache[key]
