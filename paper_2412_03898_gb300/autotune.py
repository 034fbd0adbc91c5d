"""Tile autotuning: a thin caller of the library's own tuner (pa_plan_create
with PA_PLAN_TUNE), which times candidate tile plans on the caller's data
with CUDA events and keeps the fastest.

This module only adds a cache of tuned values per shape class, in memory
and, when PA_TILE_CACHE names a file, in that JSON file.  The shape class is
(sensors, samples, frames, log2 of the ball count) for one scene, and the
list of scene shapes for a batch.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

import torch

from . import Geometry, Plan, Scene

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


def _plan_from_cache(key: str) -> Optional[Plan]:
    _load_file()
    if key not in _cache:
        return None
    v = tuple(_cache[key]) + (0,) * (7 - len(_cache[key]))
    return Plan.from_values(v[:5], frames_per_chunk=v[5], adj_chunk=v[6])


def _remember(key: str, plan: Plan) -> None:
    v = plan.values()
    _cache[key] = tuple(v["tiles"]) + (v["frames_per_chunk"], v["adj_chunk"])
    _store_file()


def tune_forward_plan(geom: Geometry, state: torch.Tensor, n: Optional[int] = None) -> Plan:
    """Fastest forward plan for this one scene (cached per shape class).
    Tuning overwrites a scratch trace buffer only."""
    n = int(state.shape[-1]) if n is None else int(n)
    key = shape_key(geom, state, n)
    plan = _plan_from_cache(key)
    if plan is None:
        sc = Scene(geom, state, n)
        plan = Plan.create([sc], tune=True)
        _remember(key, plan)
    return plan


def tune_forward(geom: Geometry, state: torch.Tensor, n: Optional[int] = None) -> tuple:
    """Tiles {sensors, samples, balls per stage, splits, pairs per sweep} of
    the fastest forward plan for this scene."""
    return tuple(tune_forward_plan(geom, state, n).values()["tiles"])


def tune_batched(scenes) -> Plan:
    """Fastest plan for the persistent batched forward (and, when every scene
    carries trace_grad and grad_state, the batched adjoint's items per grab)
    over these scenes.  Tuning overwrites the scenes' traces and grad_state."""
    key = "batched:" + ";".join(f"{sc.geom.n_sensors}x{sc.geom.n_samples}x{sc.F}x{sc.n}" for sc in scenes)
    plan = _plan_from_cache(key)
    if plan is None:
        plan = Plan.create(list(scenes), tune=True)
        _remember(key, plan)
    return plan
