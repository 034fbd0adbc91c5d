"""GB300-native (sm_103a) hot path of 4D SlingBAG (arXiv 2412.03898).

Torch-facing binding of the C ABI in include/pa.h.  Every step of the path
runs in the library's CUDA kernels; this module only checks tensors, builds
the argument structs and passes raw device pointers and the current CUDA
stream.  It raises if libpa.so is missing or a tensor is not on a CUDA
device: there is no CPU fallback.

Layouts (see include/pa.h): ball states [F, 5, stride] float32 with channels
(x, y, z, a, p) and stride % 4 == 0; deformation parameters [5, Nb, stride];
sensors [3, S]; traces [F, S, T].
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import PAError

__all__ = [
    "PAError", "Geometry", "round4", "pad_last", "deform_balls", "deform_backward", "forward", "adjoint", "residual_loss", "sumsq",
    "count_contributions", "adam_step", "device_error", "forward_plan", "forward_workspace_size",
    "PAProject", "PAProject4D", "PALoss", "Scene", "forward_batched", "adjoint_batched", "adam_step_scheduled", "step_increment",
    "Plan", "forward_4d", "adjoint_4d", "forward_4d_workspace_size", "adjoint_4d_workspace_size", "Buffers4D",
    "forward_plan_for",
    "Grid", "ubp_filter", "ubp", "splat", "maps", "ssim", "measure_unit_rates", "spatial_order", "gather_rows",
]



def _ensure_built() -> None:
    """Build libpa.so in-tree when it is missing or older than its sources."""
    from . import build as _build
    if os.path.exists(_lib.LIB_PATH) and not _build._stale():
        return
    try:
        _build.build()
    except (OSError, RuntimeError) as e:
        if not os.path.exists(_lib.LIB_PATH):
            raise ImportError(f"libpa.so is missing and could not be built: {e}") from e


_ensure_built()
_LIB = _lib.load()


def round4(n: int) -> int:
    return (int(n) + 3) // 4 * 4


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _check(t: torch.Tensor, name: str, dtype=torch.float32) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (this library has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def pad_last(x: torch.Tensor, stride: Optional[int] = None) -> torch.Tensor:
    """Copy x [..., N] into a zero-padded contiguous float32 [..., stride]
    buffer (stride = N rounded up to a multiple of 4 by default)."""
    n = x.shape[-1]
    stride = round4(n) if stride is None else int(stride)
    out = torch.zeros(*x.shape[:-1], stride, dtype=torch.float32, device=x.device)
    out[..., :n] = x
    return out


class Geometry:
    """Sensor array and acquisition scalars (pa_geom)."""

    def __init__(self, sensors: torch.Tensor, c: float, fs: float, t0: float, n_samples: int, kappa: float = 5.0,
                 sensor_range: Optional[tuple] = None):
        """sensors: [3, S] CUDA float32.  sensor_range = (begin, end) selects a
        shard of the array without copying (the pointer is offset and the row
        stride stays S): outputs then cover sensors begin..end-1 only."""
        self.sensors = _check(sensors, "sensors")
        if sensors.dim() != 2 or sensors.shape[0] != 3:
            raise ValueError("sensors must be [3, S]")
        self.c, self.fs, self.t0 = float(c), float(fs), float(t0)
        self.n_samples, self.kappa = int(n_samples), float(kappa)
        total = int(sensors.shape[1])
        b, e = (0, total) if sensor_range is None else (int(sensor_range[0]), int(sensor_range[1]))
        if not 0 <= b < e <= total:
            raise ValueError("sensor_range must satisfy 0 <= begin < end <= S")
        self.sensor_range = (b, e)
        self._struct = _lib.pa_geom(self.sensors.data_ptr() + 4 * b, e - b, total, self.c, self.fs, self.t0,
                                    self.n_samples, self.kappa)

    @property
    def n_sensors(self) -> int:
        return self.sensor_range[1] - self.sensor_range[0]

    def shard(self, begin: int, end: int) -> "Geometry":
        """The same acquisition restricted to sensors begin..end-1."""
        return Geometry(self.sensors, self.c, self.fs, self.t0, self.n_samples, self.kappa, (begin, end))

    def struct(self) -> _lib.pa_geom:
        return self._struct

    def __repr__(self):
        return (f"Geometry(S={self.n_sensors}, c={self.c}, fs={self.fs}, t0={self.t0}, T={self.n_samples}, "
                f"kappa={self.kappa})")


def _balls_struct(state: torch.Tensor, n: Optional[int]):
    _check(state, "state")
    if state.dim() == 2:
        state = state.unsqueeze(0)
    if state.dim() != 3 or state.shape[1] != 5:
        raise ValueError("state must be [F, 5, stride]")
    stride = int(state.shape[2])
    n = stride if n is None else int(n)
    return state, _lib.pa_balls(state.data_ptr(), n, stride), n


def _canon_struct(canon, omega, theta, sigma, n):
    for t, nm in ((canon, "canon"), (omega, "omega"), (theta, "theta"), (sigma, "sigma")):
        _check(t, nm)
    stride = int(canon.shape[-1])
    nb = int(omega.shape[1])
    if tuple(canon.shape) != (5, stride) or tuple(omega.shape) != (5, nb, stride) or \
            theta.shape != omega.shape or sigma.shape != omega.shape:
        raise ValueError("canon must be [5, stride] and omega/theta/sigma [5, Nb, stride]")
    n = stride if n is None else int(n)
    return _lib.pa_canon(canon.data_ptr(), omega.data_ptr(), theta.data_ptr(), sigma.data_ptr(), n, stride, nb), n


def device_error(raise_on_error: bool = True) -> int:
    """Read and clear the device error word (synchronises the stream)."""
    out = ctypes.c_int32(0)
    _lib.check(_LIB.pa_device_error(_stream(), ctypes.byref(out)), "pa_device_error")
    if raise_on_error and out.value != 0:
        raise PAError(out.value, "kernel")
    return int(out.value)


def deform_balls(canon: torch.Tensor, omega: torch.Tensor, theta: torch.Tensor, sigma: torch.Tensor,
                 t_frames: torch.Tensor, n: Optional[int] = None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Eq. 1-2: per-frame states [F, 5, stride] from the GGBall parameters."""
    cs, n = _canon_struct(canon, omega, theta, sigma, n)
    _check(t_frames, "t_frames")
    F = int(t_frames.numel())
    if out is None:
        out = torch.empty(F, 5, canon.shape[-1], dtype=torch.float32, device=canon.device)
    _check(out, "out")
    _lib.check(_LIB.pa_deform_balls(ctypes.byref(cs), t_frames.data_ptr(), F, out.data_ptr(), _stream()),
               "pa_deform_balls")
    return out


def deform_backward(canon: torch.Tensor, omega: torch.Tensor, theta: torch.Tensor, sigma: torch.Tensor,
                    t_frames: torch.Tensor, g_state: torch.Tensor, n: Optional[int] = None, out=None,
                    accumulate: bool = False):
    """Chain rule of Eq. 1-2: per-frame state gradients g_state [F, 5, stride]
    -> (g_canon [5, stride], g_omega, g_theta, g_sigma [5, Nb, stride])."""
    cs, n = _canon_struct(canon, omega, theta, sigma, n)
    _check(t_frames, "t_frames")
    _check(g_state, "g_state")
    F = int(t_frames.numel())
    if tuple(g_state.shape) != (F, 5, canon.shape[-1]):
        raise ValueError(f"g_state must be [{F}, 5, {canon.shape[-1]}], got {tuple(g_state.shape)}")
    if out is None:
        out = (torch.empty_like(canon), torch.empty_like(omega), torch.empty_like(theta), torch.empty_like(sigma))
    for o in out:
        _check(o, "out")
    grads = _lib.pa_grads(*[o.data_ptr() for o in out])
    _lib.check(_LIB.pa_deform_backward(ctypes.byref(cs), t_frames.data_ptr(), F, g_state.data_ptr(),
                                       ctypes.byref(grads), _lib.PA_ACCUMULATE if accumulate else 0, _stream()),
               "pa_deform_backward")
    return out


def selftest_bounded_wait(limit_ns: int = 2_000_000) -> None:
    """Make the bounded in-kernel wait run out (PA_ERR_TIMEOUT is then
    reported by the next device_error())."""
    _lib.check(_LIB.pa_selftest_bounded_wait(int(limit_ns), _stream()), "pa_selftest_bounded_wait")


def measure_unit_rates() -> dict:
    """Measured throughput of this GPU's FP32 FMA pipe (scalar and packed
    FP32x2) and SFU ex2, per SM per clock, and the SM clock in MHz."""
    out = (ctypes.c_double * 4)()
    _lib.check(_LIB.pa_measure_unit_rates(_stream(), out), "pa_measure_unit_rates")
    return {"ffma_lanes_per_sm_clk": out[0], "ffma2_lanes_per_sm_clk": out[1], "ex2_per_sm_clk": out[2],
            "sm_mhz": out[3]}


def _tiles(tiles: Optional[Sequence[int]]):
    if tiles is None:
        return None
    vals = [int(v) for v in tiles] + [0] * (5 - len(tiles))
    return (ctypes.c_int32 * 5)(*vals[:5])


def forward_workspace_size(geom: Geometry, state: torch.Tensor, n: Optional[int] = None,
                           tiles: Optional[Sequence[int]] = None) -> int:
    state, bs, n = _balls_struct(state, n)
    t = _tiles(tiles)
    return int(_LIB.pa_forward_workspace_size_ex(ctypes.byref(geom.struct()), ctypes.byref(bs),
                                                 int(state.shape[0]), t))


def forward_plan(geom: Geometry, state: torch.Tensor, n: Optional[int] = None,
                 tiles: Optional[Sequence[int]] = None) -> dict:
    state, bs, n = _balls_struct(state, n)
    out = (ctypes.c_int32 * 7)()
    _lib.check(_LIB.pa_forward_plan_info(ctypes.byref(geom.struct()), ctypes.byref(bs), int(state.shape[0]),
                                         _tiles(tiles), out), "pa_forward_plan_info")
    return dict(s_tile=out[0], t_tile=out[1], nb_tile=out[2], n_splits=out[3], group=out[4], ctas=out[5],
                smem=out[6])


def forward_plan_for(geom: Geometry, n: int, n_frames: int, tiles: Optional[Sequence[int]] = None) -> dict:
    """The plan pa_forward_ex would use for n balls and n_frames frames (no
    ball data needed: the query reads only the sizes)."""
    bs = _lib.pa_balls(16, int(n), round4(max(int(n), 1)))  # pointer never dereferenced by the query
    out = (ctypes.c_int32 * 7)()
    _lib.check(_LIB.pa_forward_plan_info(ctypes.byref(geom.struct()), ctypes.byref(bs), int(n_frames),
                                         _tiles(tiles), out), "pa_forward_plan_info")
    return dict(s_tile=out[0], t_tile=out[1], nb_tile=out[2], n_splits=out[3], group=out[4], ctas=out[5],
                smem=out[6])


def forward(geom: Geometry, state: torch.Tensor, n: Optional[int] = None, out: Optional[torch.Tensor] = None,
            accumulate: bool = False, uniform: bool = False, tiles: Optional[Sequence[int]] = None,
            workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Forward projection: traces [F, S, T] of the states [F, 5, stride]."""
    state, bs, n = _balls_struct(state, n)
    F = int(state.shape[0])
    if out is None:
        if accumulate:
            raise ValueError("accumulate=True needs out")
        out = torch.empty(F, geom.n_sensors, geom.n_samples, dtype=torch.float32, device=state.device)
    _check(out, "out")
    t = _tiles(tiles)
    need = int(_LIB.pa_forward_workspace_size_ex(ctypes.byref(geom.struct()), ctypes.byref(bs), F, t))
    if need > 0 and (workspace is None or workspace.numel() < need):
        workspace = torch.empty(need, dtype=torch.uint8, device=state.device)
    flags = (_lib.PA_ACCUMULATE if accumulate else 0) | (_lib.PA_PROFILE_UNIFORM if uniform else 0)
    ws_ptr = workspace.data_ptr() if need > 0 else None
    ws_n = workspace.numel() if need > 0 else 0
    _lib.check(_LIB.pa_forward_ex(ctypes.byref(geom.struct()), ctypes.byref(bs), F, out.data_ptr(), flags, t,
                                  ws_ptr, ws_n, _stream()), "pa_forward")
    return out


def adjoint(geom: Geometry, trace_grad: torch.Tensor, state: Optional[torch.Tensor] = None,
            n: Optional[int] = None, canon: Optional[torch.Tensor] = None, omega: Optional[torch.Tensor] = None,
            theta: Optional[torch.Tensor] = None, sigma: Optional[torch.Tensor] = None,
            t_frames: Optional[torch.Tensor] = None, frame_scale: Optional[torch.Tensor] = None,
            accumulate: bool = False, out=None, queue: bool = True, workspace: Optional[torch.Tensor] = None):
    """Adjoint of `forward`.  Static mode (state given): returns dL/dstate
    [F, 5, stride].  4D mode (canon, omega, theta, sigma, t_frames given):
    returns (g_canon [5, stride], g_omega, g_theta, g_sigma [5, Nb, stride]).
    queue: static mode hands (frame, ball) items to warps from a work-queue
    counter in `workspace` (256 bytes, allocated here when None); False
    deals them out in grid-stride order.  The results are the same."""
    _check(trace_grad, "trace_grad")
    F = int(trace_grad.shape[0])
    if frame_scale is not None:
        _check(frame_scale, "frame_scale")
    flags = _lib.PA_ACCUMULATE if accumulate else 0
    if state is not None:
        state, bs, n = _balls_struct(state, n)
        if out is None:
            out = torch.empty_like(state)
        grads = _lib.pa_grads(out.data_ptr(), None, None, None)
        ws_ptr, ws_n = None, 0
        if queue:
            if workspace is None or workspace.numel() < _lib.PA_ADJOINT_WORKSPACE_BYTES:
                workspace = torch.empty(_lib.PA_ADJOINT_WORKSPACE_BYTES, dtype=torch.uint8, device=state.device)
            ws_ptr, ws_n = workspace.data_ptr(), workspace.numel() * workspace.element_size()
        _lib.check(_LIB.pa_adjoint(ctypes.byref(geom.struct()), ctypes.byref(bs), None, None, F,
                                   trace_grad.data_ptr(), _ptr(frame_scale), ctypes.byref(grads), flags,
                                   ws_ptr, ws_n, _stream()),
                   "pa_adjoint")
        return out
    cs, n = _canon_struct(canon, omega, theta, sigma, n)
    _check(t_frames, "t_frames")
    if out is None:
        out = (torch.empty_like(canon), torch.empty_like(omega), torch.empty_like(theta), torch.empty_like(sigma))
    grads = _lib.pa_grads(*[o.data_ptr() for o in out])
    _lib.check(_LIB.pa_adjoint(ctypes.byref(geom.struct()), None, ctypes.byref(cs), t_frames.data_ptr(), F,
                               trace_grad.data_ptr(), _ptr(frame_scale), ctypes.byref(grads), flags, None, 0,
                               _stream()),
               "pa_adjoint")
    return out


def spatial_order(state: torch.Tensor, n: Optional[int] = None,
                  workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Morton (Z-curve) order of the ball centres of frame 0 of `state`
    ([F, 5, stride] or [5, stride]): an int32 permutation perm [n] such that
    position i of the reordered cloud holds ball perm[i] (pa_spatial_order).
    Apply it with gather_rows; a cloud stored in this order makes the
    forward's ball tiles compact in space."""
    state, bs, n = _balls_struct(state, n)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=state.device)[:n]
    need = int(_LIB.pa_spatial_order_workspace_size(n))
    workspace = _workspace(workspace, max(need, 256), state.device)
    _lib.check(_LIB.pa_spatial_order(ctypes.byref(bs), perm.data_ptr() if n > 0 else None, workspace.data_ptr(),
                                     workspace.numel(), _stream()), "pa_spatial_order")
    return perm


def gather_rows(x: torch.Tensor, perm: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """out[..., i] = x[..., perm[i]] for i < len(perm) over every leading row
    of a contiguous [..., stride] tensor (pa_gather_rows); the padding
    columns of a new `out` are zero."""
    _check(x, "x")
    _check(perm, "perm", torch.int32)
    stride = int(x.shape[-1])
    n = int(perm.numel())
    rows = x.numel() // stride if stride > 0 else 0
    if out is None:
        out = torch.zeros_like(x)
    _check(out, "out")
    if out.shape != x.shape:
        raise ValueError("out must have the shape of x")
    _lib.check(_LIB.pa_gather_rows(x.data_ptr(), out.data_ptr(), n, stride, rows, perm.data_ptr(), _stream()),
               "pa_gather_rows")
    return out


def residual_loss(pred: torch.Tensor, meas: torch.Tensor, frame_scale: Optional[torch.Tensor] = None,
                  want_loss: bool = True, want_resid: bool = False, loss_out: Optional[torch.Tensor] = None,
                  resid_out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None):
    """Per-frame FP64 loss sum (pred-meas)^2 and/or residual 2 scale (pred-meas)."""
    _check(pred, "pred")
    _check(meas, "meas")
    F = int(pred.shape[0])
    per = int(pred.numel() // max(F, 1))
    loss = None
    if want_loss:
        loss = loss_out if loss_out is not None else torch.empty(F, dtype=torch.float64, device=pred.device)
        _check(loss, "loss", torch.float64)
    resid = None
    if want_resid:
        resid = resid_out if resid_out is not None else torch.empty_like(pred)
        _check(resid, "resid")
    need = int(_LIB.pa_loss_workspace_size(per, F))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=pred.device)
    _lib.check(_LIB.pa_residual_loss(pred.data_ptr(), meas.data_ptr(), per, F, _ptr(frame_scale), _ptr(loss),
                                     _ptr(resid), workspace.data_ptr(), workspace.numel(), _stream()),
               "pa_residual_loss")
    return loss, resid


def sumsq(x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """FP64 sum of squares of a float32 CUDA tensor (gradient norms)."""
    _check(x, "x")
    out = out if out is not None else torch.empty(1, dtype=torch.float64, device=x.device)
    need = int(_LIB.pa_loss_workspace_size(x.numel(), 1))
    ws = torch.empty(max(need, 16), dtype=torch.uint8, device=x.device)
    _lib.check(_LIB.pa_sumsq(x.data_ptr(), x.numel(), out.data_ptr(), ws.data_ptr(), ws.numel(), _stream()),
               "pa_sumsq")
    return out


def count_contributions(geom: Geometry, state: torch.Tensor, n: Optional[int] = None) -> int:
    """Number of (frame, sensor, ball, sample) terms the forward sums."""
    state, bs, n = _balls_struct(state, n)
    out = torch.zeros(1, dtype=torch.int64, device=state.device)
    _lib.check(_LIB.pa_count_contributions(ctypes.byref(geom.struct()), ctypes.byref(bs), int(state.shape[0]),
                                           out.data_ptr(), _stream()), "pa_count_contributions")
    return int(out.item())


def adam_step(x: torch.Tensor, g: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    for t, nm in ((x, "x"), (g, "g"), (m, "m"), (v, "v")):
        _check(t, nm)
    _lib.check(_LIB.pa_adam_step(x.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), x.numel(), float(lr),
                                 float(beta1), float(beta2), float(eps), int(step), _stream()), "pa_adam_step")


class Scene:
    """One scene of a batched call (pa_scene): geometry, per-frame states
    [F, 5, stride] and the buffers the batched calls read or write."""

    def __init__(self, geom: Geometry, state: torch.Tensor, n: Optional[int] = None,
                 traces: Optional[torch.Tensor] = None, trace_grad: Optional[torch.Tensor] = None,
                 grad_state: Optional[torch.Tensor] = None):
        self.geom = geom
        self.state, self._balls, self.n = _balls_struct(state, n)
        self.F = int(self.state.shape[0])
        self.traces = traces
        self.trace_grad = trace_grad
        self.grad_state = grad_state

    def struct(self) -> _lib.pa_scene:
        return _lib.pa_scene(self.geom.struct(), self._balls, self.F, _ptr(self.traces), _ptr(self.trace_grad),
                             _ptr(self.grad_state))


def _scene_array(scenes):
    if len(scenes) > _lib.PA_MAX_SCENES:
        raise ValueError(f"at most {_lib.PA_MAX_SCENES} scenes per batched call")
    return (_lib.pa_scene * max(len(scenes), 1))(*[sc.struct() for sc in scenes])


class Plan:
    """Launch plan (pa_plan): forward tiles, frames per 4D launch and the
    batched adjoint's items per queue grab.  Plan.create() asks the library
    for the heuristic or, with tune=True, times the candidate plans on the
    given scenes (overwriting their traces and grad_state); Plan.from_values()
    wraps explicit values (0 = heuristic)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @classmethod
    def create(cls, scenes, tune: bool = True) -> "Plan":
        scenes = list(scenes)
        dev = scenes[0].state.device
        for sc in scenes:
            if sc.traces is None:
                sc.traces = torch.empty(sc.F, sc.geom.n_sensors, sc.geom.n_samples, dtype=torch.float32,
                                        device=dev)
            _check(sc.traces, "traces")
        arr = _scene_array(scenes)  # after the scratch traces exist
        need = int(_LIB.pa_plan_workspace_size(arr, len(scenes))) if tune else 0
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        _lib.check(_LIB.pa_plan_create(arr, len(scenes), _lib.PA_PLAN_TUNE if tune else 0, ws.data_ptr(),
                                       ws.numel(), _stream(), ctypes.byref(h)), "pa_plan_create")
        return cls(h.value)

    @classmethod
    def from_values(cls, tiles: Optional[Sequence[int]] = None, frames_per_chunk: int = 0,
                    adj_chunk: int = 0) -> "Plan":
        vals = [int(v) for v in (tiles or ())] + [0] * (5 - len(tiles or ()))
        arr = (ctypes.c_int32 * 7)(*(vals[:5] + [int(frames_per_chunk), int(adj_chunk)]))
        h = ctypes.c_void_p()
        _lib.check(_LIB.pa_plan_from_values(arr, ctypes.byref(h)), "pa_plan_from_values")
        return cls(h.value)

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def values(self) -> dict:
        v = (ctypes.c_int32 * 7)()
        t = (ctypes.c_float * 2)()
        _lib.check(_LIB.pa_plan_get(self._h, v, t), "pa_plan_get")
        return {"tiles": tuple(v[:5]), "frames_per_chunk": v[5], "adj_chunk": v[6], "forward_ms": t[0],
                "adjoint_ms": t[1], "tuned": t[0] > 0}

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and h.value:
            try:
                _LIB.pa_plan_destroy(h)
            except Exception:  # pragma: no cover (interpreter shutdown)
                pass


def _plan_arg(plan: Optional["Plan"], tiles: Optional[Sequence[int]]):
    """(plan handle or None, the Plan object to keep alive)."""
    if plan is None and tiles is not None:
        plan = Plan.from_values(tiles)
    return (plan.handle if plan is not None else None), plan


def forward_batched(scenes, tiles: Optional[Sequence[int]] = None, accumulate: bool = False,
                    workspace: Optional[torch.Tensor] = None, plan: Optional[Plan] = None):
    """Forward projection of several scenes in one persistent launch; fills
    (allocating if needed) each scene's traces [F, S, T].  plan (or tiles,
    wrapped into a plan) sets the tiles."""
    for sc in scenes:
        if sc.traces is None:
            sc.traces = torch.empty(sc.F, sc.geom.n_sensors, sc.geom.n_samples, dtype=torch.float32,
                                    device=sc.state.device)
        _check(sc.traces, "traces")
    arr = _scene_array(scenes)
    dev = scenes[0].state.device if scenes else torch.device("cuda")
    h, keep = _plan_arg(plan, tiles)
    need = int(_LIB.pa_batched_workspace_size(arr, len(scenes), h))
    workspace = _workspace(workspace, need, dev)
    _lib.check(_LIB.pa_forward_batched(arr, len(scenes), _lib.PA_ACCUMULATE if accumulate else 0, h,
                                       workspace.data_ptr(), workspace.numel(), _stream()), "pa_forward_batched")
    del keep
    return [sc.traces for sc in scenes]


def adjoint_batched(scenes, accumulate: bool = False, workspace: Optional[torch.Tensor] = None,
                    plan: Optional[Plan] = None):
    """Static-mode adjoint of several scenes in one persistent launch; reads
    each scene's trace_grad and fills its grad_state [F, 5, stride]."""
    for sc in scenes:
        _check(sc.trace_grad, "trace_grad")
        if sc.grad_state is None:
            sc.grad_state = torch.empty_like(sc.state)
        _check(sc.grad_state, "grad_state")
    arr = _scene_array(scenes)
    dev = scenes[0].state.device if scenes else torch.device("cuda")
    workspace = _workspace(workspace, 256, dev)
    h = plan.handle if plan is not None else None
    _lib.check(_LIB.pa_adjoint_batched(arr, len(scenes), _lib.PA_ACCUMULATE if accumulate else 0, h,
                                       workspace.data_ptr(), workspace.numel(), _stream()), "pa_adjoint_batched")
    return [sc.grad_state for sc in scenes]


def _deform_views(deform: torch.Tensor):
    _check(deform, "deform")
    if deform.dim() != 4 or deform.shape[0] != 3 or deform.shape[1] != 5:
        raise ValueError("deform must be [3, 5, Nb, stride] (omega, theta, sigma)")
    return deform[0], deform[1], deform[2]


def forward_4d_workspace_size(geom: Geometry, canon: torch.Tensor, deform: torch.Tensor, t_frames: torch.Tensor,
                              n: Optional[int] = None, plan: Optional[Plan] = None) -> int:
    cs, n = _canon_struct(canon, *_deform_views(deform), n)
    return int(_LIB.pa_forward_4d_workspace_size(ctypes.byref(geom.struct()), ctypes.byref(cs),
                                                 int(t_frames.numel()), plan.handle if plan else None))


def adjoint_4d_workspace_size(geom: Geometry, canon: torch.Tensor, deform: torch.Tensor, t_frames: torch.Tensor,
                              n: Optional[int] = None, plan: Optional[Plan] = None) -> int:
    cs, n = _canon_struct(canon, *_deform_views(deform), n)
    return int(_LIB.pa_adjoint_4d_workspace_size(ctypes.byref(geom.struct()), ctypes.byref(cs),
                                                 int(t_frames.numel()), plan.handle if plan else None))


def _workspace(ws: Optional[torch.Tensor], need: int, dev) -> torch.Tensor:
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    return ws


def forward_4d(geom: Geometry, canon: torch.Tensor, deform: torch.Tensor, t_frames: torch.Tensor,
               n: Optional[int] = None, out: Optional[torch.Tensor] = None, accumulate: bool = False,
               plan: Optional[Plan] = None, workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Traces [F, S, T] of the 4D sequence straight from the GGBall parameters
    (canon [5, stride], deform [3, 5, Nb, stride]): states are deformed per
    frame chunk in the workspace and never held for all frames."""
    cs, n = _canon_struct(canon, *_deform_views(deform), n)
    _check(t_frames, "t_frames")
    F = int(t_frames.numel())
    if out is None:
        if accumulate:
            raise ValueError("accumulate=True needs out")
        out = torch.empty(F, geom.n_sensors, geom.n_samples, dtype=torch.float32, device=canon.device)
    _check(out, "out")
    h = plan.handle if plan is not None else None
    need = int(_LIB.pa_forward_4d_workspace_size(ctypes.byref(geom.struct()), ctypes.byref(cs), F, h))
    workspace = _workspace(workspace, need, canon.device)
    _lib.check(_LIB.pa_forward_4d(ctypes.byref(geom.struct()), ctypes.byref(cs), t_frames.data_ptr(), F,
                                  out.data_ptr(), _lib.PA_ACCUMULATE if accumulate else 0, h, workspace.data_ptr(),
                                  workspace.numel(), _stream()), "pa_forward_4d")
    return out


def adjoint_4d(geom: Geometry, trace_grad: torch.Tensor, canon: torch.Tensor, deform: torch.Tensor,
               t_frames: torch.Tensor, n: Optional[int] = None, frame_scale: Optional[torch.Tensor] = None,
               accumulate: bool = False, out=None, plan: Optional[Plan] = None,
               workspace: Optional[torch.Tensor] = None):
    """Adjoint of forward_4d: (g_canon [5, stride], g_deform [3, 5, Nb,
    stride]), states recomputed per frame chunk."""
    cs, n = _canon_struct(canon, *_deform_views(deform), n)
    _check(t_frames, "t_frames")
    _check(trace_grad, "trace_grad")
    if frame_scale is not None:
        _check(frame_scale, "frame_scale")
    F = int(t_frames.numel())
    if out is None:
        out = (torch.empty_like(canon), torch.empty_like(deform))
    gc, gd = out
    _check(gc, "g_canon")
    _check(gd, "g_deform")
    grads = _lib.pa_grads(gc.data_ptr(), gd[0].data_ptr(), gd[1].data_ptr(), gd[2].data_ptr())
    h = plan.handle if plan is not None else None
    need = int(_LIB.pa_adjoint_4d_workspace_size(ctypes.byref(geom.struct()), ctypes.byref(cs), F, h))
    workspace = _workspace(workspace, need, canon.device)
    _lib.check(_LIB.pa_adjoint_4d(ctypes.byref(geom.struct()), ctypes.byref(cs), t_frames.data_ptr(), F,
                                  trace_grad.data_ptr(), _ptr(frame_scale), ctypes.byref(grads),
                                  _lib.PA_ACCUMULATE if accumulate else 0, h, workspace.data_ptr(), workspace.numel(),
                                  _stream()), "pa_adjoint_4d")
    return gc, gd


def adam_step_scheduled(x: torch.Tensor, g: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr0: float,
                        step: torch.Tensor, step_size: int = 160, gamma: float = 0.1, beta1: float = 0.9,
                        beta2: float = 0.999, eps: float = 1e-8) -> None:
    """Adam whose step number t (and so the step-decayed learning rate and the
    bias corrections) is read from the device int32 tensor `step`."""
    for t, nm in ((x, "x"), (g, "g"), (m, "m"), (v, "v")):
        _check(t, nm)
    _check(step, "step", torch.int32)
    _lib.check(_LIB.pa_adam_step_scheduled(x.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), x.numel(),
                                           float(lr0), float(beta1), float(beta2), float(eps), int(step_size),
                                           float(gamma), step.data_ptr(), _stream()), "pa_adam_step_scheduled")


def step_increment(step: torch.Tensor) -> None:
    _check(step, "step", torch.int32)
    _lib.check(_LIB.pa_step_increment(step.data_ptr(), _stream()), "pa_step_increment")


# ---------------------------------------------------------------------------
# Autograd wrappers (the differentiation pattern: forward and adjoint as one
# torch.autograd.Function; 4D states are recomputed in backward, not stored).
# ---------------------------------------------------------------------------

class PAProject(torch.autograd.Function):
    """states [F, 5, stride] -> traces [F, S, T]."""

    @staticmethod
    def forward(ctx, state, geom: Geometry, n: Optional[int] = None):
        ctx.geom, ctx.n = geom, n
        ctx.save_for_backward(state)
        return forward(geom, state, n)

    @staticmethod
    def backward(ctx, g):
        (state,) = ctx.saved_tensors
        gs = adjoint(ctx.geom, g.contiguous(), state=state, n=ctx.n)
        return gs, None, None


class Buffers4D:
    """Preallocated workspaces and gradient outputs of one 4D problem, so that
    an IR iteration through autograd reuses the same device buffers every
    time (and a CUDA graph of it keeps fixed addresses): the 4D calls'
    workspaces, the loss workspace, the residual and the two gradients."""

    def __init__(self, geom: Geometry, canon: torch.Tensor, deform: torch.Tensor, t_frames: torch.Tensor,
                 n: Optional[int] = None, plan: Optional[Plan] = None):
        dev = canon.device
        F = int(t_frames.numel())
        self.fws = _workspace(None, forward_4d_workspace_size(geom, canon, deform, t_frames, n, plan), dev)
        self.aws = _workspace(None, adjoint_4d_workspace_size(geom, canon, deform, t_frames, n, plan), dev)
        self.lws = _workspace(None, int(_LIB.pa_loss_workspace_size(geom.n_sensors * geom.n_samples, F)), dev)
        self.resid = torch.empty(F, geom.n_sensors, geom.n_samples, dtype=torch.float32, device=dev)
        self.g_canon = torch.zeros_like(canon)
        self.g_deform = torch.zeros_like(deform)


class PAProject4D(torch.autograd.Function):
    """(canon [5, stride], deform [3, 5, Nb, stride] = (omega, theta, sigma))
    -> traces [F, S, T] through Eq. 1-2.

    Deformed states are recomputed per frame chunk rather than stored: the
    forward runs pa_forward_4d, and backward runs pa_adjoint_4d, which deforms
    each chunk again, takes its static adjoint and applies the chain rule of
    Eq. 1-2.  Nothing of shape [F, 5, N] is kept between the two.
    fused=True makes backward use the single fused 4D adjoint kernel
    (pa_adjoint's 4D mode, no workspace at all, lower occupancy).
    bufs: optional Buffers4D whose workspaces and gradient tensors are used
    instead of fresh allocations."""

    @staticmethod
    def forward(ctx, canon, deform, geom: Geometry, t_frames, n: Optional[int] = None, plan: Optional[Plan] = None,
                bufs: Optional[Buffers4D] = None, fused: bool = False):
        traces = forward_4d(geom, canon, deform, t_frames, n, plan=plan, workspace=bufs.fws if bufs else None)
        ctx.geom, ctx.n, ctx.plan, ctx.bufs, ctx.fused = geom, n, plan, bufs, fused
        ctx.save_for_backward(canon, deform, t_frames)
        return traces

    @staticmethod
    def backward(ctx, g):
        canon, deform, t_frames = ctx.saved_tensors
        bufs = ctx.bufs
        out = (bufs.g_canon, bufs.g_deform) if bufs else (torch.empty_like(canon), torch.empty_like(deform))
        if ctx.fused:
            adjoint(ctx.geom, g.contiguous(), canon=canon, omega=deform[0], theta=deform[1], sigma=deform[2],
                    t_frames=t_frames, n=ctx.n, out=(out[0], out[1][0], out[1][1], out[1][2]))
            gc, gd = out
        else:
            gc, gd = adjoint_4d(ctx.geom, g.contiguous(), canon, deform, t_frames, ctx.n, out=out, plan=ctx.plan,
                                workspace=bufs.aws if bufs else None)
        return gc, gd, None, None, None, None, None, None


class PALoss(torch.autograd.Function):
    """(pred, meas) [F, S, T] -> per-frame FP64 loss [F]; backward gives the
    residual 2 g_f (pred - meas) (and its negative for meas)."""

    @staticmethod
    def forward(ctx, pred, meas, bufs: Optional[Buffers4D] = None):
        loss, _ = residual_loss(pred, meas, want_loss=True, workspace=bufs.lws if bufs else None)
        ctx.save_for_backward(pred, meas)
        ctx.bufs = bufs
        return loss

    @staticmethod
    def backward(ctx, gl):
        pred, meas = ctx.saved_tensors
        scale = gl.to(torch.float32).contiguous()
        bufs = ctx.bufs
        _, resid = residual_loss(pred, meas, frame_scale=scale, want_loss=False, want_resid=True,
                                 resid_out=bufs.resid if bufs else None)
        gm = -resid if ctx.needs_input_grad[1] else None
        return resid, gm, None


# ---------------------------------------------------------------------------
# Imaging (Sec. 3.1-3.2, Tab. 1): UBP comparison reconstruction, ball cloud
# -> voxels, maximum amplitude projections and SSIM.

class Grid:
    """Voxel grid [nz, ny, nx]; voxel (ix, iy, iz) centred at origin + h (ix, iy, iz) (mm)."""

    def __init__(self, origin, h: float, shape):
        self.origin = tuple(float(v) for v in origin)
        self.h = float(h)
        self.shape = tuple(int(v) for v in shape)  # (nz, ny, nx)
        nz, ny, nx = self.shape
        self._struct = _lib.pa_grid((ctypes.c_float * 3)(*self.origin), self.h, nx, ny, nz)

    @classmethod
    def cube(cls, half_width: float, n: int, center=(0.0, 0.0, 0.0)) -> "Grid":
        """n^3 voxels filling the cube center +- half_width."""
        h = 2.0 * half_width / n
        origin = [c - half_width + 0.5 * h for c in center]
        return cls(origin, h, (n, n, n))

    def struct(self):
        return self._struct


def ubp_filter(traces: torch.Tensor, fs: float, t0: float, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """UBP filtering b = 2p - 2t dp/dt along the last axis of traces [..., T]."""
    _check(traces, "traces")
    T = int(traces.shape[-1])
    if out is None:
        out = torch.empty_like(traces)
    _check(out, "out")
    _lib.check(_LIB.pa_ubp_filter(traces.data_ptr(), int(traces.numel() // T), T, float(fs), float(t0),
                                  out.data_ptr(), _stream()), "pa_ubp_filter")
    return out


def ubp(geom: Geometry, b: torch.Tensor, grid: Grid, center=(0.0, 0.0, 0.0),
        out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """UBP back-projection of filtered traces b [S, T] onto grid -> [nz, ny, nx]."""
    _check(b, "b")
    if tuple(b.shape) != (geom.n_sensors, geom.n_samples):
        raise ValueError(f"b must be [{geom.n_sensors}, {geom.n_samples}], got {tuple(b.shape)}")
    if out is None:
        out = torch.empty(grid.shape, dtype=torch.float32, device=b.device)
    _check(out, "out")
    c = (ctypes.c_float * 3)(*[float(v) for v in center])
    _lib.check(_LIB.pa_ubp(ctypes.byref(geom.struct()), c, b.data_ptr(), ctypes.byref(grid.struct()),
                           out.data_ptr(), _stream()), "pa_ubp")
    return out


def splat(state: torch.Tensor, grid: Grid, kappa: float = 5.0, n: Optional[int] = None,
          out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Ball cloud [5, stride] (one frame) -> voxel grid [nz, ny, nx]."""
    state, bs, n = _balls_struct(state, n)
    if out is None:
        out = torch.empty(grid.shape, dtype=torch.float32, device=state.device)
    _check(out, "out")
    _lib.check(_LIB.pa_splat(ctypes.byref(bs), float(kappa), ctypes.byref(grid.struct()), out.data_ptr(),
                             _stream()), "pa_splat")
    return out


def maps(vol: torch.Tensor, grid: Grid):
    """Maximum amplitude projections of vol [nz, ny, nx]: (xy [ny, nx], yz [nz, ny], xz [nz, nx])."""
    _check(vol, "vol")
    nz, ny, nx = grid.shape
    if tuple(vol.shape) != (nz, ny, nx):
        raise ValueError(f"vol must be {grid.shape}, got {tuple(vol.shape)}")
    xy = torch.empty(ny, nx, dtype=torch.float32, device=vol.device)
    yz = torch.empty(nz, ny, dtype=torch.float32, device=vol.device)
    xz = torch.empty(nz, nx, dtype=torch.float32, device=vol.device)
    _lib.check(_LIB.pa_map(vol.data_ptr(), ctypes.byref(grid.struct()), xy.data_ptr(), yz.data_ptr(),
                           xz.data_ptr(), _stream()), "pa_map")
    return xy, yz, xz


def ssim(x: torch.Tensor, y: torch.Tensor, L: float = 1.0, want_map: bool = False,
         workspace: Optional[torch.Tensor] = None, minmax: bool = False):
    """Mean SSIM of images x, y [H, W] as a device float64 scalar (and the
    map).  minmax=True scales each image to [0, 1] by its own minimum and
    maximum first (L = 1)."""
    _check(x, "x")
    _check(y, "y")
    if x.shape != y.shape or x.dim() != 2:
        raise ValueError("x and y must be equal-shape 2D images")
    H, W = int(x.shape[0]), int(x.shape[1])
    need = int(_LIB.pa_ssim_workspace_size(H, W))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=x.device)
    mean = torch.empty((), dtype=torch.float64, device=x.device)
    m = torch.empty(max(H - 10, 0), max(W - 10, 0), dtype=torch.float32, device=x.device) if want_map else None
    _lib.check(_LIB.pa_ssim(x.data_ptr(), y.data_ptr(), H, W, float(L), _lib.PA_SSIM_MINMAX if minmax else 0,
                            _ptr(m), mean.data_ptr(),
                            workspace.data_ptr(), workspace.numel(), _stream()), "pa_ssim")
    return (mean, m) if want_map else mean
