"""Iterative reconstruction (IR) driver of 4D SlingBAG on the library's
kernels (Sec. 2.2, Fig. 2 stage 2; hyper-parameters of Sec. 3.2).

One IR iteration: deform every frame (Eq. 1-2) -> forward projection of all
frames -> per-frame FP64 L2 loss and residual -> 4D adjoint -> Adam on each
parameter group with the paper's learning rates and step decay (step_size
160, drop 0.1).  The 4D adjoint is, by default, the static adjoint over the
deformed states the forward already used followed by the chain rule of
Eq. 1-2 (pa_deform_backward); fused=True uses the single fused 4D kernel
instead, which needs no per-frame gradient buffer but runs at lower
occupancy.  The optimiser type
is not named in the paper; Adam is this library's reading.

Two execution forms of the same iteration:
  - batched: all frames in one launch per kernel; the whole iteration
    (deform, forward, loss, adjoint, step counter, Adam) is captured once in
    a CUDA graph and replayed (step_graph).  The Adam step number lives in
    device memory, so the decayed learning rate and bias corrections need no
    host scalars;
  - per-frame: F plain launch sequences, one frame each, gradients
    accumulated across frames (step_per_frame).
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import (Geometry, adam_step_scheduled, adjoint, deform_backward, deform_balls, forward, residual_loss,
               step_increment)

# Sec. 3.2: initial learning rates and step decay.  The paper states the
# rates without units.  Lengths here are in mm, and the coordinate and size
# rates are read as SI metres (5e-7 m = 5e-4 mm per Adam step): taken as mm
# they could move a ball by under 1e-4 mm over the whole decay schedule.  The
# pressure and the dimensionless deformation coefficients keep their numbers.
LR_COORD = 5e-7    # m
LR_PRESSURE = 5e-4
LR_STD = 5e-7      # m
LR_DEFORM = 5e-6
MM_PER_M = 1e3
STEP_SIZE = 160
DROP_RATE = 0.1


class GGBallIR:
    """Parameters, gradients, optimiser state and preallocated buffers of one
    4D reconstruction.

    canon: [5, stride] (x, y, z, a, p); deform: [3, 5, Nb, stride] holding
    omega, theta, sigma; t_frames: [F]; meas: [F, S, T]."""

    def __init__(self, geom: Geometry, canon: torch.Tensor, deform: torch.Tensor, t_frames: torch.Tensor,
                 meas: torch.Tensor, n: Optional[int] = None, fused: bool = False, lr_scale: float = 1.0):
        self.geom = geom
        self.canon = canon
        self.deform = deform
        self.t = t_frames
        self.meas = meas
        self.n = canon.shape[-1] if n is None else int(n)
        self.F = int(t_frames.numel())
        dev = canon.device
        self.g_canon = torch.zeros_like(canon)
        self.g_deform = torch.zeros_like(deform)
        self.m_canon, self.v_canon = torch.zeros_like(canon), torch.zeros_like(canon)
        self.m_deform, self.v_deform = torch.zeros_like(deform), torch.zeros_like(deform)
        stride = canon.shape[-1]
        self.state = torch.empty(self.F, 5, stride, dtype=torch.float32, device=dev)
        self.traces = torch.empty(self.F, geom.n_sensors, geom.n_samples, dtype=torch.float32, device=dev)
        self.resid = torch.empty_like(self.traces)
        self.loss = torch.empty(self.F, dtype=torch.float64, device=dev)
        self.fused = fused
        self.lr_scale = float(lr_scale)
        self.g_state = None if fused else torch.empty(self.F, 5, stride, dtype=torch.float32, device=dev)
        self.step_count = 0
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        self._fws = None
        self._lws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)

    # -- pieces ---------------------------------------------------------------
    def _omega(self):
        return self.deform[0]

    def _grads_tuple(self):
        return (self.g_canon, self.g_deform[0], self.g_deform[1], self.g_deform[2])

    def _forward_loss_adjoint(self):
        deform_balls(self.canon, self.deform[0], self.deform[1], self.deform[2], self.t, self.n, out=self.state)
        forward(self.geom, self.state, self.n, out=self.traces, workspace=self._fws)
        residual_loss(self.traces, self.meas, want_loss=True, want_resid=True, loss_out=self.loss,
                      resid_out=self.resid, workspace=self._lws)
        self._adjoint_4d(self.resid, self.t, self.state, self.g_state, accumulate=False)

    def _adjoint_4d(self, resid, t, state, g_state, accumulate):
        if self.fused:
            adjoint(self.geom, resid, canon=self.canon, omega=self.deform[0], theta=self.deform[1],
                    sigma=self.deform[2], t_frames=t, n=self.n, out=self._grads_tuple(), accumulate=accumulate)
        else:
            adjoint(self.geom, resid, state=state, n=self.n, out=g_state)
            deform_backward(self.canon, self.deform[0], self.deform[1], self.deform[2], t, g_state, self.n,
                            out=self._grads_tuple(), accumulate=accumulate)

    def lr_scale(self) -> float:
        """Step decay of Sec. 3.2 for the iteration last taken (1-based t):
        DROP_RATE ** floor((t - 1) / STEP_SIZE)."""
        return DROP_RATE ** (max(self.step_count - 1, 0) // STEP_SIZE)

    def _adam(self):
        # one device-side step counter; every group reads t from it
        step_increment(self.step_dev)
        self.step_count += 1
        assert LR_COORD == LR_STD  # x, y, z and a rows share one launch
        for lr0, x, g, m, v in (
                (LR_COORD * MM_PER_M, self.canon[:4], self.g_canon[:4], self.m_canon[:4], self.v_canon[:4]),
                (LR_PRESSURE, self.canon[4], self.g_canon[4], self.m_canon[4], self.v_canon[4]),
                (LR_DEFORM, self.deform, self.g_deform, self.m_deform, self.v_deform)):
            adam_step_scheduled(x.reshape(-1), g.reshape(-1), m.reshape(-1), v.reshape(-1), lr0 * self.lr_scale,
                                self.step_dev, STEP_SIZE, DROP_RATE)

    def _ensure_workspace(self):
        from . import forward_workspace_size
        # all frames at once (batched) and one frame (per-frame form)
        need = max(forward_workspace_size(self.geom, self.state, self.n),
                   forward_workspace_size(self.geom, self.state[:1], self.n))
        if need > 0 and (self._fws is None or self._fws.numel() < need):
            self._fws = torch.empty(need, dtype=torch.uint8, device=self.canon.device)

    # -- iteration forms -------------------------------------------------------
    def step(self) -> torch.Tensor:
        """One batched IR iteration with plain launches."""
        self._ensure_workspace()
        self._forward_loss_adjoint()
        self._adam()
        return self.loss

    def _iteration(self):
        self._forward_loss_adjoint()
        self._adam()

    def capture(self) -> None:
        """Capture one whole iteration in a CUDA graph.  The capture itself
        does not run the iteration; the warm-up iteration before it does."""
        self._ensure_workspace()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._iteration()  # warm-up (a real iteration)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        count = self.step_count
        with torch.cuda.graph(g):
            self._iteration()
        self.step_count = count  # capture recorded, did not run
        self.graph = g

    def step_graph(self) -> torch.Tensor:
        """One batched IR iteration replayed from the graph."""
        if self.graph is None:
            self.capture()
            return self.loss
        self.graph.replay()
        self.step_count += 1
        return self.loss

    def step_per_frame(self) -> torch.Tensor:
        """The same iteration as F plain single-frame launch sequences."""
        self._ensure_workspace()
        for f in range(self.F):
            tf = self.t[f:f + 1]
            st = self.state[f:f + 1]
            deform_balls(self.canon, self.deform[0], self.deform[1], self.deform[2], tf, self.n, out=st)
            forward(self.geom, st, self.n, out=self.traces[f:f + 1], workspace=self._fws)
            residual_loss(self.traces[f:f + 1], self.meas[f:f + 1], want_loss=True, want_resid=True,
                          loss_out=self.loss[f:f + 1], resid_out=self.resid[f:f + 1], workspace=self._lws)
            self._adjoint_4d(self.resid[f:f + 1], tf, st, None if self.fused else self.g_state[f:f + 1],
                             accumulate=f > 0)
        self._adam()
        return self.loss

    # -- checkpoint / resume -----------------------------------------------------
    def state_dict(self) -> dict:
        """Everything an iteration reads and updates: parameters, Adam moments and
        the step number (device tensors are copied to host memory)."""
        return {"canon": self.canon.cpu(), "deform": self.deform.cpu(), "m_canon": self.m_canon.cpu(),
                "v_canon": self.v_canon.cpu(), "m_deform": self.m_deform.cpu(), "v_deform": self.v_deform.cpu(),
                "step": int(self.step_count), "n": int(self.n), "lr_scale": self.lr_scale}

    def load_state_dict(self, sd: dict) -> None:
        """Resume from state_dict(); the next iteration continues the schedule
        exactly (bitwise, for the same measurements and launch configuration).
        A captured graph keeps pointing at these same buffers."""
        if int(sd["n"]) != self.n or tuple(sd["canon"].shape) != tuple(self.canon.shape) or \
                tuple(sd["deform"].shape) != tuple(self.deform.shape):
            raise ValueError("checkpoint does not match this problem's shapes")
        for name in ("canon", "deform", "m_canon", "v_canon", "m_deform", "v_deform"):
            getattr(self, name).copy_(sd[name])
        self.step_count = int(sd["step"])
        self.step_dev.fill_(self.step_count)
        self.lr_scale = float(sd.get("lr_scale", self.lr_scale))

    def launches_per_step(self, per_frame: bool = False) -> int:
        from . import forward_plan
        p = forward_plan(self.geom, self.state[:1] if per_frame else self.state, self.n)
        fwd = 1 + (1 if p["n_splits"] > 1 else 0)
        adj = 1 if self.fused else 2  # fused 4D adjoint, or static adjoint + deform backward
        core = 1 + fwd + 2 + adj  # deform, forward(+split reduce), loss partial+final, adjoint
        adam = 4  # step counter + three parameter groups
        return (core * self.F if per_frame else core) + adam


def init_deformation(n_basis: int, stride: int, device, omega_scale: float = 0.0, seed: int = 0) -> torch.Tensor:
    """Deformation parameters [3, 5, Nb, stride]: omega (zero, or small random
    weights drawn from a seeded CPU generator), theta evenly spaced on [0, 1],
    sigma = 1/Nb.  Built on `device` (only random omega passes through host
    memory)."""
    d = torch.empty(3, 5, n_basis, stride, dtype=torch.float32, device=device)
    if omega_scale != 0.0:
        g = torch.Generator(device="cpu").manual_seed(seed)
        d[0] = (torch.randn(5, n_basis, stride, generator=g) * omega_scale / math.sqrt(max(n_basis, 1))).to(device)
    else:
        d[0].zero_()
    if n_basis > 1:
        d[1] = torch.linspace(0.0, 1.0, n_basis, device=device).view(1, n_basis, 1)
    else:
        d[1].zero_()
    d[2].fill_(1.0 / n_basis)
    return d
