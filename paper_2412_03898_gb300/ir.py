"""Iterative reconstruction (IR) driver of 4D SlingBAG on the library's
kernels (Sec. 2.2, Fig. 2 stage 2; hyper-parameters of Sec. 3.2).

One IR iteration goes through torch.autograd: PAProject4D (deform every
frame by Eq. 1-2 and project it, pa_forward_4d) -> PALoss (per-frame FP64 L2
loss) -> torch.autograd.grad, whose backward runs the residual kernel and
pa_adjoint_4d -> Adam on each parameter group with the paper's learning rates
and step decay (step_size 160, drop 0.1).  The deformed states are
recomputed per frame chunk in both directions and never stored for all
frames, so device memory is the canonical cloud, its deformation parameters,
their gradients and Adam moments, the traces and one frame chunk, whatever
the number of frames.  fused=True makes backward use the single fused 4D
adjoint kernel instead.  The optimiser type is not named in the paper; Adam
is this library's reading.

Two execution forms of the same iteration:
  - batched: every kernel launch covers a chunk of frames (all frames when
    they fit the chunk); the whole iteration (forward, loss, backward, step
    counter, Adam) is captured once in a CUDA graph and replayed
    (step_graph).  The Adam step number lives in device memory, so the
    decayed learning rate and bias corrections need no host scalars;
  - per-frame: F plain launch sequences, one frame each, gradients
    accumulated across frames (step_per_frame).
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import (Buffers4D, Geometry, PALoss, PAProject4D, Plan, adam_step_scheduled, adjoint, adjoint_4d,
               forward_4d, residual_loss, step_increment)

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
                 meas: torch.Tensor, n: Optional[int] = None, fused: bool = False, lr_scale: float = 1.0,
                 plan: Optional[Plan] = None):
        self.geom = geom
        self.canon = canon
        self.deform = deform
        self.t = t_frames
        self.meas = meas
        self.n = canon.shape[-1] if n is None else int(n)
        self.F = int(t_frames.numel())
        self.plan = plan
        dev = canon.device
        self.m_canon, self.v_canon = torch.zeros_like(canon), torch.zeros_like(canon)
        self.m_deform, self.v_deform = torch.zeros_like(deform), torch.zeros_like(deform)
        self.bufs = Buffers4D(geom, canon, deform, t_frames, self.n, plan)
        self.g_canon, self.g_deform = self.bufs.g_canon, self.bufs.g_deform
        self.loss = torch.zeros(self.F, dtype=torch.float64, device=dev)
        self._ones = torch.ones(self.F, dtype=torch.float64, device=dev)
        self.fused = fused
        self.lr_scale = float(lr_scale)
        self.step_count = 0
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        # per-frame form: one frame of traces and residual
        self._tr1 = None
        self._res1 = None

    # -- pieces ---------------------------------------------------------------
    def _forward_loss_adjoint(self):
        """Loss and gradients of one iteration through torch.autograd."""
        c = self.canon.detach().requires_grad_()
        d = self.deform.detach().requires_grad_()
        traces = PAProject4D.apply(c, d, self.geom, self.t, self.n, self.plan, self.bufs, self.fused)
        loss = PALoss.apply(traces, self.meas, self.bufs)
        gc, gd = torch.autograd.grad(loss, (c, d), grad_outputs=(self._ones,))
        self.loss = loss.detach()
        return gc, gd

    def lr_decay(self) -> float:
        """Step decay of Sec. 3.2 for the iteration last taken (1-based t):
        DROP_RATE ** floor((t - 1) / STEP_SIZE)."""
        return DROP_RATE ** (max(self.step_count - 1, 0) // STEP_SIZE)

    def _adam(self, gc: torch.Tensor, gd: torch.Tensor):
        # one device-side step counter; every group reads t from it
        step_increment(self.step_dev)
        self.step_count += 1
        assert LR_COORD == LR_STD  # x, y, z and a rows share one launch
        for lr0, x, g, m, v in (
                (LR_COORD * MM_PER_M, self.canon[:4], gc[:4], self.m_canon[:4], self.v_canon[:4]),
                (LR_PRESSURE, self.canon[4], gc[4], self.m_canon[4], self.v_canon[4]),
                (LR_DEFORM, self.deform, gd, self.m_deform, self.v_deform)):
            adam_step_scheduled(x.reshape(-1), g.reshape(-1), m.reshape(-1), v.reshape(-1), lr0 * self.lr_scale,
                                self.step_dev, STEP_SIZE, DROP_RATE)

    # -- iteration forms -------------------------------------------------------
    def _iteration(self):
        gc, gd = self._forward_loss_adjoint()
        self._adam(gc, gd)

    def step(self) -> torch.Tensor:
        """One batched IR iteration with plain launches."""
        self._iteration()
        return self.loss

    def capture(self) -> None:
        """Capture one whole iteration in a CUDA graph.  The capture itself
        does not run the iteration; the warm-up iteration before it does."""
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
        """The same iteration as F plain single-frame launch sequences (no
        autograd, no graph), gradients accumulated across frames."""
        dev = self.canon.device
        if self._tr1 is None:
            self._tr1 = torch.empty(1, self.geom.n_sensors, self.geom.n_samples, dtype=torch.float32, device=dev)
            self._res1 = torch.empty_like(self._tr1)
        loss = torch.empty(self.F, dtype=torch.float64, device=dev)
        for f in range(self.F):
            tf = self.t[f:f + 1]
            forward_4d(self.geom, self.canon, self.deform, tf, self.n, out=self._tr1, plan=self.plan,
                       workspace=self.bufs.fws)
            residual_loss(self._tr1, self.meas[f:f + 1], want_loss=True, want_resid=True, loss_out=loss[f:f + 1],
                          resid_out=self._res1, workspace=self.bufs.lws)
            if self.fused:
                adjoint(self.geom, self._res1, canon=self.canon, omega=self.deform[0], theta=self.deform[1],
                        sigma=self.deform[2], t_frames=tf, n=self.n, accumulate=f > 0,
                        out=(self.g_canon, self.g_deform[0], self.g_deform[1], self.g_deform[2]))
            else:
                adjoint_4d(self.geom, self._res1, self.canon, self.deform, tf, self.n, accumulate=f > 0,
                           out=(self.g_canon, self.g_deform), plan=self.plan, workspace=self.bufs.aws)
        self.loss = loss
        self._adam(self.g_canon, self.g_deform)
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

    def frames_per_chunk(self) -> int:
        """Frames per launch of the 4D calls: the plan's, else the library's
        rule, as many as keep one chunk's states and state gradients within an
        eighth of the deformation parameters' memory: floor(3 Nb / 16)."""
        if self.plan is not None and self.plan.values()["frames_per_chunk"] > 0:
            return min(self.plan.values()["frames_per_chunk"], self.F)
        nb = int(self.deform.shape[2])
        return max(1, min(self.F, 3 * nb // 16))

    def launches_per_step(self, per_frame: bool = False) -> int:
        """Kernel launches of this library per iteration (memsets excluded)."""
        from . import forward_plan_for
        K = 1 if per_frame else self.frames_per_chunk()
        chunks = self.F if per_frame else -(-self.F // K)
        tiles = self.plan.values()["tiles"] if self.plan is not None else None
        p = forward_plan_for(self.geom, self.n, K, tiles)
        fwd = 2 + (1 if p["n_splits"] > 1 else 0)  # deform, forward (+ split reduce)
        adj = 1 if self.fused else 3                # fused 4D kernel, or deform + static adjoint + chain rule
        loss = 2 + 1                                # loss partial + final; residual partial
        adam = 4                                    # step counter + three parameter groups
        if self.fused:
            return chunks * fwd + loss + adj + adam if not per_frame else self.F * (fwd + loss + 1) + adam
        return chunks * (fwd + adj) + loss + adam if not per_frame else self.F * (fwd + loss + adj) + adam


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
