"""Full-size 4D workload (1,000,000 balls in a 60 mm vessel tree, 1024 sensors
on an 80 mm hemisphere, 4096 samples, 50 frames, Nb = 65) in the launch
configuration the IR uses for it (pa_forward_4d / pa_adjoint_4d, states
recomputed per frame chunk), and through the fused 4D adjoint, checked on
sampled outputs the FP64 oracle can compute one by one: traces of 24 random
sensors at the first, middle and last frame, and the 4D gradients of 96
random balls for a residual that is non-zero on those three frames (the oracle sums its
per-frame gradients, which the chain rule of Eq. 1-2 makes exact)."""
import numpy as np
import pytest
import torch

import oracle
import pa_inputs
from gpu_common import GRAD_TOL, TRACE_TOL, dev_pad, geometry, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_large_4d_sampled_parity():
    import paper_2412_03898_gb300 as pa
    sc = pa_inputs.config_scene(4)
    n, F, nb = sc.n_balls, sc.n_frames, 65
    rng = np.random.default_rng(44)
    om, th, sg = pa_inputs.random_deform(n, nb, rng, omega_scale=0.02)
    t = pa_inputs.frame_times(F)
    geom = geometry(sc)
    canon = dev_pad(sc.balls)
    deform = torch.stack([dev_pad(x) for x in (om, th, sg)])
    omega, theta, sigma = deform[0], deform[1], deform[2]
    t_dev = torch.from_numpy(t).cuda()
    traces = pa.forward_4d(geom, canon, deform, t_dev, n)
    pa.device_error()
    frames = [0, F // 2, F - 1]
    pick_s = np.sort(rng.choice(sc.n_sensors, 24, replace=False))
    # pa_forward over all 50 frames' stored states: split partials bounded at
    # 1 GiB by frame chunks inside the call
    state = pa.deform_balls(canon, omega, theta, sigma, t_dev, n)
    ws_bytes = pa.forward_workspace_size(geom, state, n)
    assert 0 < ws_bytes <= 1 << 30
    traces_all = pa.forward(geom, state, n)
    pa.device_error()
    del state
    for f in frames:
        st_o = oracle.deform(sc.balls, om, th, sg, t[f:f + 1])
        y_o, _ = oracle.forward(st_o, sc.sensors[:, pick_s], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
        for form, tr in (("forward_4d", traces), ("forward", traces_all)):
            got = tr[f, pick_s].cpu().numpy()
            assert rel_l2(got, y_o[0]) <= TRACE_TOL, (form, f)
    del traces, traces_all

    g = torch.zeros(F, sc.n_sensors, sc.n_samples, device="cuda")
    g_host = {f: rng.standard_normal((1, sc.n_sensors, sc.n_samples)).astype(np.float32) for f in frames}
    for f in frames:
        g[f] = torch.from_numpy(g_host[f][0]).cuda()
    pick = np.sort(rng.choice(n, 96, replace=False))
    want = None
    for f in frames:
        w = oracle.adjoint_4d(sc.balls[:, pick], om[:, :, pick], th[:, :, pick], sg[:, :, pick], t[f:f + 1],
                              sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g_host[f])
        want = w if want is None else tuple(a + b for a, b in zip(want, w))
    gc, gd = pa.adjoint_4d(geom, g, canon, deform, t_dev, n)
    pa.device_error()
    fused = pa.adjoint(geom, g, canon=canon, omega=omega, theta=theta, sigma=sigma, t_frames=t_dev, n=n)
    pa.device_error()
    for form, grads in (("recompute", (gc, gd[0], gd[1], gd[2])), ("fused", fused)):
        for got, w, name in zip(grads, want, ("canon", "omega", "theta", "sigma")):
            arr = got[..., pick].cpu().numpy()
            for ch in range(5):
                assert rel_l2(arr[ch], w[ch]) <= GRAD_TOL, (form, name, ch)
