"""Every benchmark workload at its full size, in the launch configuration the
benchmark times, against the FP64 oracle: static-2k in full; 4d-100k-20f and
batched-16 on sampled outputs the oracle computes one by one (sensor traces,
ball gradients).  Tolerances: traces rel-L2 <= 1e-5, gradients <= 1e-4."""
import numpy as np
import pytest
import torch

import oracle
import pa_inputs
from gpu_common import GRAD_TOL, TRACE_TOL, dev_pad, geometry, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pa():
    import paper_2412_03898_gb300 as m
    return m


def test_static_2k_full(pa):
    sc = pa_inputs.config_scene(1)
    geom = geometry(sc)
    st = dev_pad(sc.balls)[None]
    y = pa.forward(geom, st, sc.n_balls)
    y_o, _ = oracle.forward(sc.balls, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    assert rel_l2(y.cpu().numpy(), y_o) <= TRACE_TOL
    g = np.random.default_rng(71).standard_normal(y_o.shape).astype(np.float32)
    got = pa.adjoint(geom, torch.from_numpy(g).cuda(), state=st, n=sc.n_balls)[..., :sc.n_balls].cpu().numpy()
    pa.device_error()
    want = oracle.adjoint_state(sc.balls[None], sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g)
    for ch in range(5):
        assert rel_l2(got[:, ch], want[:, ch]) <= GRAD_TOL, ch


def test_4d_100k_20f_ir_path_sampled(pa):
    """The IR's 4D path on the full workload: deform all 20 frames, forward in
    one launch, static adjoint over the frames, chain rule of Eq. 1-2."""
    sc = pa_inputs.config_scene(3)
    n, F, nb = sc.n_balls, sc.n_frames, 65
    rng = np.random.default_rng(72)
    om, th, sg = pa_inputs.random_deform(n, nb, rng, omega_scale=0.02)
    t = pa_inputs.frame_times(F)
    geom = geometry(sc)
    canon, omega, theta, sigma = (dev_pad(x) for x in (sc.balls, om, th, sg))
    t_dev = torch.from_numpy(t).cuda()
    state = pa.deform_balls(canon, omega, theta, sigma, t_dev, n)
    traces = pa.forward(geom, state, n)
    frames = [0, F // 2, F - 1]
    pick_s = np.sort(rng.choice(sc.n_sensors, 6, replace=False))
    for f in frames:
        st_o = oracle.deform(sc.balls, om, th, sg, t[f:f + 1])
        y_o, _ = oracle.forward(st_o, sc.sensors[:, pick_s], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
        assert rel_l2(traces[f, pick_s].cpu().numpy(), y_o[0]) <= TRACE_TOL, f
    g = torch.zeros_like(traces)
    g_host = {f: rng.standard_normal((1, sc.n_sensors, sc.n_samples)).astype(np.float32) for f in frames}
    for f in frames:
        g[f] = torch.from_numpy(g_host[f][0]).cuda()
    g_state = pa.adjoint(geom, g, state=state, n=n)
    got = pa.deform_backward(canon, omega, theta, sigma, t_dev, g_state, n)
    pa.device_error()
    pick = np.sort(rng.choice(n, 24, replace=False))
    want = None
    for f in frames:
        w = oracle.adjoint_4d(sc.balls[:, pick], om[:, :, pick], th[:, :, pick], sg[:, :, pick], t[f:f + 1],
                              sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g_host[f])
        want = w if want is None else tuple(a + b for a, b in zip(want, w))
    for arr, w, name in zip(got, want, ("canon", "omega", "theta", "sigma")):
        a = arr[..., pick].cpu().numpy()
        for ch in range(5):
            assert rel_l2(a[ch], w[ch]) <= GRAD_TOL, (name, ch)


def test_batched_16_sampled(pa):
    """The 16 uneven scenes as one persistent forward (with the tiles the
    autotuner picks, as timed) and one persistent adjoint; per scene, 6
    sampled sensors' traces and 24 sampled balls' gradients of one frame
    against the oracle."""
    from paper_2412_03898_gb300.autotune import tune_batched
    rng = np.random.default_rng(73)
    raw = pa_inputs.config_scene(5)
    scenes = []
    for sc in raw:
        st = dev_pad(sc.frames if sc.frames is not None else sc.balls[None])
        b = pa.Scene(geometry(sc), st, sc.n_balls)
        scenes.append(b)
    plan = tune_batched(scenes)
    for b in scenes:
        b.traces = None
    pa.forward_batched(scenes, plan=plan)
    for b in scenes:
        b.trace_grad = torch.randn_like(b.traces)
    pa.adjoint_batched(scenes)
    pa.device_error()
    for sc, b in zip(raw, scenes):
        states = sc.frames if sc.frames is not None else sc.balls[None]
        f = int(rng.integers(b.F))
        pick_s = np.sort(rng.choice(sc.n_sensors, 6, replace=False))
        y_o, _ = oracle.forward(states[f], sc.sensors[:, pick_s], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
        assert rel_l2(b.traces[f, pick_s].cpu().numpy(), y_o[0]) <= TRACE_TOL, sc.name
        pick = np.sort(rng.choice(sc.n_balls, 24, replace=False))
        g = b.trace_grad[f:f + 1].cpu().numpy()
        want = oracle.adjoint_state(states[f][None][:, :, pick], sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples,
                                    sc.kappa, g)
        got = b.grad_state[f, :, pick].cpu().numpy()
        for ch in range(5):
            assert rel_l2(got[ch], want[0, ch]) <= GRAD_TOL, (sc.name, ch)
