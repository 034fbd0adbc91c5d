"""GPU adjoint, deformation, loss and optimiser step vs the FP64 oracle
(through the C ABI).

Tolerances: gradients agree to relative L2 <= 1e-4 per group (FP32 path,
FP64 oracle); deformed states to 1e-6 relative (FP32 rounding of q0 (1+H));
FP64 losses to 1e-6 relative (each squared residual is formed in FP32)."""
import numpy as np
import pytest
import torch

import oracle
import pa_inputs
from gpu_common import GRAD_TOL, TRACE_TOL, dev_pad, geometry, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import paper_2412_03898_gb300 as m
    return m


def _geom_args(sc):
    return sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa


@pytest.mark.parametrize("seed,n,ns,T,F", [(11, 613, 19, 1024, 1), (12, 129, 40, 516, 3)])
def test_adjoint_static_parity(pa, seed, n, ns, T, F):
    sc = pa_inputs.small_scene(seed=seed, n_balls=n, n_sensors=ns, n_samples=T, n_frames=F)
    states = sc.frames if F > 1 else sc.balls[None]
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((F, ns, T)).astype(np.float32)
    geom = geometry(sc)
    got = pa.adjoint(geom, torch.from_numpy(g).cuda(), state=dev_pad(states), n=n)
    pa.device_error()
    fixed = pa.adjoint(geom, torch.from_numpy(g).cuda(), state=dev_pad(states), n=n, queue=False)
    assert torch.equal(got[..., :n], fixed[..., :n])  # work-queue and grid-stride schedules
    want = oracle.adjoint_state(states, sc.sensors, *_geom_args(sc), g)
    got = got[:, :, :n].cpu().numpy()
    for ch, name in enumerate("xyzap"):
        assert rel_l2(got[:, ch], want[:, ch]) <= GRAD_TOL, name


@pytest.mark.parametrize("T", [516, 520])
def test_adjoint_static_sensor_chunks_with_invalid_and_clipped_pairs(pa, T):
    """Sensors at three radii mixed within every 32-sensor chunk: windows
    inside the trace, windows clipped by its last sample, and windows past
    its end (no samples at all), so that the kernel compacts the valid pairs
    of a chunk and walks clipped windows.  T = 516 takes the float4 walk,
    T = 520 the 256-bit one."""
    sc = pa_inputs.small_scene(seed=17, n_balls=300, n_sensors=70, n_samples=T)
    n = sc.n_balls
    rng = np.random.default_rng(17)
    end = sc.c * (sc.t0 + (T - 1) / sc.fs)  # distance of the last sample
    scale = np.array([1.0, end / 40.0, 2.0], np.float32)[rng.integers(0, 3, sc.n_sensors)]
    sens = (sc.sensors * scale[None, :]).astype(np.float32)
    g = rng.standard_normal((1, sc.n_sensors, T)).astype(np.float32)
    geom = geometry(sc, sensors=sens)
    st = dev_pad(sc.balls)[None].contiguous()
    got = pa.adjoint(geom, torch.from_numpy(g).cuda(), state=st, n=n)
    pa.device_error()
    fixed = pa.adjoint(geom, torch.from_numpy(g).cuda(), state=st, n=n, queue=False)
    assert torch.equal(got[..., :n], fixed[..., :n])
    want = oracle.adjoint_state(sc.balls[None], sens, *_geom_args(sc), g)
    got = got[..., :n].cpu().numpy()
    for ch, name in enumerate("xyzap"):
        assert rel_l2(got[:, ch], want[:, ch]) <= GRAD_TOL, name


def test_adjoint_frame_scale_and_accumulate(pa):
    sc = pa_inputs.small_scene(seed=13, n_balls=100, n_sensors=8, n_samples=512, n_frames=2)
    rng = np.random.default_rng(1)
    g = torch.from_numpy(rng.standard_normal((2, 8, 512)).astype(np.float32)).cuda()
    geom = geometry(sc)
    st = dev_pad(sc.frames)
    base = pa.adjoint(geom, g, state=st, n=100)
    scale = torch.tensor([2.0, -0.5], device="cuda")
    scaled = pa.adjoint(geom, g, state=st, n=100, frame_scale=scale)
    torch.testing.assert_close(scaled[0], 2.0 * base[0], rtol=1e-6, atol=0)
    torch.testing.assert_close(scaled[1], -0.5 * base[1], rtol=1e-6, atol=0)
    acc = base.clone()
    pa.adjoint(geom, g, state=st, n=100, accumulate=True, out=acc)
    torch.testing.assert_close(acc, 2.0 * base, rtol=1e-6, atol=0)


def test_deform_parity(pa):
    rng = np.random.default_rng(21)
    n, nb, F = 1001, 65, 17
    canon = pa_inputs.small_scene(seed=21, n_balls=n, n_sensors=1, n_samples=64).balls
    om, th, sg = pa_inputs.random_deform(n, nb, rng, omega_scale=0.05)
    t = pa_inputs.frame_times(F)
    got = pa.deform_balls(dev_pad(canon), dev_pad(om), dev_pad(th), dev_pad(sg), torch.from_numpy(t).cuda(), n)
    pa.device_error()
    want = oracle.deform(canon, om, th, sg, t)
    got = got[:, :, :n].cpu().numpy()
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-3)
    assert err.max() <= 1e-6


def test_adjoint_4d_parity(pa):
    rng = np.random.default_rng(31)
    n, nb, F = 203, 65, 5
    sc = pa_inputs.small_scene(seed=31, n_balls=n, n_sensors=24, n_samples=1024)
    om, th, sg = pa_inputs.random_deform(n, nb, rng, omega_scale=0.05)
    t = pa_inputs.frame_times(F)
    g = rng.standard_normal((F, 24, 1024)).astype(np.float32)
    args = [dev_pad(x) for x in (sc.balls, om, th, sg)]
    gc, go, gt, gs = pa.adjoint(geometry(sc), torch.from_numpy(g).cuda(), canon=args[0], omega=args[1],
                                theta=args[2], sigma=args[3], t_frames=torch.from_numpy(t).cuda(), n=n)
    pa.device_error()
    want = oracle.adjoint_4d(sc.balls, om, th, sg, t, sc.sensors, *_geom_args(sc), g)
    for got, w, name in ((gc, want[0], "canon"), (go, want[1], "omega"), (gt, want[2], "theta"),
                         (gs, want[3], "sigma")):
        got = got[..., :n].cpu().numpy()
        for ch in range(5):
            assert rel_l2(got[ch], w[ch]) <= GRAD_TOL, (name, ch)


def test_loss_and_residual_parity(pa):
    rng = np.random.default_rng(41)
    F, S, T = 3, 17, 1028
    pred = rng.standard_normal((F, S, T)).astype(np.float32)
    meas = rng.standard_normal((F, S, T)).astype(np.float32)
    scale = np.array([1.0, 0.5, -2.0], dtype=np.float32)
    loss, resid = pa.residual_loss(torch.from_numpy(pred).cuda(), torch.from_numpy(meas).cuda(),
                                   frame_scale=torch.from_numpy(scale).cuda(), want_loss=True, want_resid=True)
    want = oracle.loss(pred, meas)
    np.testing.assert_allclose(loss.cpu().numpy(), want, rtol=1e-6)
    d = pred.astype(np.float64) - meas.astype(np.float64)
    np.testing.assert_allclose(resid.cpu().numpy(), 2 * scale[:, None, None] * d, rtol=1e-6, atol=1e-6)
    x = torch.from_numpy(pred).cuda()
    assert pa.sumsq(x).item() == pytest.approx(float(np.sum(pred.astype(np.float64) ** 2)), rel=1e-6)


def test_adam_step_matches_plain_torch_reference(pa):
    torch.manual_seed(0)
    n = 1030
    x = torch.randn(n, device="cuda")
    g = torch.randn(n, device="cuda")
    m = torch.randn(n, device="cuda") * 0.1
    v = torch.rand(n, device="cuda") * 0.1
    xr, mr, vr, gr = (t.cpu().clone() for t in (x, m, v, g))
    lr, b1, b2, eps, step = 1e-3, 0.9, 0.999, 1e-8, 7
    pa.adam_step(x, g, m, v, lr, step, b1, b2, eps)
    mr = b1 * mr + (1 - b1) * gr
    vr = b2 * vr + (1 - b2) * gr * gr
    xr = xr - lr * (mr / (1 - b1 ** step)) / ((vr / (1 - b2 ** step)).sqrt() + eps)
    # the kernel fuses b*m + (1-b)*g into one FMA; near cancellation that
    # differs from the two-rounding reference by ~ulp of the operands
    torch.testing.assert_close(x.cpu(), xr, rtol=1e-5, atol=1e-7)
    torch.testing.assert_close(m.cpu(), mr, rtol=1e-5, atol=1e-7)
    torch.testing.assert_close(v.cpu(), vr, rtol=1e-5, atol=1e-8)


def test_autograd_functions(pa):
    sc = pa_inputs.small_scene(seed=51, n_balls=150, n_sensors=10, n_samples=512, n_frames=2)
    geom = geometry(sc)
    st = dev_pad(sc.frames).requires_grad_(True)
    meas = torch.zeros(2, 10, 512, device="cuda")
    y = pa.PAProject.apply(st, geom, 150)
    loss = pa.PALoss.apply(y, meas).sum()
    loss.backward()
    y_o, _ = oracle.forward(sc.frames, sc.sensors, *_geom_args(sc))
    g_o = oracle.adjoint_state(sc.frames, sc.sensors, *_geom_args(sc), 2 * y_o)
    assert loss.item() == pytest.approx(float(np.sum(y_o ** 2)), rel=1e-5)
    got = st.grad[:, :, :150].cpu().numpy()
    for ch in range(5):
        assert rel_l2(got[:, ch], g_o[:, ch]) <= GRAD_TOL


@pytest.mark.parametrize("fused,frames_per_chunk", [(False, 0), (False, 3), (True, 0)])
def test_autograd_4d(pa, fused, frames_per_chunk):
    """PAProject4D (states recomputed per frame chunk in forward and
    backward, or the fused 4D adjoint kernel) against the oracle's traces and
    4D gradients, with chunks that divide F unevenly."""
    rng = np.random.default_rng(61)
    n, nb, F = 120, 8, 4
    sc = pa_inputs.small_scene(seed=61, n_balls=n, n_sensors=12, n_samples=512)
    om, th, sg = pa_inputs.random_deform(n, nb, rng)
    t = torch.from_numpy(pa_inputs.frame_times(F)).cuda()
    canon = dev_pad(sc.balls).requires_grad_(True)
    deform = torch.stack([dev_pad(x) for x in (om, th, sg)]).requires_grad_(True)
    plan = pa.Plan.from_values(frames_per_chunk=frames_per_chunk) if frames_per_chunk else None
    y = pa.PAProject4D.apply(canon, deform, geometry(sc), t, n, plan, None, fused)
    # a random upstream gradient: a constant one makes every true gradient a
    # near-cancelling sum (~1e-6 of its terms), which no FP32 path resolves
    up = rng.standard_normal(tuple(y.shape)).astype(np.float32)
    y.backward(torch.from_numpy(up).cuda())
    st_o = oracle.deform(sc.balls, om, th, sg, t.cpu().numpy())
    y_o, _ = oracle.forward(st_o, sc.sensors, *_geom_args(sc))
    assert rel_l2(y.detach().cpu().numpy(), y_o) <= TRACE_TOL
    want = oracle.adjoint_4d(sc.balls, om, th, sg, t.cpu().numpy(), sc.sensors, *_geom_args(sc), up)
    for got, w in zip((canon.grad, deform.grad[0], deform.grad[1], deform.grad[2]), want):
        assert rel_l2(got[..., :n].cpu().numpy(), w) <= GRAD_TOL


@pytest.mark.slow
def test_adjoint_full_size_sampled_balls(pa):
    """Static 100k-ball workload with all 576 sensors; gradients of 256 random
    balls against the oracle (which computes only those balls)."""
    sc = pa_inputs.config_scene(2)
    geom = geometry(sc)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((1, sc.n_sensors, sc.n_samples)).astype(np.float32)
    got = pa.adjoint(geom, torch.from_numpy(g).cuda(), state=dev_pad(sc.balls)[None], n=sc.n_balls)
    pa.device_error()
    pick = np.sort(rng.choice(sc.n_balls, 256, replace=False))
    want = oracle.adjoint_state(sc.balls[:, pick], sc.sensors, *_geom_args(sc), g)
    got = got[0][:, pick].cpu().numpy()
    for ch in range(5):
        assert rel_l2(got[ch], want[0, ch]) <= GRAD_TOL


def test_adjoint_wide_and_float4_walks_agree(pa):
    # A 32-byte aligned residual with T % 8 == 0 takes the 256-bit walk; the
    # same values at a 16-byte (not 32-byte) aligned address take the float4
    # walk.  Both must match the oracle and each other (summation order only).
    sc = pa_inputs.small_scene(seed=71, n_balls=701, n_sensors=23, n_samples=1024)
    geom = geometry(sc)
    st = dev_pad(sc.balls)[None]
    g = np.random.default_rng(71).standard_normal((1, sc.n_sensors, sc.n_samples)).astype(np.float32)
    g32 = torch.from_numpy(g).cuda()
    assert g32.data_ptr() % 32 == 0
    buf = torch.empty(g.size + 4, device="cuda")
    g16 = buf[4:].view(1, sc.n_sensors, sc.n_samples)
    g16.copy_(g32)
    assert g16.data_ptr() % 16 == 0 and g16.data_ptr() % 32 != 0
    wide = pa.adjoint(geom, g32, state=st, n=sc.n_balls)[..., :sc.n_balls].cpu().numpy()
    narrow = pa.adjoint(geom, g16, state=st, n=sc.n_balls)[..., :sc.n_balls].cpu().numpy()
    pa.device_error()
    want = oracle.adjoint_state(sc.balls[None], sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g)
    for ch in range(5):
        assert rel_l2(wide[:, ch], want[:, ch]) <= GRAD_TOL, ch
        assert rel_l2(narrow[:, ch], want[:, ch]) <= GRAD_TOL, ch
        assert rel_l2(wide[:, ch], narrow[:, ch]) <= 1e-5, ch


def test_4d_calls_chunks_edges_and_accumulate(pa):
    """pa_forward_4d equals pa_deform_balls + pa_forward_ex per frame chunk (the
    same launches), for chunk sizes that do and do not divide F and larger
    than F; pa_adjoint_4d accumulates; empty clouds and zero frames."""
    rng = np.random.default_rng(91)
    n, nb, F = 211, 5, 7
    sc = pa_inputs.small_scene(seed=91, n_balls=n, n_sensors=9, n_samples=516)
    om, th, sg = pa_inputs.random_deform(n, nb, rng)
    geom = geometry(sc)
    t = torch.from_numpy(pa_inputs.frame_times(F)).cuda()
    canon = dev_pad(sc.balls)
    deform = torch.stack([dev_pad(x) for x in (om, th, sg)])
    g = torch.from_numpy(rng.standard_normal((F, 9, 516)).astype(np.float32)).cuda()
    ref_gc, ref_gd = None, None
    for K in (1, 3, 7, 20):
        plan = pa.Plan.from_values(frames_per_chunk=K)
        y = pa.forward_4d(geom, canon, deform, t, n, plan=plan)
        for f0 in range(0, F, K):
            k = min(K, F - f0)
            st = pa.deform_balls(canon, deform[0], deform[1], deform[2], t[f0:f0 + k].contiguous(), n)
            assert torch.equal(y[f0:f0 + k], pa.forward(geom, st, n)), (K, f0)
        gc, gd = pa.adjoint_4d(geom, g, canon, deform, t, n, plan=plan)
        if ref_gc is None:
            ref_gc, ref_gd = gc, gd
        else:  # chunking changes only the order of the per-chunk sums
            torch.testing.assert_close(gc[:, :n], ref_gc[:, :n], rtol=1e-5, atol=1e-6 * float(ref_gc.abs().max()))
            torch.testing.assert_close(gd[..., :n], ref_gd[..., :n], rtol=1e-5, atol=1e-6 * float(ref_gd.abs().max()))
    gc2, gd2 = pa.adjoint_4d(geom, g, canon, deform, t, n, out=(ref_gc.clone(), ref_gd.clone()), accumulate=True)
    # (padding columns past n are never written)
    torch.testing.assert_close(gc2[:, :n], 2 * ref_gc[:, :n], rtol=1e-6, atol=1e-7 * float(ref_gc[:, :n].abs().max()))
    torch.testing.assert_close(gd2[..., :n], 2 * ref_gd[..., :n], rtol=1e-6,
                               atol=1e-7 * float(ref_gd[..., :n].abs().max()))
    # empty cloud: zero traces, nothing to accumulate; zero frames: zero gradients
    y0 = pa.forward_4d(geom, canon, deform, t, 0)
    assert not torch.any(y0)
    z = pa.adjoint_4d(geom, g[:0].contiguous(), canon, deform, t[:0].contiguous(), n,
                      out=(torch.full_like(canon, 5.0), torch.full_like(deform, 5.0)))
    assert not torch.any(z[0][:, :n]) and not torch.any(z[1][..., :n])
    pa.device_error()
