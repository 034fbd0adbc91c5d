"""Chain rule of Eq. 1-2 on its own (pa_deform_backward), and the unfused 4D
adjoint it enables: deform -> static adjoint -> deform backward, against the
FP64 oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import pa_inputs
from gpu_common import GRAD_TOL, dev_pad, geometry, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import paper_2412_03898_gb300 as m
    return m


def _params(seed, n, nb):
    rng = np.random.default_rng(seed)
    canon = pa_inputs.small_scene(seed=seed, n_balls=n, n_sensors=1, n_samples=64).balls
    om, th, sg = pa_inputs.random_deform(n, nb, rng, omega_scale=0.05)
    return rng, canon, om, th, sg


@pytest.mark.parametrize("n,nb,F", [(1001, 65, 17), (5, 1, 1), (130, 7, 50)])
def test_deform_backward_parity(pa, n, nb, F):
    rng, canon, om, th, sg = _params(51, n, nb)
    t = pa_inputs.frame_times(F)
    g = rng.standard_normal((F, 5, n)).astype(np.float32)
    got = pa.deform_backward(dev_pad(canon), dev_pad(om), dev_pad(th), dev_pad(sg), torch.from_numpy(t).cuda(),
                             dev_pad(g), n)
    pa.device_error()
    want = oracle.deform_backward(canon, om, th, sg, t, g)
    for arr, w, name in zip(got, want, ("canon", "omega", "theta", "sigma")):
        arr = arr[..., :n].cpu().numpy()
        for ch in range(5):
            assert rel_l2(arr[ch], w[ch]) <= GRAD_TOL, (name, ch)


def test_deform_backward_accumulate(pa):
    rng, canon, om, th, sg = _params(52, 257, 65)
    F = 4
    t = torch.from_numpy(pa_inputs.frame_times(F)).cuda()
    g = dev_pad(rng.standard_normal((F, 5, 257)).astype(np.float32))
    args = [dev_pad(x) for x in (canon, om, th, sg)]
    base = pa.deform_backward(*args, t, g, 257)
    acc = tuple(b.clone() for b in base)
    pa.deform_backward(*args, t, g, 257, out=acc, accumulate=True)
    for a, b in zip(acc, base):  # the padding columns past n are never written
        torch.testing.assert_close(a[..., :257], 2.0 * b[..., :257], rtol=1e-6, atol=0)


def test_deform_backward_domain_error(pa):
    rng, canon, om, th, sg = _params(53, 64, 3)
    sg = sg.copy()
    sg[2, 1, 10] = 0.0
    t = torch.from_numpy(pa_inputs.frame_times(3)).cuda()
    g = dev_pad(rng.standard_normal((3, 5, 64)).astype(np.float32))
    out = pa.deform_backward(*[dev_pad(x) for x in (canon, om, th, sg)], t, g, 64)
    with pytest.raises(pa.PAError):
        pa.device_error()
    # the skipped term gets zero gradient; the others are finite
    assert float(out[1][2, 1, 10]) == 0.0 and float(out[2][2, 1, 10]) == 0.0
    assert all(bool(torch.isfinite(o).all()) for o in out)


def test_unfused_4d_adjoint_matches_oracle(pa):
    rng = np.random.default_rng(31)
    n, nb, F = 203, 65, 5
    sc = pa_inputs.small_scene(seed=31, n_balls=n, n_sensors=24, n_samples=1024)
    om, th, sg = pa_inputs.random_deform(n, nb, rng, omega_scale=0.05)
    t = pa_inputs.frame_times(F)
    g = rng.standard_normal((F, 24, 1024)).astype(np.float32)
    args = [dev_pad(x) for x in (sc.balls, om, th, sg)]
    t_dev = torch.from_numpy(t).cuda()
    geom = geometry(sc)
    state = pa.deform_balls(*args, t_dev, n)
    g_state = pa.adjoint(geom, torch.from_numpy(g).cuda(), state=state, n=n)
    got = pa.deform_backward(*args, t_dev, g_state, n)
    fused = pa.adjoint(geom, torch.from_numpy(g).cuda(), canon=args[0], omega=args[1], theta=args[2],
                       sigma=args[3], t_frames=t_dev, n=n)
    pa.device_error()
    want = oracle.adjoint_4d(sc.balls, om, th, sg, t, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g)
    for arr, fu, w, name in zip(got, fused, want, ("canon", "omega", "theta", "sigma")):
        a = arr[..., :n].cpu().numpy()
        for ch in range(5):
            assert rel_l2(a[ch], w[ch]) <= GRAD_TOL, (name, ch)
            assert rel_l2(a[ch], fu[..., :n].cpu().numpy()[ch]) <= GRAD_TOL, (name, ch)
