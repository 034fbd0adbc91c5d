"""Batched persistent launches over several uneven scenes (through the C ABI).

Each scene's result must equal the single-scene entry point's bit for bit
(the same per-item code runs, only the work order differs), and agree with the
FP64 oracle to the trace / gradient tolerances."""
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


def _scenes():
    # uneven ball, sensor, sample and frame counts (ragged against every tile)
    specs = [(11, 1301, 37, 1028, 3), (12, 257, 5, 516, 1), (13, 2049, 19, 2052, 2), (14, 77, 64, 256, 4),
             (15, 603, 1, 1024, 1)]
    out = []
    for seed, n, s, t, f in specs:
        sc = pa_inputs.small_scene(seed=seed, n_balls=n, n_sensors=s, n_samples=t, n_frames=f)
        out.append(sc)
    return out


def _states(sc):
    return sc.frames if sc.frames is not None else sc.balls[None]


@pytest.mark.parametrize("tiles", [(12, 2048, 256, 1, 8), (16, 1536, 512, 1, 16), (7, 512, 128, 1, 2)])
def test_forward_batched_equals_single_and_oracle(pa, tiles):
    scs = _scenes()
    batch = [pa.Scene(geometry(sc), dev_pad(_states(sc)), sc.n_balls) for sc in scs]
    pa.forward_batched(batch, tiles=tiles)
    pa.device_error()
    for sc, b in zip(scs, batch):
        single = pa.forward(geometry(sc), dev_pad(_states(sc)), sc.n_balls, tiles=tiles)
        assert torch.equal(b.traces, single)
        y_o, _ = oracle.forward(_states(sc), sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
        assert rel_l2(b.traces.cpu().numpy(), y_o) <= TRACE_TOL


def test_forward_batched_default_tiles_and_accumulate(pa):
    scs = _scenes()
    batch = [pa.Scene(geometry(sc), dev_pad(_states(sc)), sc.n_balls) for sc in scs]
    pa.forward_batched(batch)
    first = [b.traces.clone() for b in batch]
    pa.forward_batched(batch, accumulate=True)
    for f0, b in zip(first, batch):
        torch.testing.assert_close(b.traces, 2 * f0, rtol=1e-6, atol=1e-7 * float(f0.abs().max()))


def test_forward_batched_empty_scenes(pa):
    sc = _scenes()[1]
    empty = pa.Scene(geometry(sc), torch.zeros(2, 5, 4, device="cuda"), 0)
    empty.traces = torch.full((2, sc.n_sensors, sc.n_samples), 7.0, device="cuda")
    real = pa.Scene(geometry(sc), dev_pad(_states(sc)), sc.n_balls)
    pa.forward_batched([empty, real])
    assert not torch.any(empty.traces)
    assert torch.any(real.traces)
    with pytest.raises(ValueError):
        pa.forward_batched([real] * 65)


def test_adjoint_batched_equals_single_and_oracle(pa):
    scs = _scenes()
    rng = np.random.default_rng(3)
    batch = []
    for sc in scs:
        st = dev_pad(_states(sc))
        g = torch.from_numpy(rng.standard_normal((st.shape[0], sc.n_sensors, sc.n_samples)).astype(np.float32))
        batch.append(pa.Scene(geometry(sc), st, sc.n_balls, trace_grad=g.cuda()))
    pa.adjoint_batched(batch)
    pa.device_error()
    for sc, b in zip(scs, batch):
        single = pa.adjoint(b.geom, b.trace_grad, state=b.state, n=sc.n_balls)
        assert torch.equal(b.grad_state[..., :sc.n_balls], single[..., :sc.n_balls])
        want = oracle.adjoint_state(_states(sc), sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa,
                                    b.trace_grad.cpu().numpy())
        got = b.grad_state[..., :sc.n_balls].cpu().numpy()
        for ch in range(5):
            assert rel_l2(got[:, ch], want[:, ch]) <= GRAD_TOL


def test_tune_batched_accepts_every_default_candidate(pa):
    from paper_2412_03898_gb300 import autotune
    scs = _scenes()
    batch = [pa.Scene(geometry(sc), dev_pad(_states(sc)), sc.n_balls) for sc in scs]
    best = autotune.tune_batched(batch, reps=1)
    assert tuple(best) in [tuple(c) for c in autotune.DEFAULT_CANDIDATES]
    pa.forward_batched(batch, tiles=best)
    pa.device_error()
    for sc, b in zip(scs, batch):
        y_o, _ = oracle.forward(_states(sc), sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
        assert rel_l2(b.traces.cpu().numpy(), y_o) <= TRACE_TOL
