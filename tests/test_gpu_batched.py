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


def test_plan_through_the_c_abi_tunes_and_matches_oracle(pa):
    """pa_plan_create (timed candidates) called through ctypes, then
    pa_forward_batched and pa_adjoint_batched with that plan: each scene equals
    the oracle, and the plan reads back as tuned with legal values."""
    import ctypes
    from paper_2412_03898_gb300 import _lib
    lib = _lib.load()
    scs = _scenes()
    rng = np.random.default_rng(9)
    batch = []
    for sc in scs:
        st = dev_pad(_states(sc))
        b = pa.Scene(geometry(sc), st, sc.n_balls)
        b.traces = torch.empty(b.F, sc.n_sensors, sc.n_samples, device="cuda")
        b.trace_grad = torch.from_numpy(
            rng.standard_normal((b.F, sc.n_sensors, sc.n_samples)).astype(np.float32)).cuda()
        b.grad_state = torch.empty_like(st)
        batch.append(b)
    arr = (_lib.pa_scene * len(batch))(*[b.struct() for b in batch])
    need = lib.pa_plan_workspace_size(arr, len(batch))
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = ctypes.c_void_p()
    assert lib.pa_plan_create(arr, len(batch), _lib.PA_PLAN_TUNE, ws.data_ptr(), ws.numel(), stream,
                              ctypes.byref(h)) == 0
    vals = (ctypes.c_int32 * 7)()
    ms = (ctypes.c_float * 2)()
    assert lib.pa_plan_get(h, vals, ms) == 0
    # tiles: a timed candidate, or all 0 when the built-in heuristic won
    assert 0 <= vals[0] <= 16 and vals[1] % 4 == 0 and vals[4] in (0, 1, 2, 4, 8, 16) and vals[6] in (1, 2, 4, 8, 16)
    assert ms[0] > 0 and ms[1] > 0
    for b in batch:
        b.traces.fill_(3.0)
    assert lib.pa_forward_batched(arr, len(batch), 0, h, ws.data_ptr(), ws.numel(), stream) == 0
    assert lib.pa_adjoint_batched(arr, len(batch), 0, h, ws.data_ptr(), ws.numel(), stream) == 0
    pa.device_error()
    lib.pa_plan_destroy(h)
    for sc, b in zip(scs, batch):
        y_o, _ = oracle.forward(_states(sc), sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
        assert rel_l2(b.traces.cpu().numpy(), y_o) <= TRACE_TOL
        want = oracle.adjoint_state(_states(sc), sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa,
                                    b.trace_grad.cpu().numpy())
        got = b.grad_state[..., :sc.n_balls].cpu().numpy()
        for ch in range(5):
            assert rel_l2(got[:, ch], want[:, ch]) <= GRAD_TOL


def test_single_scene_plan_and_autotune_cache(pa, tmp_path, monkeypatch):
    """A one-scene tuned plan (ball splits by the planner) drives pa_forward_ex
    to the oracle's traces; the autotuner's file cache round-trips it."""
    from paper_2412_03898_gb300 import autotune
    monkeypatch.setenv("PA_TILE_CACHE", str(tmp_path / "tiles.json"))
    monkeypatch.setattr(autotune, "_cache", {})
    sc = _scenes()[2]
    st = dev_pad(_states(sc))
    geom = geometry(sc)
    plan = autotune.tune_forward_plan(geom, st, sc.n_balls)
    v = plan.values()
    assert v["tuned"] and v["forward_ms"] > 0
    y = pa.forward(geom, st, sc.n_balls, tiles=v["tiles"])
    y_o, _ = oracle.forward(_states(sc), sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    assert rel_l2(y.cpu().numpy(), y_o) <= TRACE_TOL
    monkeypatch.setattr(autotune, "_cache", {})
    again = autotune.tune_forward_plan(geom, st, sc.n_balls)  # from the file, not re-timed
    assert again.values()["tiles"] == v["tiles"] and not again.values()["tuned"]


def test_forward_batched_ball_splits_equal_single_and_accumulate(pa):
    """With ball splits (partials in the workspace, summed in split order)
    every scene's traces equal pa_forward_ex's with the same tiles and split
    count bit for bit; accumulate adds onto existing traces."""
    tiles = (16, 1536, 256, 3, 16)
    scs = _scenes()
    batch = [pa.Scene(geometry(sc), dev_pad(_states(sc)), sc.n_balls) for sc in scs]
    pa.forward_batched(batch, tiles=tiles)
    pa.device_error()
    for sc, b in zip(scs, batch):
        single = pa.forward(geometry(sc), dev_pad(_states(sc)), sc.n_balls, tiles=tiles)
        assert torch.equal(b.traces, single), sc.name
    first = [b.traces.clone() for b in batch]
    pa.forward_batched(batch, tiles=tiles, accumulate=True)
    for f0, b in zip(first, batch):
        torch.testing.assert_close(b.traces, 2 * f0, rtol=1e-6, atol=1e-7 * float(f0.abs().max()))
