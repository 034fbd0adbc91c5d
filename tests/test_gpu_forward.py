"""GPU forward projection vs the FP64 oracle (through the C ABI).

Tolerance: traces agree to relative L2 <= 1e-5 (FP32 path against FP64).
Sizes span several sensor tiles, sample tiles and TMA ball stages, with
ragged tails in each (N, S, T not multiples of the tile sizes)."""
import numpy as np
import pytest
import torch

import oracle
import pa_inputs
from gpu_common import TRACE_TOL, dev_pad, geometry, max_rel_elem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import paper_2412_03898_gb300 as m
    return m


def _oracle_traces(sc, state=None):
    y, n = oracle.forward(sc.balls if state is None else state, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples,
                          sc.kappa)
    return y, n


@pytest.mark.parametrize("tiles", [None, (8, 256, 128, 3, 4), (5, 1024, 64, 1, 1), (16, 128, 512, 2, 8), (1, 1028, 4, 7, 2),
                                   (12, 1536, 384, 0, 16)])
def test_forward_parity_tiles(pa, tiles):
    sc = pa_inputs.small_scene(seed=1, n_balls=1003, n_sensors=37, n_samples=1028)
    geom = geometry(sc)
    state = dev_pad(sc.balls)[None]
    y = pa.forward(geom, state, sc.n_balls, tiles=tiles)
    pa.device_error()
    y_o, _ = _oracle_traces(sc)
    got = y.cpu().numpy()
    assert rel_l2(got, y_o) <= TRACE_TOL
    assert max_rel_elem(got, y_o) <= 2e-5


@pytest.mark.parametrize("group", [8, 1])
def test_forward_long_windows(pa, group):
    # kappa = 8 and 0.5-0.9 mm balls: windows of 210-380 samples, many
    # 32-sample steps per group
    sc = pa_inputs.small_scene(seed=9, n_balls=301, n_sensors=13, n_samples=1536, a_range=(0.5, 0.9), kappa=8.0)
    geom = geometry(sc)
    y = pa.forward(geom, dev_pad(sc.balls)[None], sc.n_balls, tiles=(8, 1536, 128, 0, group))
    pa.device_error()
    y_o, _ = _oracle_traces(sc)
    assert rel_l2(y.cpu().numpy(), y_o) <= TRACE_TOL


def _wide_radius_scene():
    # radii log-uniform over 0.03-1.5 mm: about 23 quarter-octave radius
    # classes, so the per-tile class order wraps modulo 16, and windows from
    # 8 to 400 samples; the widest are clipped at sample 0
    sc = pa_inputs.small_scene(seed=11, n_balls=3001, n_sensors=19, n_samples=1024)
    rng = np.random.default_rng(11)
    sc.balls[3] = np.exp(rng.uniform(np.log(0.03), np.log(1.5), sc.n_balls)).astype(np.float32)
    return sc


@pytest.mark.parametrize("tiles", [None, (8, 512, 100, 2, 16), (16, 1024, 512, 0, 8), (3, 256, 36, 5, 4)])
def test_forward_parity_wide_radius_range(pa, tiles):
    sc = _wide_radius_scene()
    y = pa.forward(geometry(sc), dev_pad(sc.balls)[None], sc.n_balls, tiles=tiles)
    pa.device_error()
    y_o, _ = _oracle_traces(sc)
    assert rel_l2(y.cpu().numpy(), y_o) <= TRACE_TOL


def test_adjoint_parity_wide_radius_range(pa):
    from gpu_common import GRAD_TOL
    sc = _wide_radius_scene()
    g = np.random.default_rng(12).standard_normal((1, sc.n_sensors, sc.n_samples)).astype(np.float32)
    got = pa.adjoint(geometry(sc), torch.from_numpy(g).cuda(), state=dev_pad(sc.balls)[None], n=sc.n_balls)
    pa.device_error()
    want = oracle.adjoint_state(sc.balls[None], sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g)
    got = got[..., :sc.n_balls].cpu().numpy()
    for ch in range(5):
        assert rel_l2(got[:, ch], want[:, ch]) <= GRAD_TOL, ch


def test_forward_multiframe_and_accumulate(pa):
    sc = pa_inputs.small_scene(seed=2, n_balls=517, n_sensors=9, n_samples=512, n_frames=4)
    geom = geometry(sc)
    state = dev_pad(sc.frames)
    y = pa.forward(geom, state, sc.n_balls)
    y_o, _ = _oracle_traces(sc, sc.frames)
    assert rel_l2(y.cpu().numpy(), y_o) <= TRACE_TOL
    base = torch.randn_like(y) * float(y.abs().max())
    out = base.clone()
    pa.forward(geom, state, sc.n_balls, out=out, accumulate=True, tiles=(4, 128, 64, 3))
    # out = base + y rounded once more: compare within a few ulps of |base| + |y|
    tol = 4e-7 * float((base.abs() + y.abs()).max())
    np.testing.assert_allclose((out - base).cpu().numpy(), y.cpu().numpy(), rtol=0, atol=tol)
    pa.device_error()


def test_forward_uniform_profile(pa):
    sc = pa_inputs.small_scene(seed=3, n_balls=200, n_sensors=6, n_samples=512)
    geom = geometry(sc)
    y = pa.forward(geom, dev_pad(sc.balls)[None], sc.n_balls, uniform=True)
    y_o, _ = oracle.forward(sc.balls, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa,
                            profile=oracle.PROFILE_UNIFORM)
    # the uniform pulse jumps at its window edges, where an fp32/fp64 edge
    # decision can differ by one sample; compare in L2 only
    assert rel_l2(y.cpu().numpy(), y_o) <= 1e-3
    pa.device_error()


def test_forward_deterministic(pa):
    sc = pa_inputs.small_scene(seed=4, n_balls=2000, n_sensors=16, n_samples=1024)
    geom = geometry(sc)
    st = dev_pad(sc.balls)[None]
    a = pa.forward(geom, st, sc.n_balls, tiles=(8, 512, 128, 4))
    b = pa.forward(geom, st, sc.n_balls, tiles=(8, 512, 128, 4))
    assert torch.equal(a, b)


def test_forward_edge_cases(pa):
    sc = pa_inputs.small_scene(seed=5, n_balls=64, n_sensors=3, n_samples=64, t0=0.0)
    geom = geometry(sc)
    # no balls -> zeros
    z = pa.forward(geom, torch.zeros(1, 5, 4, device="cuda"), 0)
    assert not torch.any(z)
    # inactive balls contribute nothing; one active ball, windows clipped by T
    balls = np.zeros((5, 3), dtype=np.float32)
    balls[:, 0] = [0.1, 0.2, -0.1, 0.0, 1.0]   # a = 0
    balls[:, 1] = [0.3, 0.1, 0.2, 0.2, 0.0]    # p = 0
    balls[:, 2] = [0.0, 0.0, 0.0, 0.3, 0.7]    # active
    T = 8
    R = float(np.linalg.norm(sc.sensors[:, 0]))
    t0 = (R - 0.3) / sc.c  # window straddles the first samples and T
    sc2 = pa_inputs.Scene("edge", balls, sc.sensors[:, :1].copy(), sc.c, sc.fs, t0, T, sc.kappa)
    g2 = geometry(sc2)
    y = pa.forward(g2, dev_pad(balls)[None], 3)
    y_o, cnt = oracle.forward(balls, sc2.sensors, sc2.c, sc2.fs, sc2.t0, T, sc2.kappa)
    assert cnt > 0
    assert rel_l2(y.cpu().numpy(), y_o) <= TRACE_TOL
    assert pa.count_contributions(g2, dev_pad(balls)[None], 3) == cnt
    pa.device_error()


def test_domain_error_is_reported(pa):
    balls = np.array([[0.0], [0.0], [0.0], [0.3], [1.0]], dtype=np.float32)
    sens = np.array([[0.5], [0.0], [0.0]], dtype=np.float32)  # inside kappa*a
    sc = pa_inputs.Scene("dom", balls, sens, 1.5, 40.0, 0.0, 64, 5.0)
    y = pa.forward(geometry(sc), dev_pad(balls)[None], 1)
    assert pa.device_error(raise_on_error=False) == pa._lib.PA_ERR_DOMAIN
    assert not torch.any(y)
    assert pa.device_error(raise_on_error=False) == 0  # cleared


def test_invalid_arguments_are_rejected(pa):
    sc = pa_inputs.small_scene(seed=6, n_balls=10, n_sensors=2, n_samples=64)
    geom = geometry(sc)
    st = dev_pad(sc.balls)[None]
    with pytest.raises(pa.PAError):
        pa.forward(geom, st, 10, tiles=(17, 0, 0, 0))
    with pytest.raises(pa.PAError):  # more balls per stage than any shared memory holds
        pa.forward(geom, st, 10, tiles=(16, 0, 8196, 0, 8))
    with pytest.raises(pa.PAError):  # the batched entry point checks the same bound
        pa.forward_batched([pa.Scene(geom, st, 10)], tiles=(16, 0, 8196, 0, 8))
    bad = pa.Geometry(geom.sensors, sc.c, sc.fs, sc.t0, 62, sc.kappa)  # T % 4 != 0
    with pytest.raises(pa.PAError):
        pa.forward(bad, st, 10)


def test_count_contributions_matches_oracle(pa):
    sc = pa_inputs.small_scene(seed=7, n_balls=777, n_sensors=21, n_samples=1024)
    _, cnt = _oracle_traces(sc)
    got = pa.count_contributions(geometry(sc), dev_pad(sc.balls)[None], sc.n_balls)
    # an fp32 vs fp64 decision on a sample lying on a window edge can differ
    assert abs(got - cnt) <= max(2, 1e-5 * cnt)


@pytest.mark.slow
def test_forward_full_size_single_split_accuracy(pa):
    """One ball split: each trace sample accumulates ~2,000 cancelling pulses
    of the 100k balls in one CTA; the compensated accumulation must keep the
    traces within tolerance (a plain FP32 running sum measured 1.4e-5)."""
    sc = pa_inputs.config_scene(2)
    geom = geometry(sc)
    y = pa.forward(geom, dev_pad(sc.balls)[None], sc.n_balls, tiles=(12, 2048, 512, 1, 8))
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(sc.n_sensors, 8, replace=False))
    y_o, _ = oracle.forward(sc.balls, sc.sensors[:, pick], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    assert rel_l2(y[0, pick].cpu().numpy(), y_o[0]) <= TRACE_TOL


@pytest.mark.slow
def test_forward_full_size_sampled_sensors(pa):
    """Static 100k-ball vessel tree, 576 sensors, T = 4096 in the bench's
    launch configuration; 12 random sensors checked against the oracle."""
    sc = pa_inputs.config_scene(2)
    geom = geometry(sc)
    st = dev_pad(sc.balls)[None]
    y = pa.forward(geom, st, sc.n_balls)
    pa.device_error()
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(sc.n_sensors, 12, replace=False))
    y_o, _ = oracle.forward(sc.balls, sc.sensors[:, pick], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    got = y[0, pick].cpu().numpy()
    assert rel_l2(got, y_o[0]) <= TRACE_TOL


@pytest.mark.parametrize("tiles", [None, (8, 256, 128, 3, 4), (16, 1536, 512, 0, 8), (1, 1028, 4, 7, 2)])
def test_forward_plan_and_workspace_size_are_consistent(pa, tiles):
    sc = pa_inputs.small_scene(seed=1, n_balls=1003, n_sensors=37, n_samples=1028, n_frames=3)
    geom = geometry(sc)
    state = dev_pad(sc.frames)
    F, S, T = 3, sc.n_sensors, sc.n_samples
    p = pa.forward_plan(geom, state, sc.n_balls, tiles=tiles)
    n_st, n_tt = -(-S // p["s_tile"]), -(-T // p["t_tile"])
    assert p["ctas"] == F * n_st * n_tt * p["n_splits"]
    assert p["t_tile"] % 4 == 0 and p["nb_tile"] % 4 == 0 and 1 <= p["s_tile"] <= 16
    assert p["group"] in (1, 2, 4, 8, 16)
    assert p["smem"] <= torch.cuda.get_device_properties(0).shared_memory_per_block_optin
    if tiles is not None:
        assert (p["s_tile"], p["t_tile"], p["nb_tile"]) == tuple(min(v, lim) for v, lim in zip(tiles[:3], (16, T, 1 << 30)))
    ws = pa.forward_workspace_size(geom, state, sc.n_balls, tiles=tiles)
    assert ws == (4 * p["n_splits"] * F * S * T if p["n_splits"] > 1 else 0)
    # the ssim workspace covers its partials
    assert pa._LIB.pa_ssim_workspace_size(64, 80) >= 8 * ((54 + 15) // 16) * ((70 + 15) // 16)
    assert pa._LIB.pa_ssim_workspace_size(10, 80) == 0
