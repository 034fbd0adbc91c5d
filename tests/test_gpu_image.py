"""Imaging kernels (UBP, ball cloud -> voxels, MAP, SSIM) against the FP64
oracle, through the C ABI.

Tolerances (derived from the FP32 arithmetic of each kernel):
  - UBP filter: elementwise FP32, rel-L2 <= 1e-6;
  - UBP back-projection: rel-L2 <= 1e-4 over the volume.  The fractional
    sample index d fs/c of a ~60 mm path is formed in FP32 (and d from an
    approximate reciprocal square root), ~4e-4 samples of error; against a
    pulse ~3-10 samples wide that is <= 1e-4 relative per term;
  - splat: rel-L2 <= 1e-5 (FP32 exponent argument and ex2, ~1e-6);
  - MAP: bit-exact (max of the same FP32 volume);
  - SSIM: mean within 1e-5, map within 1e-4 (FP32 local variances)."""
import numpy as np
import pytest
import torch

import oracle
import pa_inputs
from gpu_common import dev_pad, rel_l2

pytestmark = pytest.mark.gpu

UBP_TOL = 1e-4
SPLAT_TOL = 1e-5


@pytest.fixture(scope="module")
def pa():
    import paper_2412_03898_gb300 as m
    return m


def test_ubp_filter_parity(pa):
    rng = np.random.default_rng(61)
    p = rng.standard_normal((3, 17, 1028)).astype(np.float32)
    got = pa.ubp_filter(torch.from_numpy(p).cuda(), 40.0, 2.5).cpu().numpy()
    want = oracle.ubp_filter(p, 40.0, 2.5)
    assert rel_l2(got, want) <= 1e-6


@pytest.mark.parametrize("n_sensors", [96, 1100])  # 1100 > one 1024-sensor shared-memory chunk
def test_ubp_parity(pa, n_sensors):
    rng = np.random.default_rng(62)
    sens = pa_inputs.fibonacci_sphere(n_sensors, 20.0)
    c, fs, t0, T = 1.5, 40.0, 0.0, 1536
    balls = np.stack([rng.uniform(-3, 3, 40), rng.uniform(-3, 3, 40), rng.uniform(-3, 3, 40),
                      rng.uniform(0.15, 0.4, 40), rng.uniform(0.2, 1.0, 40)]).astype(np.float32)
    y, _ = oracle.forward(balls[None], sens, c, fs, t0, T, 5.0)
    b = oracle.ubp_filter(y[0], fs, t0).astype(np.float32)
    geom = pa.Geometry(torch.from_numpy(sens).cuda(), c, fs, t0, T, 5.0)
    grid = pa.Grid((-3.3, -3.1, -2.9), 0.3, (19, 21, 23))  # ragged against the 8 x 8 x 4 bricks
    got = pa.ubp(geom, torch.from_numpy(b).cuda(), grid).cpu().numpy()
    want = oracle.ubp(b, sens, np.zeros(3), c, fs, t0, np.array(grid.origin), grid.h, grid.shape)
    assert rel_l2(got, want) <= UBP_TOL


def test_ubp_off_centre_array_and_out_of_range_samples(pa):
    # hemisphere array with a shifted centre; part of the grid lies beyond the
    # last sample (those terms are 0) and behind some sensors (left out)
    rng = np.random.default_rng(63)
    sens = (pa_inputs.fibonacci_hemisphere(200, 15.0) + np.array([[1.0], [-0.5], [2.0]], dtype=np.float32))
    c, fs, t0, T = 1.5, 40.0, 3.0, 512
    b = rng.standard_normal((200, T)).astype(np.float32)
    geom = pa.Geometry(torch.from_numpy(sens).cuda(), c, fs, t0, T, 5.0)
    grid = pa.Grid((-12.0, -12.0, -4.0), 1.1, (13, 22, 22))
    center = (1.0, -0.5, 2.0)
    got = pa.ubp(geom, torch.from_numpy(b).cuda(), grid, center=center).cpu().numpy()
    want = oracle.ubp(b, sens, np.array(center), c, fs, t0, np.array(grid.origin), grid.h, grid.shape)
    assert rel_l2(got, want) <= UBP_TOL


def test_splat_parity(pa):
    rng = np.random.default_rng(64)
    n = 300
    balls = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(-2, 2, n),
                      rng.uniform(0.1, 0.4, n), rng.uniform(-0.5, 1.0, n)]).astype(np.float32)
    balls[3, 7] = 0.0  # inactive ball
    balls[4, 9] = 0.0
    grid = pa.Grid((-2.5, -2.4, -2.3), 0.13, (33, 35, 37))  # ragged against the 16^3 bricks
    got = pa.splat(dev_pad(balls), grid, 5.0, n).cpu().numpy()
    want = oracle.splat(balls, 5.0, np.array(grid.origin), grid.h, grid.shape)
    assert rel_l2(got, want) <= SPLAT_TOL


def test_splat_dense_brick_drains_its_list(pa):
    # 3000 balls inside one 16^3 brick: the per-CTA list is drained several times
    rng = np.random.default_rng(65)
    n = 3000
    balls = np.stack([rng.uniform(0, 1.5, n), rng.uniform(0, 1.5, n), rng.uniform(0, 1.5, n),
                      rng.uniform(0.05, 0.15, n), rng.uniform(0.2, 1.0, n)]).astype(np.float32)
    grid = pa.Grid((0.0, 0.0, 0.0), 0.1, (16, 16, 16))
    got = pa.splat(dev_pad(balls), grid, 3.0, n).cpu().numpy()
    want = oracle.splat(balls, 3.0, np.array(grid.origin), grid.h, grid.shape)
    assert rel_l2(got, want) <= SPLAT_TOL
    again = pa.splat(dev_pad(balls), grid, 3.0, n).cpu().numpy()
    assert np.array_equal(got, again)  # deterministic


def test_maps_bit_exact(pa):
    rng = np.random.default_rng(66)
    v = rng.standard_normal((9, 70, 45)).astype(np.float32)
    grid = pa.Grid((0, 0, 0), 1.0, v.shape)
    xy, yz, xz = pa.maps(torch.from_numpy(v).cuda(), grid)
    w = oracle.maps(v)
    for got, want in zip((xy, yz, xz), w):
        assert np.array_equal(got.cpu().numpy(), want.astype(np.float32))


def test_ssim_parity(pa):
    rng = np.random.default_rng(67)
    x = rng.random((45, 67)).astype(np.float32)
    y = np.clip(0.7 * x + 0.3 * rng.random(x.shape) ** 2, 0, 1).astype(np.float32)
    mean, m = pa.ssim(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 1.0, want_map=True)
    want, wmap = oracle.ssim(x, y, 1.0, want_map=True)
    assert abs(float(mean) - want) <= 1e-5
    assert np.abs(m.cpu().numpy() - wmap).max() <= 1e-4
    same = pa.ssim(torch.from_numpy(x).cuda(), torch.from_numpy(x).cuda())
    assert abs(float(same) - 1.0) <= 1e-5


def test_ssim_minmax_parity(pa):
    # reconstructions in arbitrary units against a [0, 1] ground truth
    rng = np.random.default_rng(68)
    x = (3.0 * rng.random((64, 40)) - 1.0).astype(np.float32)
    y = np.clip(x + 0.2 * rng.standard_normal(x.shape), -1, 2).astype(np.float32)
    mean, m = pa.ssim(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), want_map=True, minmax=True)
    want, wmap = oracle.ssim(x, y, want_map=True, minmax=True)
    assert abs(float(mean) - want) <= 1e-5
    assert np.abs(m.cpu().numpy() - wmap).max() <= 1e-4
    flat = pa.ssim(torch.full((20, 20), 3.0, device="cuda"), torch.full((20, 20), 3.0, device="cuda"), minmax=True)
    assert abs(float(flat) - 1.0) <= 1e-6  # both constant -> both 0 -> identical


def test_imaging_rejects_bad_arguments(pa):
    g = pa.Grid((0, 0, 0), 1.0, (4, 4, 4))
    v = torch.zeros(4, 4, 4, device="cuda")
    with pytest.raises(pa.PAError):
        pa.maps(v, pa.Grid((0, 0, 0), 0.0, (4, 4, 4)))
    with pytest.raises(pa.PAError):
        pa.ssim(torch.zeros(10, 10, device="cuda"), torch.zeros(10, 10, device="cuda"))
    with pytest.raises(pa.PAError):
        pa.splat(torch.zeros(5, 4, device="cuda"), g, kappa=0.0)


def test_imaging_edge_cases(pa):
    # empty ball cloud -> zero volume (the output is overwritten)
    grid = pa.Grid((0.0, 0.0, 0.0), 0.5, (3, 5, 7))
    vol = torch.full(grid.shape, 9.0, device="cuda")
    pa.splat(torch.zeros(5, 4, device="cuda"), grid, 5.0, 0, out=vol)
    assert not torch.any(vol)
    # one sensor; a grid whose samples all fall past the last one -> zeros
    sens = np.array([[0.0], [0.0], [-20.0]], dtype=np.float32)
    b = np.random.default_rng(69).standard_normal((1, 64)).astype(np.float32)
    geom = pa.Geometry(torch.from_numpy(sens).cuda(), 1.5, 40.0, 0.0, 64, 5.0)
    near = pa.Grid((0.0, 0.0, -19.5), 0.1, (2, 2, 2))   # d ~ 0.5 mm -> samples ~13
    far = pa.Grid((0.0, 0.0, 10.0), 0.1, (2, 2, 2))     # d ~ 30 mm -> samples ~800 > 63
    bt = torch.from_numpy(b).cuda()
    got = pa.ubp(geom, bt, near).cpu().numpy()
    want = oracle.ubp(b, sens, np.zeros(3), 1.5, 40.0, 0.0, np.array(near.origin), near.h, near.shape)
    assert rel_l2(got, want) <= UBP_TOL
    assert not torch.any(pa.ubp(geom, bt, far))
    # 1 x 1 x 1 MAPs and an SSIM with a single window position
    one = torch.tensor([[[2.5]]], device="cuda")
    for m in pa.maps(one, pa.Grid((0, 0, 0), 1.0, (1, 1, 1))):
        assert float(m) == 2.5
    rng = np.random.default_rng(70)
    x, y = rng.random((11, 11)).astype(np.float32), rng.random((11, 11)).astype(np.float32)
    got = float(pa.ssim(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()))
    assert abs(got - oracle.ssim(x, y)) <= 1e-5


@pytest.mark.slow
def test_full_size_heart_sampled_lines(pa):
    """The bench's imaging workload (simulated heart frame 0, 1,024 sensors,
    UBP and splat onto 256^3 voxels of 0.2 mm), checked on three sampled voxel
    lines along x that the oracle computes one by one."""
    sc = pa_inputs.heart_phantom()
    n = sc.n_balls
    st = dev_pad(sc.frames[0])
    geom = pa.Geometry(torch.from_numpy(sc.sensors).cuda(), sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    y = pa.forward(geom, st[None], n)[0].contiguous()
    b = pa.ubp_filter(y, sc.fs, sc.t0)
    grid = pa.Grid.cube(25.6, 256)
    vol = pa.ubp(geom, b, grid).cpu().numpy()
    gt = pa.splat(st, grid, sc.kappa, n).cpu().numpy()
    pa.device_error()
    b_h = b.cpu().numpy()
    for iz, iy in ((128, 128), (120, 140), (131, 97)):
        origin = np.array([grid.origin[0], grid.origin[1] + grid.h * iy, grid.origin[2] + grid.h * iz])
        line_u = oracle.ubp(b_h, sc.sensors, np.zeros(3), sc.c, sc.fs, sc.t0, origin, grid.h, (1, 1, 256))[0, 0]
        assert rel_l2(vol[iz, iy], line_u) <= UBP_TOL, (iz, iy)
        line_s = oracle.splat(sc.frames[0], sc.kappa, origin, grid.h, (1, 1, 256))[0, 0]
        assert rel_l2(gt[iz, iy], line_s) <= SPLAT_TOL, (iz, iy)
