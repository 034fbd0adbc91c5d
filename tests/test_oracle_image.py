"""Pins of the imaging oracles (UBP, point cloud -> voxels, MAP, SSIM) against
facts outside their own code: exact results of the finite-difference and
interpolation steps on polynomials, the exactness of universal
back-projection for a closed spherical detector surface (Xu and Wang's
theorem: the back-projection of a Gaussian ball's signals returns the ball),
the Gaussian integral, and an independent SSIM built from scipy's Gaussian
filter."""
import math

import numpy as np
import pytest

import oracle
import pa_inputs


def test_ubp_filter_exact_on_quadratics():
    # b = 2p - 2t dp/dt; central differences are exact on quadratics and the
    # one-sided end differences on linear functions
    fs, t0, T = 40.0, 3.0, 64
    t = t0 + np.arange(T) / fs
    al, be, ga = 0.7, -1.3, 0.25
    p = al + be * t + ga * t * t
    b = oracle.ubp_filter(p[None], fs, t0)[0]
    want = 2 * al - 2 * ga * t * t
    np.testing.assert_allclose(b[1:-1], want[1:-1], rtol=0, atol=1e-12)
    lin = al + be * t
    bl = oracle.ubp_filter(lin[None], fs, t0)[0]
    np.testing.assert_allclose(bl, 2 * al + 0 * t, rtol=0, atol=1e-12)


def test_ubp_filter_matches_analytic_derivative_of_the_radiator():
    # a finely sampled single-ball trace: b against 2P - 2t dP/dt with the
    # analytic derivative of the outgoing Gaussian pulse
    p, a, R, c, fs, t0 = 0.8, 0.3, 20.0, 1.5, 2000.0, 12.0
    T = 8192
    t = t0 + np.arange(T) / fs
    tau = R - c * t
    E = np.exp(-tau ** 2 / (2 * a * a))
    P = p / (2 * R) * tau * E
    dP = p / (2 * R) * (-c) * E * (1 - tau ** 2 / (a * a))
    b = oracle.ubp_filter(P[None], fs, t0)[0]
    want = 2 * P - 2 * t * dP
    err = np.linalg.norm(b[1:-1] - want[1:-1]) / np.linalg.norm(want)
    assert err < 1e-5


def test_ubp_interpolation_and_geometry_exact_for_linear_traces():
    # one sensor facing the centre, b linear in the sample index: the voxel
    # value is alpha + beta (d/c - t0) fs exactly
    sens = np.array([[0.0], [0.0], [-30.0]])
    center = np.zeros(3)
    c, fs, t0, T = 1.5, 40.0, 1.0, 4096
    al, be = 0.3, 0.01
    b = (al + be * np.arange(T))[None]
    origin = np.array([-0.7, -0.4, -1.0])
    h, shape = 0.35, (4, 3, 5)
    vol = oracle.ubp(b, sens, center, c, fs, t0, origin, h, shape)
    nz, ny, nx = shape
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.stack([origin[0] + h * ix, origin[1] + h * iy, origin[2] + h * iz])
    d = np.sqrt(((r - sens[:, 0, None, None, None]) ** 2).sum(0))
    np.testing.assert_allclose(vol, al + be * (d / c - t0) * fs, rtol=1e-12, atol=1e-12)


def test_ubp_mirror_sensors_weight_by_inverse_square_distance():
    # two sensors on the x axis facing each other: on the axis cos = 1, so the
    # value is the 1/d^2-weighted mean of their (constant) traces
    L = 25.0
    sens = np.array([[-L, L], [0.0, 0.0], [0.0, 0.0]])
    b = np.stack([np.full(4096, 2.0), np.full(4096, -1.0)])
    vol = oracle.ubp(b, sens, np.zeros(3), 1.5, 40.0, 0.0, np.array([-3.0, 0.0, 0.0]), 3.0, (1, 1, 3))[0, 0]
    xs = np.array([-3.0, 0.0, 3.0])
    w1, w2 = 1 / (xs + L) ** 2, 1 / (L - xs) ** 2
    np.testing.assert_allclose(vol, (2.0 * w1 - 1.0 * w2) / (w1 + w2), rtol=1e-12)


def test_ubp_constant_traces_give_the_constant():
    sens = pa_inputs.fibonacci_sphere(64, 30.0)
    b = np.full((64, 4096), 0.37)
    vol = oracle.ubp(b, sens, np.zeros(3), 1.5, 40.0, 0.0, np.array([-2.0, -2.0, -2.0]), 1.0, (5, 5, 5))
    np.testing.assert_allclose(vol, 0.37, rtol=1e-12)


def test_ubp_reconstructs_a_gaussian_ball_inside_a_closed_sphere():
    # Xu-Wang exactness: UBP from a closed spherical surface returns the
    # initial pressure; with 3000 point sensors and fine sampling the
    # discretisation error is a few 1e-3
    p, a = 1.0, 0.5
    n_s, Rs = 3000, 15.0
    sens = pa_inputs.fibonacci_sphere(n_s, Rs)
    c, fs, t0, T = 1.5, 400.0, 0.0, 6000
    ball = np.array([[0.2], [-0.1], [0.15], [a], [p]])
    y, _ = oracle.forward(ball[None], sens, c, fs, t0, T, 5.0)
    b = oracle.ubp_filter(y[0], fs, t0)
    h = 0.25
    origin = np.array([0.2 - 2 * a, -0.1, 0.15])
    xs = origin[0] + h * np.arange(9)
    vol = oracle.ubp(b, sens, np.zeros(3), c, fs, t0, origin, h, (1, 1, 9))[0, 0]
    want = p * np.exp(-(xs - 0.2) ** 2 / (2 * a * a))
    assert abs(vol[4] - p) < 0.02 * p
    np.testing.assert_allclose(vol, want, rtol=0, atol=0.03 * p)


def test_splat_gaussian_integral_and_centre_value():
    p, a, kappa = 1.7, 0.6, 5.0
    h = a / 4
    n = int(2 * kappa * a / h) + 3
    origin = np.full(3, -h * (n // 2))
    ball = np.array([[0.0], [0.0], [0.0], [a], [p]])
    vol = oracle.splat(ball, kappa, origin, h, (n, n, n))
    assert vol[n // 2, n // 2, n // 2] == pytest.approx(p, rel=1e-15)
    tail = math.erfc(kappa / math.sqrt(2)) + math.sqrt(2 / math.pi) * kappa * math.exp(-kappa ** 2 / 2)
    want = p * (2 * math.pi) ** 1.5 * a ** 3 * (1 - tail)
    # a Riemann sum of a Gaussian at h = a/4 is accurate to ~1e-30; the
    # truncated sphere's voxelised boundary leaves ~1e-6
    assert vol.sum() * h ** 3 == pytest.approx(want, rel=1e-5)


def test_splat_truncation_edge_and_superposition():
    a, kappa = 0.5, 3.0
    h = 0.1
    edge = kappa * a
    ball = np.array([[0.0], [0.0], [0.0], [a], [1.0]])
    # voxels at x = edge - h/2 ... on a line through the centre
    origin = np.array([edge - 0.05, 0.0, 0.0])
    vol = oracle.splat(ball, kappa, origin, h, (1, 1, 2))[0, 0]
    assert vol[0] == pytest.approx(math.exp(-(edge - 0.05) ** 2 / (2 * a * a)), rel=1e-14)
    assert vol[1] == 0.0
    two = np.concatenate([ball, np.array([[0.3], [0.1], [0.0], [0.4], [-2.0]])], axis=1)
    o = np.array([-0.5, -0.5, -0.5])
    v2 = oracle.splat(two, kappa, o, 0.25, (5, 5, 5))
    v0 = oracle.splat(two[:, :1], kappa, o, 0.25, (5, 5, 5))
    v1 = oracle.splat(two[:, 1:], kappa, o, 0.25, (5, 5, 5))
    np.testing.assert_allclose(v2, v0 + v1, rtol=1e-14, atol=1e-15)


def test_maps_are_axis_maxima():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((4, 5, 6))
    xy, yz, xz = oracle.maps(v)
    assert xy.shape == (5, 6) and yz.shape == (4, 5) and xz.shape == (4, 6)
    for iy in range(5):
        for ix in range(6):
            assert xy[iy, ix] == max(v[iz, iy, ix] for iz in range(4))


def test_ssim_identity_constant_and_symmetry():
    rng = np.random.default_rng(6)
    x = rng.random((24, 31))
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1)
    assert oracle.ssim(x, x) == pytest.approx(1.0, abs=1e-14)
    assert oracle.ssim(x, y) == pytest.approx(oracle.ssim(y, x), abs=1e-14)
    assert oracle.ssim(x, y) < 1.0
    c1, c2 = 0.3, 0.8
    C1 = 0.01 ** 2
    cst = oracle.ssim(np.full((12, 12), c1), np.full((12, 12), c2))
    assert cst == pytest.approx((2 * c1 * c2 + C1) / (c1 * c1 + c2 * c2 + C1), rel=1e-12)


def test_ssim_matches_an_independent_separable_gaussian_filter():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(7)
    x = rng.random((40, 37))
    y = 0.6 * x + 0.4 * rng.random(x.shape)
    L = 1.0

    def filt(z):  # 11-tap Gaussian, sigma 1.5 (radius 5), then the positions where the window fits
        return ndimage.gaussian_filter(z, 1.5, truncate=5 / 1.5, mode="constant")[5:-5, 5:-5]

    mx, my = filt(x), filt(y)
    sx, sy, sxy = filt(x * x) - mx * mx, filt(y * y) - my * my, filt(x * y) - mx * my
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    m = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2))
    got, gmap = oracle.ssim(x, y, L, want_map=True)
    np.testing.assert_allclose(gmap, m, rtol=0, atol=1e-12)
    assert got == pytest.approx(m.mean(), abs=1e-12)


def test_ssim_minmax_is_invariant_to_affine_intensity_changes():
    rng = np.random.default_rng(8)
    x = rng.random((30, 30))
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1)
    base = oracle.ssim(oracle.minmax01(x), oracle.minmax01(y), 1.0)
    assert oracle.ssim(5.0 * x - 2.0, 0.01 * y + 7.0, minmax=True) == pytest.approx(base, abs=1e-12)
