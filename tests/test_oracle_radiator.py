"""Pins of the oracle's radiator (forward projection) to facts that do not
come from the oracle itself: the 3D wave equation, its initial condition,
a brute-force spherical-mean quadrature of the initial pressure, the textbook
uniform-ball N-pulse, symmetries and invariances.

The paper names the radiator (Sec. 2.2, last paragraph: SlingBAG's
differentiable rapid radiator) but does not print it; the reading used is the
exact Poisson solution for a Gaussian initial pressure of peak p0 and standard
deviation a0 (Sec. 2.1).
"""
import math

import numpy as np
import pytest

import oracle
from bruteforce import smoothed_pressure, smoothed_target

C = 1.5


def _d4(f, x, h):
    """4th-order central first derivative."""
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


def _dd4(f, x, h):
    """4th-order central second derivative."""
    return (-f(x + 2 * h) + 16 * f(x + h) - 30 * f(x) + 16 * f(x - h) - f(x - 2 * h)) / (12 * h * h)


# ---------------------------------------------------------------------------
# The full closed form (both terms) solves the Cauchy problem of the wave
# equation with p(., 0) = Gaussian and dp/dt(., 0) = 0; by uniqueness that
# fixes it completely.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("R_over_a", [0.3, 1.0, 2.5, 6.0])
def test_full_solution_initial_value(R_over_a):
    p, a = 0.7, 0.25
    R = R_over_a * a
    got = oracle.pressure_full(p, a, R, 0.0)
    want = p * math.exp(-R * R / (2 * a * a))
    assert got == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("R_over_a", [0.5, 2.0, 5.0])
def test_full_solution_zero_initial_velocity(R_over_a):
    p, a = 1.3, 0.2
    R = R_over_a * a
    h = 1e-3 * a
    dpdt = _d4(lambda ct: oracle.pressure_full(p, a, R, ct), 0.0, h)
    assert abs(dpdt) <= 1e-9 * p / a


def test_full_solution_wave_equation():
    """d2P/d(ct)2 = d2P/dR2 + (2/R) dP/dR for the radially symmetric field."""
    rng = np.random.default_rng(7)
    p, a = 0.9, 0.3
    for _ in range(25):
        R = a * rng.uniform(1.5, 20.0)
        ct = R + a * rng.uniform(-3.0, 3.0)
        h = 2e-3 * a
        ptt = _dd4(lambda s: oracle.pressure_full(p, a, R, s), ct, h)
        prr = _dd4(lambda r: oracle.pressure_full(p, a, r, ct), R, h)
        pr = _d4(lambda r: oracle.pressure_full(p, a, r, ct), R, h)
        scale = p / (2 * R) / a  # magnitude of the second derivatives
        assert abs(ptt - prr - 2.0 / R * pr) <= 1e-6 * scale


def test_forward_equals_outgoing_term_of_full_solution():
    """The forward projection samples the full solution (the mirror term is
    below double precision at R/a > 40)."""
    balls = np.array([[0.3], [-0.2], [0.1], [0.25], [0.8]])
    sens = np.array([[40.0], [0.0], [0.0]])
    fs, t0, T, kappa = 40.0, 20.0, 1024, 5.0
    y, n = oracle.forward(balls, sens, C, fs, t0, T, kappa)
    R = math.dist(balls[:3, 0], sens[:, 0])
    ks = np.nonzero(y[0, 0])[0]
    assert n == len(ks) > 10
    for k in ks:
        ct = C * (t0 + k / fs)
        assert y[0, 0, k] == pytest.approx(oracle.pressure_full(0.8, 0.25, R, ct), rel=1e-13, abs=1e-16)


def test_forward_wave_equation_on_sensor_stencil():
    """Traces at a 13-point sensor stencil satisfy y_tt = c^2 lap(y) inside the
    window, which pins the 1/R spreading and the travelling-wave form."""
    a, p = 0.2, 1.0
    hx = a / 25.0
    fs = C / hx  # time step matches the space step
    r0 = np.array([30.0, 10.0, -20.0])
    R0 = float(np.linalg.norm(r0))
    offs = [(0, 0, 0)]
    for ax in range(3):
        for m in (-2, -1, 1, 2):
            o = [0, 0, 0]
            o[ax] = m
            offs.append(tuple(o))
    sens = np.array([r0 + hx * np.array(o) for o in offs]).T
    balls = np.array([[0.0], [0.0], [0.0], [a], [p]])
    t0 = (R0 - 6 * a) / C
    T = int(12 * a / hx) + 40
    y, _ = oracle.forward(balls, sens, C, fs, t0, T, 8.0)
    y = y[0]
    idx = {o: i for i, o in enumerate(offs)}
    c0 = y[idx[(0, 0, 0)]]
    lap = np.zeros(T)
    for ax in range(3):
        def at(m):
            o = [0, 0, 0]
            o[ax] = m
            return y[idx[tuple(o)]]
        lap += (-at(2) + 16 * at(1) - 30 * c0 + 16 * at(-1) - at(-2)) / (12 * hx * hx)
    k = np.arange(2, T - 2)
    ytt = (-c0[k + 2] + 16 * c0[k + 1] - 30 * c0[k] + 16 * c0[k - 1] - c0[k - 2]) / (12 * (1 / fs) ** 2)
    tau = R0 - C * (t0 + k / fs)
    inside = np.abs(tau) < 4.5 * a
    scale = np.max(np.abs(ytt[inside]))
    resid = ytt[inside] - C * C * lap[k][inside]
    assert np.max(np.abs(resid)) <= 1e-4 * scale


@pytest.mark.slow
def test_forward_matches_bruteforce_spherical_means():
    """Voxelised initial pressure + numerical spherical means (no closed form)
    agree with the oracle's traces smoothed by the same kernel."""
    a, p = 0.2, 0.9
    ball = np.array([1.0, -0.5, 0.7, a, p])
    for sensor in (np.array([38.0, 5.0, -3.0]), np.array([-10.0, 20.0, -30.0])):
        R = float(np.linalg.norm(sensor - ball[:3]))
        w = a / 4.0
        delta = w / 6.0
        fs = C / delta
        t0 = (R - 10 * a) / C
        T = int(20 * a / delta)
        y, _ = oracle.forward(ball[:, None], sensor[:, None], C, fs, t0, T, 8.0)
        y = y[0, 0]
        k = np.arange(T)
        tau = R - C * (t0 + k / fs)
        sel = k[np.abs(tau) <= 4.0 * a][::4]
        s_vals = C * (t0 + sel / fs)
        smooth = smoothed_target(y, delta, w, sel, s_vals)
        bf = smoothed_pressure(ball, sensor, s_vals, w, a / 8.0)
        err = np.linalg.norm(bf - smooth) / np.linalg.norm(smooth)
        assert err < 1e-9, err


@pytest.mark.slow
def test_uniform_ball_bruteforce_matches_textbook_n_pulse():
    """Validates the brute-force tool itself on the textbook uniform ball:
    p(R - ct)/(2R) on |R - ct| <= a, smoothed analytically by a Gaussian."""
    from scipy.special import ndtr
    a, p = 0.3, 1.0
    ball = np.array([0.0, 0.0, 0.0, a, p])
    sensor = np.array([0.0, 25.0, -20.0])
    R = float(np.linalg.norm(sensor))
    w = a / 4
    s_vals = R + np.linspace(-1.6 * a, 1.6 * a, 41)
    bf = smoothed_pressure(ball, sensor, s_vals, w, a / 24.0, profile="uniform", sub=3)
    gw = lambda u: np.exp(-u * u / (2 * w * w)) / (math.sqrt(2 * math.pi) * w)
    def npulse_smoothed(s):
        tau = R - s
        return p / (2 * R) * (tau * (ndtr((tau + a) / w) - ndtr((tau - a) / w))
                              + w * w * (gw(tau + a) - gw(tau - a)))
    ds = 1e-4 * a
    d_ds = (npulse_smoothed(s_vals + ds) - npulse_smoothed(s_vals - ds)) / (2 * ds)
    want = npulse_smoothed(s_vals) * (1 - w * w / s_vals ** 2) + (w * w / s_vals) * d_ds
    err = np.linalg.norm(bf - want) / np.linalg.norm(want)
    assert err < 2e-3, err


def test_uniform_profile_is_n_pulse():
    a, p = 0.3, 0.6
    balls = np.array([[0.0], [0.0], [0.0], [a], [p]])
    sens = np.array([[0.0], [30.0], [-10.0]])
    R = math.sqrt(1000.0)
    fs, t0, T = 40.0, 18.0, 512
    y, n = oracle.forward(balls, sens, C, fs, t0, T, 5.0, profile=oracle.PROFILE_UNIFORM)
    k = np.arange(T)
    tau = R - C * (t0 + k / fs)
    inside = np.abs(tau) <= a
    assert n == inside.sum()
    np.testing.assert_allclose(y[0, 0][inside], p * tau[inside] / (2 * R), rtol=1e-13)
    assert np.all(y[0, 0][~inside] == 0.0)


# ---------------------------------------------------------------------------
# Symmetries, special values, invariances
# ---------------------------------------------------------------------------

def test_antisymmetry_about_arrival_time():
    """With R/c on a sample, y(R/c + j/fs) = -y(R/c - j/fs) and y(R/c) = 0."""
    a, p = 0.22, 0.5
    balls = np.array([[0.0], [0.0], [0.0], [a], [p]])
    sens = np.array([[37.5], [0.0], [0.0]])  # R/c = 25 us = sample 1000 at fs=40, t0=0
    y, _ = oracle.forward(balls, sens, C, 40.0, 0.0, 2048, 5.0)
    y = y[0, 0]
    k0 = 1000
    assert abs(y[k0]) <= 1e-15
    j = np.arange(1, 40)
    scale = np.max(np.abs(y))
    np.testing.assert_allclose(y[k0 + j], -y[k0 - j], rtol=0, atol=1e-13 * scale)
    assert np.max(np.abs(y[k0 + j])) > 0.1 * scale


def test_peak_value_at_tau_equal_a():
    """At tau = a the pulse equals p a e^{-1/2} / (2R) (its extremum)."""
    a, p = 0.375, 0.8  # a is a whole number of samples (c/fs = 0.0375)
    balls = np.array([[0.0], [0.0], [0.0], [a], [p]])
    sens = np.array([[0.0], [0.0], [-37.5]])
    y, _ = oracle.forward(balls, sens, C, 40.0, 0.0, 2048, 5.0)
    k = 1000 - 10  # tau = +a
    R = 37.5
    assert y[0, 0, k] == pytest.approx(p * a * math.exp(-0.5) / (2 * R), rel=1e-13)
    assert np.argmax(y[0, 0]) == k


def test_energy_integral():
    """sum_k y^2 / fs -> p^2 a^3 sqrt(pi) / (8 R^2 c) (the integral of the
    squared pulse over time; sampling error is exponentially small)."""
    a, p = 0.25, 0.7
    balls = np.array([[0.5], [0.2], [-0.3], [a], [p]])
    sens = np.array([[20.0], [-30.0], [-25.0]])
    R = math.dist(balls[:3, 0], sens[:, 0])
    fs = 40.0
    y, _ = oracle.forward(balls, sens, C, fs, 0.0, 4096, 8.0)
    energy = np.sum(y[0, 0] ** 2) / fs
    want = p * p * a ** 3 * math.sqrt(math.pi) / (8 * R * R * C)
    assert energy == pytest.approx(want, rel=1e-10)


def test_window_is_exactly_the_closed_support():
    """Brute force over all samples: a ball contributes at k iff
    |R - c t_k| <= kappa a and 0 <= k < T (the count of contributions too)."""
    rng = np.random.default_rng(3)
    n, ns, T = 40, 6, 700
    balls = np.stack([rng.uniform(-4, 4, n), rng.uniform(-4, 4, n), rng.uniform(-4, 4, n),
                      rng.uniform(0.1, 0.3, n), rng.uniform(0.2, 1.0, n)])
    sens = np.array([[40.0 * math.cos(q), 40.0 * math.sin(q), -5.0] for q in rng.uniform(0, 6.28, ns)]).T
    fs, t0, kappa = 40.0, 12.0, 5.0
    _, count = oracle.forward(balls, sens, C, fs, t0, T, kappa)
    k = np.arange(T)
    want = 0
    for s in range(ns):
        for b in range(n):
            R = math.dist(balls[:3, b], sens[:, s])
            want += int(np.sum(np.abs(R - C * (t0 + k / fs)) <= kappa * balls[3, b]))
    assert count == want


def test_linearity_in_pressure_and_superposition():
    rng = np.random.default_rng(11)
    n = 12
    balls = np.stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-3, 3, n),
                      rng.uniform(0.1, 0.3, n), rng.uniform(0.2, 1.0, n)])
    sens = np.array([[40.0, 0.0, 0.0], [0.0, -35.0, -15.0], [10.0, 10.0, -37.0]]).T
    args = (C, 40.0, 15.0, 1024, 5.0)
    y, _ = oracle.forward(balls, sens, *args)
    b2 = balls.copy()
    b2[4] *= 2.0
    y2, _ = oracle.forward(b2, sens, *args)
    np.testing.assert_array_equal(y2, 2.0 * y)  # scaling by 2 is exact
    parts = sum(oracle.forward(balls[:, i:i + 1], sens, *args)[0] for i in range(n))
    np.testing.assert_allclose(parts, y, rtol=0, atol=1e-14 * np.max(np.abs(y)))


def test_joint_rigid_motion_invariance():
    rng = np.random.default_rng(5)
    n = 20
    balls = np.stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-3, 3, n),
                      rng.uniform(0.1, 0.3, n), rng.uniform(0.2, 1.0, n)])
    sens = np.array([[40.0, 0.0, 0.0], [0.0, -35.0, -15.0], [10.0, 10.0, -37.0], [-20, 30, -10]]).T
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    shift = rng.uniform(-5, 5, 3)
    rb = balls.copy()
    rb[:3] = q @ balls[:3] + shift[:, None]
    rs = q @ sens + shift[:, None]
    args = (C, 40.0, 15.0, 1024, 8.0)
    y, _ = oracle.forward(balls, sens, *args)
    yr, _ = oracle.forward(rb, rs, *args)
    np.testing.assert_allclose(yr, y, rtol=0, atol=1e-10 * np.max(np.abs(y)))


def test_zero_size_or_pressure_contributes_nothing_and_domain_error():
    balls = np.array([[0.0, 1.0, 2.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0],
                      [0.0, 0.2, -0.1], [1.0, 0.0, 1.0]])
    sens = np.array([[40.0], [0.0], [0.0]])
    y, n = oracle.forward(balls, sens, C, 40.0, 20.0, 1024, 5.0)
    assert n == 0 and not np.any(y)
    inside = np.array([[0.0], [0.0], [0.0], [0.3], [1.0]])
    with pytest.raises(oracle.OracleError):
        oracle.forward(inside, np.array([[1.0], [0.0], [0.0]]), C, 40.0, 0.0, 256, 5.0)
