"""Pins of the oracle's deformation (Eq. 1-2) to special cases with known
values: neutral weights, a single basis at and around its centre, linearity
in the weights, channel independence and the multiplicative form of Eq. 1."""
import math

import numpy as np
import pytest

import oracle
import pa_inputs


def _canon(rng, n):
    return np.stack([rng.uniform(-5, 5, n), rng.uniform(-5, 5, n), rng.uniform(-5, 5, n),
                     rng.uniform(0.1, 0.4, n), rng.uniform(0.2, 1.0, n)])


def test_zero_weights_reproduce_the_static_cloud():
    """omega = 0: every frame is the canonical cloud (single-frame SlingBAG)."""
    rng = np.random.default_rng(0)
    canon = _canon(rng, 17)
    om, th, sg = pa_inputs.deform_init(17, 65)
    out = oracle.deform(canon, om, th, sg, pa_inputs.frame_times(9))
    for f in range(9):
        np.testing.assert_array_equal(out[f], canon)


def test_single_basis_values():
    """Nb = 1: H(theta) = omega, H(theta +- sigma) = omega e^{-1/2},
    H(theta +- 2 sigma) = omega e^{-2}."""
    canon = np.array([[2.0], [-1.0], [0.5], [0.3], [0.7]])
    omega = np.array([0.3, -0.2, 0.1, 0.25, -0.4]).reshape(5, 1, 1)
    theta = np.full((5, 1, 1), 0.4)
    sigma = np.full((5, 1, 1), 0.125)
    t = np.array([0.4, 0.4 + 0.125, 0.4 - 0.125, 0.4 + 0.25, 0.4 - 0.25])
    out = oracle.deform(canon, omega, theta, sigma, t)
    for f, fac in enumerate([1.0, math.exp(-0.5), math.exp(-0.5), math.exp(-2.0), math.exp(-2.0)]):
        for ch in range(5):
            want = canon[ch, 0] * (1 + omega[ch, 0, 0] * fac)
            assert out[f, ch, 0] == pytest.approx(want, rel=1e-15)


def test_linear_in_weights_and_channels_independent():
    rng = np.random.default_rng(1)
    n, nb = 8, 6
    canon = _canon(rng, n)
    om, th, sg = (x.astype(np.float64) for x in pa_inputs.random_deform(n, nb, rng))
    t = pa_inputs.frame_times(5).astype(np.float64)
    h1 = oracle.deform(canon, om, th, sg, t) / canon[None] - 1.0
    h2 = oracle.deform(canon, 2 * om, th, sg, t) / canon[None] - 1.0
    np.testing.assert_allclose(h2, 2 * h1, rtol=1e-12, atol=1e-15)
    om3 = om.copy()
    om3[3] += 0.1  # change only the size channel
    out1 = oracle.deform(canon, om, th, sg, t)
    out3 = oracle.deform(canon, om3, th, sg, t)
    for ch in (0, 1, 2, 4):
        np.testing.assert_array_equal(out1[:, ch], out3[:, ch])
    assert np.all(out1[:, 3] != out3[:, 3])


def test_multiplicative_form_keeps_origin_fixed():
    """Eq. 1 scales coordinates: a ball at the origin never moves."""
    rng = np.random.default_rng(3)
    canon = np.array([[0.0], [0.0], [0.0], [0.2], [1.0]])
    om, th, sg = (x.astype(np.float64) for x in pa_inputs.random_deform(1, 4, rng, omega_scale=0.5))
    out = oracle.deform(canon, om, th, sg, pa_inputs.frame_times(6))
    assert not np.any(out[:, :3])


def test_nonpositive_width_is_a_domain_error():
    canon = np.array([[1.0], [1.0], [1.0], [0.2], [1.0]])
    om, th, sg = pa_inputs.deform_init(1, 3)
    sg = sg.astype(np.float64)
    sg[2, 1, 0] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.deform(canon, om, th, sg, np.array([0.5]))


def test_frame_times_are_normalised():
    np.testing.assert_array_equal(pa_inputs.frame_times(1), [0.0])
    np.testing.assert_allclose(pa_inputs.frame_times(5), [0, 0.25, 0.5, 0.75, 1.0])
