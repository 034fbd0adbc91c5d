"""Pins of the oracle's adjoint (gradients of the forward projection and of
the Eq. 1-2 chain rule) by central finite differences of the oracle's own
forward projection, and by the dot-product identity of the linear p map.

The paper states that the baseline attributes and all (theta, sigma, omega)
are learnable (Sec. 2.2) and that the L2 loss drives them (Sec. 2.2, last
paragraph); the adjoint is the exact gradient of that loss.
"""
import math

import numpy as np
import pytest

import oracle
import pa_inputs

C, FS = 1.5, 40.0


def _scene(rng, n=4, ns=3, T=600, t0=15.0):
    balls = np.stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-3, 3, n),
                      rng.uniform(0.15, 0.3, n), rng.uniform(0.2, 1.0, n)])
    sens = pa_inputs.fibonacci_hemisphere(ns, 35.0).astype(np.float64)
    return balls, sens, (C, FS, t0, T, 8.0)


def _functional(state, sens, geom, g):
    y, _ = oracle.forward(state, sens, *geom)
    return float(np.sum(y * g))


def _fd4(fun, x0, h):
    """4th-order central difference of fun at offset 0 along one parameter."""
    return (-fun(2 * h) + 8 * fun(h) - 8 * fun(-h) + fun(-2 * h)) / (12 * h)


def test_adjoint_state_matches_finite_differences():
    rng = np.random.default_rng(21)
    balls, sens, geom = _scene(rng)
    T = geom[3]
    g = rng.standard_normal((1, sens.shape[1], T))
    grad = oracle.adjoint_state(balls, sens, *geom, g)[0]
    for ch in range(5):
        for b in range(balls.shape[1]):
            h = 1e-4 * (balls[3, b] if ch < 4 else balls[4, b])

            def fun(dh):
                q = balls.copy()
                q[ch, b] += dh
                return _functional(q, sens, geom, g)
            fd = _fd4(fun, 0.0, h)
            scale = max(abs(fd), 1e-3 * np.max(np.abs(grad[ch])))
            assert abs(grad[ch, b] - fd) <= 1e-6 * scale, (ch, b, grad[ch, b], fd)


def test_adjoint_dot_product_identity_in_pressure():
    """y is linear in p: <F p, g> = <p, F^T g> with F^T g the p-gradient."""
    rng = np.random.default_rng(8)
    balls, sens, geom = _scene(rng, n=30, ns=5)
    g = rng.standard_normal((1, 5, geom[3]))
    lhs = _functional(balls, sens, geom, g)
    gp = oracle.adjoint_state(balls, sens, *geom, g)[0, 4]
    rhs = float(np.dot(balls[4], gp))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_zero_for_inactive_balls():
    rng = np.random.default_rng(2)
    balls, sens, geom = _scene(rng, n=3)
    balls[3, 0] = 0.0   # zero size
    balls[4, 1] = 0.0   # zero pressure
    g = rng.standard_normal((1, sens.shape[1], geom[3]))
    grad = oracle.adjoint_state(balls, sens, *geom, g)[0]
    assert not np.any(grad[:, 0]) and not np.any(grad[:, 1])
    assert np.all(grad[:, 2] != 0)


def test_loss_is_exact_sum_of_squares():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((3, 4, 50))
    b = rng.standard_normal((3, 4, 50))
    got = oracle.loss(a, b)
    for f in range(3):
        assert got[f] == pytest.approx(math.fsum(((a[f] - b[f]) ** 2).ravel()), rel=1e-14)


def test_adjoint_4d_matches_finite_differences():
    """Gradients w.r.t. canonical attributes and every (omega, theta, sigma)
    through Eq. 1-2 and the forward projection."""
    rng = np.random.default_rng(31)
    n, nb, nf, ns = 3, 3, 4, 3
    canon, sens, geom = _scene(rng, n=n, ns=ns)
    omega, theta, sigma = pa_inputs.random_deform(n, nb, rng, omega_scale=0.05)
    omega, theta, sigma = (x.astype(np.float64) for x in (omega, theta, sigma))
    t = pa_inputs.frame_times(nf).astype(np.float64)
    g = rng.standard_normal((nf, ns, geom[3]))

    def L(cn, om, th, sg):
        st = oracle.deform(cn, om, th, sg, t)
        return _functional(st, sens, geom, g)

    gc, go, gt, gs = oracle.adjoint_4d(canon, omega, theta, sigma, t, sens, *geom, g)
    params = [canon, omega, theta, sigma]
    grads = [gc, go, gt, gs]
    for pi, (P, G) in enumerate(zip(params, grads)):
        for idx in np.ndindex(P.shape):
            # step on each parameter's natural scale: the ball size for
            # coordinates and size, p for pressure, 1e-3 for weights, the
            # basis width for centres and widths
            if pi == 0:
                h = 1e-4 * (canon[3, idx[1]] if idx[0] < 4 else canon[4, idx[1]])
            elif pi == 1:
                h = 1e-4
            else:
                h = 1e-4 * sigma[idx]

            def fun(dh):
                q = [x.copy() for x in params]
                q[pi][idx] += dh
                return L(*q)
            fd = _fd4(fun, 0.0, h)
            scale = max(abs(fd), 1e-3 * np.max(np.abs(G)))
            assert abs(G[idx] - fd) <= 1e-6 * scale, (pi, idx, G[idx], fd)
