"""Brute-force photoacoustic pressure from Poisson's spherical-mean formula.

Independent of the oracle's closed form: the initial pressure is voxelised
and the pressure at a sensor is obtained numerically from

    p(r, t) = d/dt [ t * M_{ct}[p_init](r) ],  M_s = mean of p_init over the
    sphere of radius s around r,

which with s = c t becomes p = d/ds [ Phi(s) / (4 pi s) ], Phi(s) being the
surface integral of p_init over that sphere.  Phi is estimated by summing
voxel masses with a narrow normalised Gaussian kernel g_w(d_v - s) in the
distance d_v of each voxel from the sensor.  The derivative in s is taken
analytically through the kernel.

Smoothing Phi (rather than p) along s gives, exactly,
    P_w(s) = (p*g_w)(s) (1 - w^2/s^2) + (w^2/s) (p*g_w')(s),
which `smoothed_target` evaluates from samples of p.
"""
from __future__ import annotations

import math

import numpy as np


def _voxels_gauss(ball, h, extent):
    x, y, z, a, p = (float(v) for v in ball)
    m = int(math.ceil(extent * a / h))
    g = np.arange(-m, m + 1) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    r2 = X * X + Y * Y + Z * Z
    val = p * np.exp(-r2 / (2 * a * a)) * h ** 3
    keep = val > 0
    return np.stack([X[keep] + x, Y[keep] + y, Z[keep] + z]), val[keep]


def _voxels_uniform(ball, h, sub):
    """Uniform ball of radius a: voxel masses by sub x sub x sub supersampling."""
    x, y, z, a, p = (float(v) for v in ball)
    m = int(math.ceil(a / h)) + 1
    g = np.arange(-m, m + 1) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    frac = np.zeros_like(X)
    offs = (np.arange(sub) + 0.5) / sub - 0.5
    for ox in offs:
        for oy in offs:
            for oz in offs:
                rr = (X + ox * h) ** 2 + (Y + oy * h) ** 2 + (Z + oz * h) ** 2
                frac += rr <= a * a
    frac /= sub ** 3
    keep = frac > 0
    return np.stack([X[keep] + x, Y[keep] + y, Z[keep] + z]), p * frac[keep] * h ** 3


def smoothed_pressure(ball, sensor, s_values, w, h, profile="gauss", extent=7.0, sub=3):
    """Pressure at `sensor` for travelled distances s = c t in `s_values`,
    smoothed along s by a Gaussian of standard deviation w."""
    if profile == "gauss":
        pos, mass = _voxels_gauss(ball, h, extent)
    else:
        pos, mass = _voxels_uniform(ball, h, sub)
    d = np.sqrt(((pos - np.asarray(sensor, dtype=np.float64)[:, None]) ** 2).sum(axis=0))
    order = np.argsort(d)
    d = d[order]
    mass = mass[order]
    out = np.empty(len(s_values))
    cut = 9.0 * w
    norm = 1.0 / (math.sqrt(2 * math.pi) * w)
    for i, s in enumerate(s_values):
        lo, hi = np.searchsorted(d, [s - cut, s + cut])
        u = d[lo:hi] - s
        g = norm * np.exp(-u * u / (2 * w * w))
        # d/ds [ sum m g(d - s) / (4 pi s) ]
        out[i] = (np.sum(mass[lo:hi] * g * u) / (w * w) / s - np.sum(mass[lo:hi] * g) / (s * s)) / (4 * math.pi)
    return out


def gaussian_smooth_samples(y, delta, w, out_index, deriv=False):
    """Riemann-sum convolution of uniformly sampled y (spacing delta, the
    sample axis running along increasing s) with a normalised Gaussian of
    standard deviation w (or its derivative), evaluated at out_index."""
    j = np.arange(len(y))
    norm = delta / (math.sqrt(2 * math.pi) * w)
    res = np.empty(len(out_index))
    for i, k in enumerate(out_index):
        u = (k - j) * delta
        g = norm * np.exp(-u * u / (2 * w * w))
        if deriv:
            g = g * (-u / (w * w))
        res[i] = np.sum(y * g)
    return res


def smoothed_target(y, delta, w, out_index, s_values):
    """What smoothed_pressure returns for a field whose samples along s are y."""
    pg = gaussian_smooth_samples(y, delta, w, out_index)
    pdg = gaussian_smooth_samples(y, delta, w, out_index, deriv=True)
    s = np.asarray(s_values, dtype=np.float64)
    return pg * (1 - w * w / (s * s)) + (w * w / s) * pdg
