"""Seeded synthetic inputs for the 4D Gaussian-ball photoacoustic workloads.

This module only *generates* inputs (sensor layouts, phantoms, ground-truth
motion, deformation-parameter initialisations).  It contains none of the
method's arithmetic: no deformation function, no radiator, no loss.  Both the
FP64 oracle tests and the CUDA path draw their inputs from here, so that the
two implementations never share computational code.

Geometry conventions: lengths in mm, times in microseconds, sampling rate in
MHz, sound speed in mm/us.  Ball state channels are ordered (x, y, z, a, p):
centre, Gaussian standard deviation ("size", a0 in Sec. 2.1) and peak initial
pressure (p0 in Sec. 2.1).

Workload recipes follow the paper's geometry style: Fibonacci sensor layouts
(Sec. 3.1, 3.2), a phantom centred in a cube inside the array (Sec. 3.1,
3.2), vessel-like structures (Sec. 3.2) and pulsation-type motion (Sec. 3.1).
The paper's own ground-truth volumes and its rat-liver data are not
available, so these seeded phantoms stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "CH_X", "CH_Y", "CH_Z", "CH_A", "CH_P", "N_CH",
    "Scene", "fibonacci_hemisphere", "fibonacci_sphere", "tube_phantom",
    "vessel_tree", "gt_motion_frames", "frame_times", "deform_init",
    "random_deform", "config_scene", "CONFIG_NAMES", "small_scene",
]

CH_X, CH_Y, CH_Z, CH_A, CH_P = range(5)
N_CH = 5

GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


@dataclasses.dataclass
class Scene:
    """One synthetic workload.

    balls:   float32 [5, N] canonical state (x, y, z, a, p)
    sensors: float32 [3, S] sensor positions
    c, fs, t0, n_samples, kappa: acquisition scalars
    frames:  optional float32 [F, 5, N] ground-truth per-frame states
    axis:    optional float32 [3, N] closest tube-axis point per ball
    """
    name: str
    balls: np.ndarray
    sensors: np.ndarray
    c: float
    fs: float
    t0: float
    n_samples: int
    kappa: float
    n_frames: int = 1
    frames: Optional[np.ndarray] = None
    axis: Optional[np.ndarray] = None

    @property
    def n_balls(self) -> int:
        return int(self.balls.shape[1])

    @property
    def n_sensors(self) -> int:
        return int(self.sensors.shape[1])


def fibonacci_sphere(n: int, radius: float) -> np.ndarray:
    """n points on a full sphere by the golden-angle spiral (Sec. 3.1 layout)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - 2.0 * (i + 0.5) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * GOLDEN_ANGLE
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z]) * radius
    return pts.astype(np.float32)


def fibonacci_hemisphere(n: int, radius: float) -> np.ndarray:
    """n points on the lower hemisphere (z <= 0) by the golden-angle spiral."""
    i = np.arange(n, dtype=np.float64)
    z = -(i + 0.5) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * GOLDEN_ANGLE
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z]) * radius
    return pts.astype(np.float32)


def _fill_tube(rng, p0, p1, radius, n):
    """n points uniform inside the cylinder p0->p1 of the given radius,
    sorted along the axis (spatially coherent order).  Returns (pts, axis)."""
    d = p1 - p0
    length = float(np.linalg.norm(d))
    u = d / max(length, 1e-12)
    # orthonormal frame around the axis
    helper = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(u, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    s = np.sort(rng.uniform(0.0, length, n))
    rr = radius * np.sqrt(rng.uniform(0.0, 1.0, n))
    th = rng.uniform(0.0, 2.0 * np.pi, n)
    axis = p0[None, :] + s[:, None] * u[None, :]
    pts = axis + (rr * np.cos(th))[:, None] * e1[None, :] + (rr * np.sin(th))[:, None] * e2[None, :]
    return pts, axis


def tube_phantom(n_balls: int, n_tubes: int, tube_radius: float, cube: float,
                 a_range, p_range, rng) -> tuple[np.ndarray, np.ndarray]:
    """Straight tubes with random endpoints in a cube of side `cube` centred at
    the origin; ball centres uniform inside the tubes (equal share per tube)."""
    half = cube / 2.0
    counts = np.full(n_tubes, n_balls // n_tubes)
    counts[: n_balls - counts.sum()] += 1
    pts, axes = [], []
    for t in range(n_tubes):
        p0 = rng.uniform(-half + tube_radius, half - tube_radius, 3)
        p1 = rng.uniform(-half + tube_radius, half - tube_radius, 3)
        q, ax = _fill_tube(rng, p0, p1, tube_radius, int(counts[t]))
        pts.append(q)
        axes.append(ax)
    pts = np.concatenate(pts)
    axes = np.concatenate(axes)
    a = rng.uniform(a_range[0], a_range[1], n_balls)
    p = rng.uniform(p_range[0], p_range[1], n_balls)
    balls = np.stack([pts[:, 0], pts[:, 1], pts[:, 2], a, p]).astype(np.float32)
    return balls, axes.T.astype(np.float32)


def _tree_segments(rng, n_tubes: int, cube: float):
    """Recursive bifurcation: a root enters near the -x face and splits in two
    at each node until n_tubes segments exist.  Radii are log-uniform in
    [0.2, 1.5] mm, assigned in decreasing order by depth (root thickest)."""
    half = cube / 2.0
    radii = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(1.5), n_tubes)))[::-1]
    segs = []
    start = np.array([-half * 0.9, rng.uniform(-0.2, 0.2) * half, rng.uniform(-0.2, 0.2) * half])
    direction = np.array([1.0, rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2)])
    frontier = [(start, direction / np.linalg.norm(direction))]
    while len(segs) < n_tubes and frontier:
        p0, u = frontier.pop(0)
        r = float(radii[len(segs)])
        length = rng.uniform(0.25, 0.45) * cube
        p1 = p0 + length * u
        # shorten so the segment stays inside the cube (with its radius)
        lim = half - r
        for _ in range(60):
            if np.all(np.abs(p1) <= lim):
                break
            length *= 0.9
            p1 = p0 + length * u
        p1 = np.clip(p1, -lim, lim)
        segs.append((p0, p1, r))
        # two children rotated by +-(20..45) degrees about a random normal
        for sign in (1.0, -1.0):
            ang = sign * rng.uniform(np.radians(20), np.radians(45))
            nrm = np.cross(u, rng.normal(size=3))
            nrm /= np.linalg.norm(nrm)
            # Rodrigues rotation of u about nrm
            v = (u * math.cos(ang) + np.cross(nrm, u) * math.sin(ang)
                 + nrm * np.dot(nrm, u) * (1 - math.cos(ang)))
            frontier.append((p1.copy(), v / np.linalg.norm(v)))
    return segs


def vessel_tree(n_balls: int, cube: float, a_range, p_range, rng,
                n_tubes: int = 20) -> tuple[np.ndarray, np.ndarray]:
    """Vessel-like phantom: n_tubes branching tubes in a cube of side `cube`
    centred at the origin; ball counts proportional to tube volume."""
    segs = _tree_segments(rng, n_tubes, cube)
    vols = np.array([math.pi * r * r * np.linalg.norm(p1 - p0) for p0, p1, r in segs])
    counts = np.floor(n_balls * vols / vols.sum()).astype(np.int64)
    counts[np.argmax(vols)] += n_balls - counts.sum()
    pts, axes = [], []
    for (p0, p1, r), k in zip(segs, counts):
        if k == 0:
            continue
        q, ax = _fill_tube(rng, p0, p1, r, int(k))
        pts.append(q)
        axes.append(ax)
    pts = np.concatenate(pts)
    axes = np.concatenate(axes)
    a = rng.uniform(a_range[0], a_range[1], n_balls)
    p = rng.uniform(p_range[0], p_range[1], n_balls)
    balls = np.stack([pts[:, 0], pts[:, 1], pts[:, 2], a, p]).astype(np.float32)
    return balls, axes.T.astype(np.float32)


def frame_times(n_frames: int) -> np.ndarray:
    """Normalised frame times t_f = f/(F-1) (t = 0 for a single frame)."""
    if n_frames <= 1:
        return np.zeros(max(n_frames, 0), dtype=np.float32)
    return (np.arange(n_frames, dtype=np.float64) / (n_frames - 1)).astype(np.float32)


def gt_motion_frames(balls: np.ndarray, axis: np.ndarray, n_frames: int,
                     amplitude: float = 0.1, period: float = 8.0,
                     drift=(0.3, 0.3, 0.2)) -> np.ndarray:
    """Ground-truth per-frame states: every ball moves radially away from its
    tube axis by the factor 1 + amplitude*sin(2 pi f / period), its size scales
    by the same factor, and the whole phantom drifts rigidly by
    (f/(F-1)) * drift (|drift| <= 0.5 mm).  Returns float32 [F, 5, N]."""
    F = n_frames
    out = np.empty((F, 5, balls.shape[1]), dtype=np.float32)
    pos = balls[:3].astype(np.float64)
    ax = axis.astype(np.float64)
    d = np.asarray(drift, dtype=np.float64)
    for f in range(F):
        g = 1.0 + amplitude * math.sin(2.0 * math.pi * f / period)
        frac = f / (F - 1) if F > 1 else 0.0
        q = ax + g * (pos - ax) + frac * d[:, None]
        out[f, :3] = q
        out[f, 3] = balls[3].astype(np.float64) * g
        out[f, 4] = balls[4]
    return out


def deform_init(n_balls: int, n_basis: int):
    """Neutral deformation parameters: omega = 0 (every frame equals the
    canonical cloud), centres evenly spaced on [0, 1], widths 1/Nb.
    Returns (omega, theta, sigma), each float32 [5, Nb, N]."""
    omega = np.zeros((5, n_basis, n_balls), dtype=np.float32)
    th = np.linspace(0.0, 1.0, n_basis, dtype=np.float64) if n_basis > 1 else np.zeros(1)
    theta = np.broadcast_to(th[None, :, None], (5, n_basis, n_balls)).astype(np.float32)
    sigma = np.full((5, n_basis, n_balls), 1.0 / n_basis, dtype=np.float32)
    return omega, theta.copy(), sigma


def random_deform(n_balls: int, n_basis: int, rng, omega_scale=0.02,
                  sigma_range=(0.05, 0.4)):
    """Random deformation parameters for tests: small weights so that the
    deformed attributes stay close to the canonical ones."""
    omega = (rng.standard_normal((5, n_basis, n_balls)) * omega_scale / math.sqrt(max(n_basis, 1))).astype(np.float32)
    theta = rng.uniform(0.0, 1.0, (5, n_basis, n_balls)).astype(np.float32)
    sigma = rng.uniform(sigma_range[0], sigma_range[1], (5, n_basis, n_balls)).astype(np.float32)
    return omega, theta, sigma


CONFIG_NAMES = {
    1: "static-2k: 2,000 balls / 5 tubes in a 10 mm cube, 64 sensors R=40 mm, T=1024",
    2: "static-100k: 100,000-ball vessel tree in a 30 mm cube, 576 sensors R=55 mm, T=4096",
    3: "4d-100k-20f: 100,000 canonical balls, 20 frames, 576 sensors R=55 mm, T=4096",
    4: "4d-1m-50f: 1,000,000-ball vessel tree in a 60 mm cube, 1024 sensors R=80 mm, T=4096, 50 frames",
    5: "batched-16: 16 uneven scenes, N log-uniform [1e4, 5e5], S in {256,576,1024}, T in [2048,4096], F in [1,10]",
}


def config_scene(cfg: int, n_balls: Optional[int] = None) -> Scene | list[Scene]:
    """The five benchmark workloads.  `n_balls` optionally overrides the ball
    count (for reduced-size test variants of the same recipe)."""
    c, fs, kappa = 1.5, 40.0, 5.0
    if cfg == 1:
        rng = np.random.default_rng(0)
        n = n_balls or 2000
        balls, axis = tube_phantom(n, 5, 0.5, 10.0, (0.1, 0.3), (0.2, 1.0), rng)
        return Scene("static-2k", balls, fibonacci_hemisphere(64, 40.0), c, fs, 20.0, 1024, kappa, 1, None, axis)
    if cfg == 2:
        rng = np.random.default_rng(1)
        n = n_balls or 100_000
        balls, axis = vessel_tree(n, 30.0, (0.1, 0.4), (0.2, 1.0), rng)
        return Scene("static-100k", balls, fibonacci_hemisphere(576, 55.0), c, fs, 0.0, 4096, kappa, 1, None, axis)
    if cfg == 3:
        rng = np.random.default_rng(2)
        n = n_balls or 100_000
        balls, axis = vessel_tree(n, 30.0, (0.1, 0.4), (0.2, 1.0), rng)
        F = 20
        frames = gt_motion_frames(balls, axis, F)
        return Scene("4d-100k-20f", frames[0].copy(), fibonacci_hemisphere(576, 55.0), c, fs, 0.0, 4096, kappa, F, frames, axis)
    if cfg == 4:
        rng = np.random.default_rng(3)
        n = n_balls or 1_000_000
        balls, axis = vessel_tree(n, 60.0, (0.1, 0.4), (0.2, 1.0), rng)
        F = 50
        return Scene("4d-1m-50f", balls, fibonacci_hemisphere(1024, 80.0), c, fs, 0.0, 4096, kappa, F, None, axis)
    if cfg == 5:
        scenes = []
        for i in range(16):
            rng = np.random.default_rng(4 + i)
            n = int(round(math.exp(rng.uniform(math.log(1e4), math.log(5e5)))))
            if n_balls is not None:
                n = max(64, int(n * n_balls / 1e5))
            S = int(rng.choice([256, 576, 1024]))
            T = int(rng.integers(512, 1025)) * 4
            F = int(rng.integers(1, 11))
            balls, axis = vessel_tree(n, 30.0, (0.1, 0.4), (0.2, 1.0), rng)
            frames = gt_motion_frames(balls, axis, F) if F > 1 else None
            scenes.append(Scene(f"batched-{i}", balls, fibonacci_hemisphere(S, 55.0), c, fs, 0.0, T, kappa, F, frames, axis))
        return scenes
    raise ValueError(f"unknown config {cfg}")


def small_scene(seed: int, n_balls: int, n_sensors: int, n_samples: int,
                n_frames: int = 1, radius: float = 40.0, cube: float = 10.0,
                a_range=(0.1, 0.3), t0: float = 20.0, kappa: float = 5.0) -> Scene:
    """A small tube phantom for parity tests: several tiles and ragged tails
    are obtained by choosing sizes that are not multiples of the tile sizes."""
    rng = np.random.default_rng(seed)
    balls, axis = tube_phantom(n_balls, 3, 0.5, cube, a_range, (0.2, 1.0), rng)
    frames = gt_motion_frames(balls, axis, n_frames) if n_frames > 1 else None
    return Scene(f"small-{seed}", balls, fibonacci_hemisphere(n_sensors, radius), 1.5, 40.0, t0,
                 n_samples, kappa, n_frames, frames, axis)


def heart_phantom(n_frames: int = 17, spacing: float = 0.4, a: float = 0.25, seed: int = 7) -> Scene:
    """The "simulated heart" of the paper's first simulation (Sec. 3.1), built
    from Gaussian balls: three mutually perpendicular rectangular slabs of
    uniform pressure (stationary) and a Gaussian ellipsoid at the centre whose
    pressure and size pulse over the frames, inside the cube (-25.6, 25.6) mm^3,
    seen by 1,024 sensors on a full Fibonacci sphere of radius 60 mm.  The
    paper gives no dimensions for the slabs or the ellipsoid; these are chosen
    to fill the cube's centre: slabs 30 x 8 x 2 mm along x, y and z, ellipsoid
    semi-axes (6, 4.5, 3.5) mm scaled by 1 + 0.15 sin(2 pi f / F) with peak
    pressure 1 + 0.3 sin(2 pi f / F).

    Slab balls sit on a jittered lattice of the given spacing (same every
    frame); ellipsoid balls on a lattice whose positions scale with the
    ellipsoid and whose pressure follows the Gaussian profile
    exp(-r_e^2 / 2), r_e the ellipsoidal radius in units of the semi-axes,
    kept out to r_e <= 2.  Returns a Scene whose `frames` holds the F states
    (the ball count is the same in every frame)."""
    rng = np.random.default_rng(seed)

    def lattice(ext):
        axes = [np.arange(-e / 2 + spacing / 2, e / 2, spacing) for e in ext]
        g = np.stack(np.meshgrid(*axes, indexing="ij")).reshape(3, -1)
        return g + rng.uniform(-0.1 * spacing, 0.1 * spacing, g.shape)

    slabs = []
    for ext in ((30.0, 8.0, 2.0), (2.0, 30.0, 8.0), (8.0, 2.0, 30.0)):
        slabs.append(lattice(ext))
    slab_pos = np.concatenate(slabs, axis=1)
    semi = np.array([6.0, 4.5, 3.5])
    unit = lattice(tuple(4.0 * semi)) / semi[:, None]  # in units of the semi-axes
    re2 = (unit ** 2).sum(0)
    unit = unit[:, re2 <= 4.0]
    re2 = re2[re2 <= 4.0]
    n_slab, n_ell = slab_pos.shape[1], unit.shape[1]
    frames = np.empty((n_frames, 5, n_slab + n_ell), dtype=np.float32)
    for f in range(n_frames):
        ph = math.sin(2.0 * math.pi * f / n_frames)
        scale, peak = 1.0 + 0.15 * ph, 1.0 + 0.3 * ph
        frames[f, :3, :n_slab] = slab_pos
        frames[f, 3, :n_slab] = a
        frames[f, 4, :n_slab] = 0.6
        frames[f, :3, n_slab:] = unit * semi[:, None] * scale
        frames[f, 3, n_slab:] = a * scale
        frames[f, 4, n_slab:] = peak * np.exp(-re2 / 2.0)
    sensors = fibonacci_sphere(1024, 60.0)
    return Scene("heart-sim1", frames[0].copy(), sensors, 1.5, 40.0, 0.0, 4096, 5.0, n_frames, frames, None)
