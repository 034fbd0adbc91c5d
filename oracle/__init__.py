"""FP64 CPU oracle for the 4D SlingBAG hot path (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference leg
of ``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.  The arithmetic lives in ``pa_oracle.c`` (plain
double-precision loop nests, OpenMP over independent output rows); this module
compiles it with gcc on first use and marshals numpy arrays in and out.

All inputs are promoted to float64 exactly (fp32 -> fp64 is exact), so the
oracle measures the method, not input rounding.

Parity pins: see tests/test_oracle_radiator.py, tests/test_oracle_adjoint.py
and tests/test_oracle_deform.py.  Every function here is pinned by at least
one of them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "pa_oracle_image.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PROFILE_GAUSS = 0
PROFILE_UNIFORM = 1
ERR_DOMAIN = 2


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile pa_oracle.c and pa_oracle_image.c into liboracle.so (IEEE
    double, no fast-math)."""
    if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS):
        return _LIB
    tmp = f"{_LIB}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(ctypes.c_double)
            I64P = ctypes.POINTER(ctypes.c_int64)
            i32, i64, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.oracle_max_threads.restype = i32
            lib.oracle_pressure_full.restype = d
            lib.oracle_pressure_full.argtypes = [d, d, d, d]
            lib.oracle_deform.restype = i32
            lib.oracle_deform.argtypes = [i64, i32, P, P, P, P, i32, P, P]
            lib.oracle_forward.restype = i32
            lib.oracle_forward.argtypes = [i32, i64, P, i32, P, d, d, d, i32, d, i32, P, I64P, I64P, i32]
            lib.oracle_loss.restype = i32
            lib.oracle_loss.argtypes = [i32, i64, P, P, P]
            lib.oracle_adjoint_state.restype = i32
            lib.oracle_adjoint_state.argtypes = [i32, i64, P, i32, P, d, d, d, i32, d, P, P, i32]
            lib.oracle_deform_backward.restype = i32
            lib.oracle_deform_backward.argtypes = [i64, i32, P, P, P, P, i32, P, P, P, P, P, P]
            lib.oracle_adjoint_4d.restype = i32
            lib.oracle_adjoint_4d.argtypes = [i64, i32, P, P, P, P, i32, P, i32, P, d, d, d, i32, d,
                                              P, P, P, P, P, i32]
            lib.oracle_ubp_filter.restype = i32
            lib.oracle_ubp_filter.argtypes = [i32, i32, d, d, P, P]
            lib.oracle_ubp.restype = i32
            lib.oracle_ubp.argtypes = [i32, i32, P, P, d, d, d, P, P, d, i32, i32, i32, P, i32]
            lib.oracle_splat.restype = i32
            lib.oracle_splat.argtypes = [i64, P, d, P, d, i32, i32, i32, P, i32]
            lib.oracle_ssim.restype = i32
            lib.oracle_ssim.argtypes = [i32, i32, P, P, d, P, P]
            _lib = lib
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def pressure_full(p, a, R, ct) -> float:
    """Both terms of the Poisson solution for one Gaussian ball."""
    return float(_load().oracle_pressure_full(float(p), float(a), float(R), float(ct)))


def deform(canon, omega, theta, sigma, t) -> np.ndarray:
    """Eq. 1-2.  canon [5,N]; omega/theta/sigma [5,Nb,N]; t [F] -> [F,5,N]."""
    canon, omega, theta, sigma, t = map(_d, (canon, omega, theta, sigma, t))
    n = canon.shape[1]
    nb = omega.shape[1]
    nf = t.shape[0]
    out = np.zeros((nf, 5, n))
    rc = _load().oracle_deform(n, nb, _p(canon), _p(omega), _p(theta), _p(sigma), nf, _p(t), _p(out))
    if rc:
        raise OracleError(f"oracle_deform failed ({rc})")
    return out


def forward(state, sensors, c, fs, t0, n_samples, kappa, profile=PROFILE_GAUSS,
            nthreads=0, allow_domain=False):
    """Forward projection.  state [F,5,N] (or [5,N]); sensors [3,S].
    Returns (traces [F,S,T], n_contributions)."""
    state = _d(state)
    if state.ndim == 2:
        state = state[None]
    sensors = _d(sensors)
    nf, _, n = state.shape
    ns = sensors.shape[1]
    out = np.zeros((nf, ns, int(n_samples)))
    cnt = ctypes.c_int64(0)
    bad = ctypes.c_int64(0)
    rc = _load().oracle_forward(nf, n, _p(state), ns, _p(sensors), float(c), float(fs), float(t0),
                                int(n_samples), float(kappa), int(profile), _p(out),
                                ctypes.byref(cnt), ctypes.byref(bad), int(nthreads))
    if rc and not (rc == ERR_DOMAIN and allow_domain):
        raise OracleError(f"oracle_forward failed ({rc}); domain pairs={bad.value}")
    return out, int(cnt.value)


def loss(pred, meas) -> np.ndarray:
    """Per-frame sum of squared residuals.  pred/meas [F,S,T] -> [F]."""
    pred, meas = _d(pred), _d(meas)
    nf = pred.shape[0]
    per = int(np.prod(pred.shape[1:]))
    out = np.zeros(nf)
    _load().oracle_loss(nf, per, _p(pred), _p(meas), _p(out))
    return out


def adjoint_state(state, sensors, c, fs, t0, n_samples, kappa, g, nthreads=0,
                  allow_domain=False):
    """dL/d(state) given g = dL/dy.  state [F,5,N]; g [F,S,T] -> [F,5,N]."""
    state = _d(state)
    if state.ndim == 2:
        state = state[None]
    sensors, g = _d(sensors), _d(g)
    nf, _, n = state.shape
    ns = sensors.shape[1]
    out = np.zeros((nf, 5, n))
    rc = _load().oracle_adjoint_state(nf, n, _p(state), ns, _p(sensors), float(c), float(fs), float(t0),
                                      int(n_samples), float(kappa), _p(g), _p(out), int(nthreads))
    if rc and not (rc == ERR_DOMAIN and allow_domain):
        raise OracleError(f"oracle_adjoint_state failed ({rc})")
    return out


def deform_backward(canon, omega, theta, sigma, t, gstate):
    """Chain rule of Eq. 1-2.  Returns (g_canon [5,N], g_omega, g_theta, g_sigma [5,Nb,N])."""
    canon, omega, theta, sigma, t, gstate = map(_d, (canon, omega, theta, sigma, t, gstate))
    n = canon.shape[1]
    nb = omega.shape[1]
    nf = t.shape[0]
    gc = np.zeros((5, n))
    go, gt, gs = (np.zeros((5, nb, n)) for _ in range(3))
    _load().oracle_deform_backward(n, nb, _p(canon), _p(omega), _p(theta), _p(sigma), nf, _p(t),
                                   _p(gstate), _p(gc), _p(go), _p(gt), _p(gs))
    return gc, go, gt, gs


def adjoint_4d(canon, omega, theta, sigma, t, sensors, c, fs, t0, n_samples, kappa, g,
               nthreads=0):
    """Full 4D adjoint: (g_canon [5,N], g_omega, g_theta, g_sigma [5,Nb,N])."""
    canon, omega, theta, sigma, t, sensors, g = map(_d, (canon, omega, theta, sigma, t, sensors, g))
    n = canon.shape[1]
    nb = omega.shape[1]
    nf = t.shape[0]
    ns = sensors.shape[1]
    gc = np.zeros((5, n))
    go, gt, gs = (np.zeros((5, nb, n)) for _ in range(3))
    rc = _load().oracle_adjoint_4d(n, nb, _p(canon), _p(omega), _p(theta), _p(sigma), nf, _p(t), ns,
                                   _p(sensors), float(c), float(fs), float(t0), int(n_samples),
                                   float(kappa), _p(g), _p(gc), _p(go), _p(gt), _p(gs), int(nthreads))
    if rc:
        raise OracleError(f"oracle_adjoint_4d failed ({rc})")
    return gc, go, gt, gs


# ---------------------------------------------------------------------------
# Imaging side (pa_oracle_image.c): UBP comparison reconstruction, point
# cloud -> voxels, maximum amplitude projections and SSIM (Sec. 3.1-3.2).

def ubp_filter(traces, fs, t0):
    """b = 2 p - 2 t dp/dt per sensor trace; traces [..., S, T] -> same shape."""
    p = _d(traces)
    shp = p.shape
    T = shp[-1]
    p2 = p.reshape(-1, T)
    b = np.zeros_like(p2)
    rc = _load().oracle_ubp_filter(p2.shape[0], T, float(fs), float(t0), _p(p2), _p(b))
    if rc != 0:
        raise OracleError(f"oracle_ubp_filter: {rc}")
    return b.reshape(shp)


def ubp(b, sensors, center, c, fs, t0, origin, h, shape, nthreads=0):
    """Back-projection of filtered traces b [S, T] onto a grid of shape
    (nz, ny, nx) -> volume [nz, ny, nx]."""
    b, sensors, center, origin = map(_d, (b, sensors, center, origin))
    ns, T = b.shape
    nz, ny, nx = shape
    vol = np.zeros((nz, ny, nx))
    rc = _load().oracle_ubp(ns, T, _p(sensors), _p(center), float(c), float(fs), float(t0), _p(b), _p(origin),
                            float(h), nx, ny, nz, _p(vol), int(nthreads))
    if rc != 0:
        raise OracleError(f"oracle_ubp: {rc}")
    return vol


def splat(state, kappa, origin, h, shape, nthreads=0):
    """Truncated Gaussian-ball pressure sum on a grid: state [5, N] -> [nz, ny, nx]."""
    state, origin = _d(state), _d(origin)
    n = state.shape[1]
    nz, ny, nx = shape
    vol = np.zeros((nz, ny, nx))
    rc = _load().oracle_splat(n, _p(state), float(kappa), _p(origin), float(h), nx, ny, nz, _p(vol), int(nthreads))
    if rc != 0:
        raise OracleError(f"oracle_splat: {rc}")
    return vol


def maps(vol):
    """Maximum amplitude projections of a volume [nz, ny, nx]: (XY = max over
    z [ny, nx], YZ = max over x [nz, ny], XZ = max over y [nz, nx])."""
    v = np.asarray(vol, dtype=np.float64)
    return v.max(axis=0), v.max(axis=2), v.max(axis=1)


def minmax01(x):
    """Scale an image to [0, 1] by its own minimum and maximum (a constant
    image becomes 0)."""
    x = _d(x)
    lo, hi = x.min(), x.max()
    return (x - lo) / (hi - lo) if hi > lo else np.zeros_like(x)


def ssim(x, y, L=1.0, want_map=False, minmax=False):
    """Mean SSIM of two images [H, W] (and the map over valid positions);
    minmax=True compares the [0, 1]-scaled images with L = 1."""
    x, y = _d(x), _d(y)
    if minmax:
        x, y, L = minmax01(x), minmax01(y), 1.0
    H, W = x.shape
    m = np.zeros((H - 10, W - 10))
    out = np.zeros(1)
    rc = _load().oracle_ssim(H, W, _p(x), _p(y), float(L), _p(m), _p(out))
    if rc != 0:
        raise OracleError(f"oracle_ssim: {rc}")
    return (float(out[0]), m) if want_map else float(out[0])
