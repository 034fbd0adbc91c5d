"""Shared helpers of the GPU parity tests: seeded inputs moved to the device
and comparison metrics.  No method arithmetic here."""
from __future__ import annotations

import numpy as np
import torch

TRACE_TOL = 1e-5   # relative L2 of traces vs the FP64 oracle (FP32 path)
GRAD_TOL = 1e-4    # relative L2 per gradient group vs the FP64 oracle


def rel_l2(got, want) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.linalg.norm(want)
    return float(np.linalg.norm(got - want) / den) if den > 0 else float(np.linalg.norm(got))


def max_rel_elem(got, want) -> float:
    """Largest element error relative to the largest |want| of the tensor."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.max(np.abs(want))
    return float(np.max(np.abs(got - want)) / scale) if scale > 0 else float(np.max(np.abs(got)))


def dev_pad(a: np.ndarray, dev="cuda") -> torch.Tensor:
    """numpy [..., N] -> zero-padded float32 CUDA tensor [..., round4(N)]."""
    import paper_2412_03898_gb300 as pa
    return pa.pad_last(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev))


def geometry(sc, dev="cuda", sensors=None):
    import paper_2412_03898_gb300 as pa
    s = sc.sensors if sensors is None else sensors
    return pa.Geometry(torch.from_numpy(np.ascontiguousarray(s, dtype=np.float32)).to(dev), sc.c, sc.fs, sc.t0,
                       sc.n_samples, sc.kappa)
