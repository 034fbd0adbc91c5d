"""Writes tests/golden/oracle_small.json: a small forward/adjoint case
computed by the FP64 oracle only (regression fixture for the oracle; any
later change to the oracle's arithmetic shows up here).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import pa_inputs  # noqa: E402


def case():
    sc = pa_inputs.small_scene(seed=123, n_balls=7, n_sensors=3, n_samples=512)
    rng = np.random.default_rng(99)
    g = rng.standard_normal((1, 3, 512)).astype(np.float32)
    return sc, g


def main():
    sc, g = case()
    y, n = oracle.forward(sc.balls, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    grad = oracle.adjoint_state(sc.balls, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g)
    out = {
        "_note": "generated by tests/golden/make_golden.py from oracle/ only",
        "n_contributions": n,
        "trace_nonzero": {f"{s},{k}": float(y[0, s, k]) for s in range(3) for k in np.nonzero(y[0, s])[0][::7]},
        "grad_state": grad[0].tolist(),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
