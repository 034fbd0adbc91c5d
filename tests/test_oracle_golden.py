"""Regression of the oracle against its committed fixture and the paper's
printed constants."""
import json
import os

import numpy as np

import oracle
from golden.make_golden import case

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_committed_fixture():
    with open(os.path.join(HERE, "golden", "oracle_small.json")) as fh:
        gold = json.load(fh)
    sc, g = case()
    y, n = oracle.forward(sc.balls, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    assert n == gold["n_contributions"]
    for key, val in gold["trace_nonzero"].items():
        s, k = map(int, key.split(","))
        assert abs(y[0, s, k] - val) <= 1e-13 * abs(val)
    grad = oracle.adjoint_state(sc.balls, sc.sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g)
    np.testing.assert_allclose(grad[0], np.array(gold["grad_state"]), rtol=1e-12, atol=0)


def test_paper_constants_fixture():
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as fh:
        c = json.load(fh)
    assert c["n_basis"]["value"] == 65
    assert c["step_size"]["value"] == 160 and c["drop_rate"]["value"] == 0.1
    assert abs(c["hours_reference_frame"]["value"] + c["hours_4d"]["value"] - 5.98) < 1e-9
