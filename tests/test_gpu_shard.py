"""Sharding of the path by sensors (how several GPUs would split it): a
sensor shard is an offset into the sensor array, the forward projection of
each shard equals that slice of the full result, and the per-shard adjoint
gradients sum to the full gradient (the one all-reduce a multi-GPU adjoint
needs)."""
import numpy as np
import pytest
import torch

import pa_inputs
from gpu_common import dev_pad, geometry

pytestmark = pytest.mark.gpu


def test_sensor_shards_forward_and_adjoint():
    import paper_2412_03898_gb300 as pa
    sc = pa_inputs.small_scene(seed=9, n_balls=700, n_sensors=37, n_samples=1024, n_frames=2)
    geom = geometry(sc)
    st = dev_pad(sc.frames)
    full = pa.forward(geom, st, sc.n_balls, tiles=(8, 1024, 256, 1, 8))
    bounds = [(0, 13), (13, 30), (30, 37)]
    for b, e in bounds:
        part = pa.forward(geom.shard(b, e), st, sc.n_balls, tiles=(8, 1024, 256, 1, 8))
        # same per-sensor code and tiles: bitwise the same traces
        assert torch.equal(part, full[:, b:e])
    rng = np.random.default_rng(2)
    g = torch.from_numpy(rng.standard_normal((2, 37, 1024)).astype(np.float32)).cuda()
    gfull = pa.adjoint(geom, g, state=st, n=sc.n_balls)
    acc = torch.zeros_like(gfull)
    for b, e in bounds:
        acc += pa.adjoint(geom.shard(b, e), g[:, b:e].contiguous(), state=st, n=sc.n_balls)
    n = sc.n_balls
    torch.testing.assert_close(acc[..., :n], gfull[..., :n], rtol=1e-5, atol=1e-6 * float(gfull.abs().max()))
