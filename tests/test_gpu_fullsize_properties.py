"""Properties that hold at any size, checked on every output of full-size
workloads in the launch configuration the benchmark times (the FP64 oracle
checks only sampled outputs at these sizes):

- superposition: the forward is linear in the set of balls, so the traces of
  the cloud equal the sum of the traces of its two halves (a ball with p = 0
  contributes nothing), up to FP32 summation order;
- the adjoint's inner-product identity for the pressure-linear part: with
  L = <F(state), g>, sum_b p_b dL/dp_b = L exactly (y is homogeneous of
  degree one in p), which ties every trace sample of the forward to every
  ball gradient of the adjoint, so a tile-seam or window-edge error in either
  kernel breaks it;
- doubling every p doubles every trace sample bitwise (power-of-two scaling
  is exact through the whole path);
- the adjoint's work-queue and grid-stride schedules give bitwise the same
  gradients.

Workloads: static-100k (all 100k balls, 576 sensors x 4096 samples) and the
canonical frame of the 1M-ball workload (1024 sensors x 4096 samples)."""
import numpy as np
import pytest
import torch

import pa_inputs
from gpu_common import dev_pad, geometry

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("cfg", [2, 4])
def test_full_size_superposition_inner_product_and_scaling(cfg):
    import paper_2412_03898_gb300 as pa
    sc = pa_inputs.config_scene(cfg)
    n = sc.n_balls
    geom = geometry(sc)
    st = dev_pad(sc.balls)[None].contiguous()
    y = pa.forward(geom, st, n)
    pa.device_error()

    # superposition over an index split of the cloud
    half = n // 2
    sa, sb = st.clone(), st.clone()
    sa[0, 4, half:] = 0.0
    sb[0, 4, :half] = 0.0
    ysum = pa.forward(geom, sa, n).double() + pa.forward(geom, sb, n).double()
    err = float((ysum - y.double()).norm() / y.double().norm())
    assert err <= 1e-6, err

    # exact scaling by two in p
    s2 = st.clone()
    s2[0, 4] *= 2.0
    assert torch.equal(pa.forward(geom, s2, n), 2.0 * y)

    # inner-product identity, with g close to y so that <y, g> ~ ||y||^2
    rng = np.random.default_rng(100 + cfg)
    noise = torch.from_numpy(rng.standard_normal(tuple(y.shape)).astype(np.float32)).cuda()
    g = (y + 0.5 * y.pow(2).mean().sqrt() * noise).contiguous()
    lhs = float((y.double() * g.double()).sum())
    gs = pa.adjoint(geom, g, state=st, n=n)
    pa.device_error()
    # the work-queue schedule (default) and the grid-stride one compute each
    # (frame, ball) item whole in one warp: bitwise the same gradients
    assert torch.equal(gs[..., :n], pa.adjoint(geom, g, state=st, n=n, queue=False)[..., :n])
    rhs = float((st[0, 4, :n].double() * gs[0, 4, :n].double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
