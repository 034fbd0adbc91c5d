"""Spatial (Morton) order of a cloud and the row gather (pa_spatial_order,
pa_gather_rows) through the C ABI.  The order is a storage layout: the
permutation must equal a host replay of its definition (float32 cells of the
bounding box, interleaved bits, stable sort), and the forward and adjoint of a
reordered cloud must equal the originals up to summation order."""
import numpy as np
import pytest
import torch

import pa_inputs
from gpu_common import GRAD_TOL, dev_pad, geometry, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    import paper_2412_03898_gb300 as m
    return m


def _spread3(v):
    v = v.astype(np.int64) & 0x3FF
    v = (v | (v << 16)) & 0x030000FF
    v = (v | (v << 8)) & 0x0300F00F
    v = (v | (v << 4)) & 0x030C30C3
    v = (v | (v << 2)) & 0x09249249
    return v


def _host_order(balls):
    x = np.ascontiguousarray(balls[:3], dtype=np.float32)
    lo, hi = x.min(axis=1), x.max(axis=1)
    ext = float((hi - lo).astype(np.float32).max())
    a = balls[3].astype(np.float64)
    k = int(np.rint(np.log2(a[a > 0].mean()))) if np.any(a > 0) else -126
    k = max(-126, min(k, 100))
    while k < 100 and 2.0 ** k * 1024.0 < ext:
        k += 1
    t = (x - lo[:, None]) * np.float32(2.0 ** -k)
    q = np.clip(np.floor(t.astype(np.float32)).astype(np.int64), 0, 1023)
    code = _spread3(q[0]) | (_spread3(q[1]) << 1) | (_spread3(q[2]) << 2)
    return np.argsort(code, kind="stable")


@pytest.mark.parametrize("n", [1, 2047, 5003])
def test_spatial_order_matches_host_replay(pa, n):
    sc = pa_inputs.small_scene(seed=31, n_balls=n, n_sensors=8, n_samples=256)
    perm = pa.spatial_order(dev_pad(sc.balls), n)
    assert perm.dtype == torch.int32 and perm.numel() == n
    np.testing.assert_array_equal(perm.cpu().numpy(), _host_order(sc.balls))


def test_spatial_order_full_size_and_gather(pa):
    sc = pa_inputs.config_scene(2)
    n = sc.n_balls
    st = dev_pad(sc.balls)
    perm = pa.spatial_order(st, n)
    p = perm.cpu().numpy()
    np.testing.assert_array_equal(np.sort(p), np.arange(n))
    np.testing.assert_array_equal(p, _host_order(sc.balls))
    out = pa.gather_rows(st, perm)
    want = torch.zeros_like(st)
    want[:, :n] = st[:, perm.long()]
    assert torch.equal(out, want)


def test_reordered_cloud_gives_the_same_traces_and_permuted_gradients(pa):
    sc = pa_inputs.small_scene(seed=32, n_balls=3001, n_sensors=37, n_samples=1024)
    n = sc.n_balls
    geom = geometry(sc)
    st = dev_pad(sc.balls)[None].contiguous()
    perm = pa.spatial_order(st, n)
    st2 = pa.gather_rows(st, perm)
    y = pa.forward(geom, st, n).double()
    y2 = pa.forward(geom, st2, n).double()
    assert float((y2 - y).norm() / y.norm()) <= 1e-6
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(tuple(y.shape)).astype(np.float32)).cuda()
    gs = pa.adjoint(geom, g, state=st, n=n)[0, :, :n]
    gs2 = pa.adjoint(geom, g, state=st2, n=n)[0, :, :n]
    # the adjoint of ball perm[i] is computed alone in either layout: bitwise equal
    assert torch.equal(gs2, gs[:, perm.long()])


def test_gather_rows_of_deformation_parameters(pa):
    rng = np.random.default_rng(5)
    n, nb = 777, 7
    om = dev_pad(rng.standard_normal((5, nb, n)).astype(np.float32))
    perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    out = pa.gather_rows(om, perm)
    assert torch.equal(out[..., :n], om[..., perm.long()])
    assert torch.count_nonzero(out[..., n:]) == 0
