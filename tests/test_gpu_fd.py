"""GPU gradients of the 4D path against FP64 finite differences.

The whole differentiable chain as the IR runs it -- PAProject4D (states
deformed per frame chunk by Eq. 1-2, pa_forward_4d; backward pa_adjoint_4d)
and PALoss (the per-frame L2 loss of Sec. 2.2, last paragraph) through
torch.autograd -- is compared, per parameter group (the canonical
attributes and every omega, theta, sigma, all learnable by Sec. 2.2), with
4th-order central differences of the same loss evaluated by the FP64
oracle's deformation and forward projection.  kappa = 8 puts the window
edges at exp(-32) of the peak, so the truncated forward is smooth to FP64
precision at the steps used; the inputs are FP32 values promoted exactly."""
import numpy as np
import pytest
import torch

import oracle
import pa_inputs
from gpu_common import GRAD_TOL, dev_pad, rel_l2

pytestmark = pytest.mark.gpu

C, FS, T0, T, KAPPA = 1.5, 40.0, 15.0, 600, 8.0


def _fd4(fun, h):
    return (-fun(2 * h) + 8 * fun(h) - 8 * fun(-h) + fun(-2 * h)) / (12 * h)


@pytest.mark.parametrize("frames_per_chunk", [0, 2])
def test_autograd_4d_gradients_match_fp64_finite_differences(frames_per_chunk):
    import paper_2412_03898_gb300 as pa
    rng = np.random.default_rng(77)
    n, nb, F, S = 5, 3, 5, 6
    canon = np.stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-3, 3, n),
                      rng.uniform(0.15, 0.3, n), rng.uniform(0.2, 1.0, n)]).astype(np.float32)
    om, th, sg = pa_inputs.random_deform(n, nb, rng, omega_scale=0.05)
    sens = pa_inputs.fibonacci_hemisphere(S, 35.0).astype(np.float32)
    t = pa_inputs.frame_times(F).astype(np.float32)
    meas = (0.01 * rng.standard_normal((F, S, T))).astype(np.float32)
    geom_args = (C, FS, T0, T, KAPPA)

    # GPU: loss and gradients through autograd
    geom = pa.Geometry(torch.from_numpy(sens).cuda(), C, FS, T0, T, KAPPA)
    c_d = dev_pad(canon).requires_grad_(True)
    d_d = torch.stack([dev_pad(x) for x in (om, th, sg)]).requires_grad_(True)
    t_d = torch.from_numpy(t).cuda()
    plan = pa.Plan.from_values(frames_per_chunk=frames_per_chunk) if frames_per_chunk else None
    y = pa.PAProject4D.apply(c_d, d_d, geom, t_d, n, plan)
    loss = pa.PALoss.apply(y, torch.from_numpy(meas).cuda()).sum()
    loss.backward()
    pa.device_error()
    got = [c_d.grad[:, :n].cpu().numpy().astype(np.float64)] + \
          [d_d.grad[i][..., :n].cpu().numpy().astype(np.float64) for i in range(3)]

    # FP64: central differences of the same loss through the oracle
    params = [x.astype(np.float64) for x in (canon, om, th, sg)]
    t64, sens64, meas64 = t.astype(np.float64), sens.astype(np.float64), meas.astype(np.float64)

    def L(ps):
        y_o, _ = oracle.forward(oracle.deform(*ps, t64), sens64, *geom_args)
        return float(np.sum((y_o - meas64) ** 2))

    want = [np.zeros_like(p) for p in params]
    for pi, P in enumerate(params):
        for idx in np.ndindex(P.shape):
            if pi == 0:
                h = 1e-4 * (params[0][3, idx[1]] if idx[0] < 4 else params[0][4, idx[1]])
            elif pi == 1:
                h = 1e-4
            else:
                h = 1e-4 * params[3][idx]

            def fun(dh):
                q = [x.copy() for x in params]
                q[pi][idx] += dh
                return L(q)
            want[pi][idx] = _fd4(fun, h)
    names = ("canon", "omega", "theta", "sigma")
    for g, w, name in zip(got, want, names):
        if name == "canon":
            for ch in range(5):
                assert rel_l2(g[ch], w[ch]) <= GRAD_TOL, (name, ch, rel_l2(g[ch], w[ch]))
        else:
            assert rel_l2(g, w) <= GRAD_TOL, (name, rel_l2(g, w))
