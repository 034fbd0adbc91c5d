"""pa_residual_loss_noalloc: the loss/residual entry point that allocates
nothing, for callers that cannot allocate device memory where they call the
library (a plugin whose host application owns every device allocation, or a
C caller with no allocator at hand that must not call cudaMalloc).

It is compared, through the C ABI, with pa_residual_loss (which takes a
caller-provided workspace) on two calls in a row, since every call reuses
the library's fixed scratch array.  This file is collected last so that a
run stopping at its first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, pred, meas, scale, loss, resid):
    F = pred.shape[0]
    per = pred.numel() // F
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.pa_residual_loss_noalloc(pred.data_ptr(), meas.data_ptr(), per, F, scale.data_ptr(),
                                        loss.data_ptr(), resid.data_ptr(), stream)


def _call_with_workspace(lib, pred, meas, scale, loss, resid):
    F = pred.shape[0]
    per = pred.numel() // F
    need = lib.pa_loss_workspace_size(per, F)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.pa_residual_loss(pred.data_ptr(), meas.data_ptr(), per, F, scale.data_ptr(), loss.data_ptr(),
                                resid.data_ptr(), ws.data_ptr(), ws.numel(), stream)


def test_noalloc_loss_matches_workspace_version_twice():
    import paper_2412_03898_gb300 as pa
    lib = pa._lib.load()
    rng = np.random.default_rng(2024)
    # two different problems in a row, so the second call runs over the
    # partial sums the first one left in the shared array
    for F, S, T in ((5, 37, 1028), (3, 576, 4096)):
        pred = torch.from_numpy(rng.standard_normal((F, S, T)).astype(np.float32)).cuda()
        meas = torch.from_numpy(rng.standard_normal((F, S, T)).astype(np.float32)).cuda()
        scale = torch.from_numpy(rng.uniform(0.5, 2.0, F).astype(np.float32)).cuda()
        loss_a = torch.empty(F, dtype=torch.float64, device="cuda")
        loss_b = torch.empty(F, dtype=torch.float64, device="cuda")
        resid_a = torch.empty_like(pred)
        resid_b = torch.empty_like(pred)
        assert _call_noalloc(lib, pred, meas, scale, loss_a, resid_a) == 0
        assert _call_with_workspace(lib, pred, meas, scale, loss_b, resid_b) == 0
        torch.cuda.synchronize()
        # same kernels, same reduction order: the FP64 losses agree to 1e-12
        # relative (the parity tolerance of the loss is 1e-6), residuals exactly
        np.testing.assert_allclose(loss_a.cpu().numpy(), loss_b.cpu().numpy(), rtol=1e-12)
        assert torch.equal(resid_a, resid_b)
