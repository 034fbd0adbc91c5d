"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point include/pa.h declares, and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pa.h")).read()
    return sorted(set(re.findall(r"PA_API\s+[\w\s\*]*?\b(pa_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_03898_gb300 import build
    build.build()
    from paper_2412_03898_gb300 import _lib
    return _lib.load()


def test_header_declares_the_hot_path():
    names = _declared()
    for must in ("pa_deform_balls", "pa_forward", "pa_adjoint", "pa_residual_loss"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_2412_03898_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()


def test_status_strings_and_version(lib):
    assert lib.pa_version() >= 100
    assert b"INVALID" in lib.pa_status_string(1)
    assert b"DOMAIN" in lib.pa_status_string(2)


def test_invalid_geometry_rejected_on_host(lib):
    from paper_2412_03898_gb300 import _lib
    g = _lib.pa_geom(None, 4, 4, 1.5, 40.0, 0.0, 64, 5.0)  # NULL sensors
    b = _lib.pa_balls(None, 0, 0)
    assert lib.pa_forward(ctypes.byref(g), ctypes.byref(b), 1, None, 0, None, 0, None) == _lib.PA_ERR_INVALID_ARG
    g2 = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 62, 5.0)  # T % 4 != 0 (pointer never dereferenced)
    assert lib.pa_forward(ctypes.byref(g2), ctypes.byref(b), 1, None, 0, None, 0, None) == _lib.PA_ERR_INVALID_ARG
    g3 = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 64, 9.0)  # kappa out of range
    assert lib.pa_forward(ctypes.byref(g3), ctypes.byref(b), 1, None, 0, None, 0, None) == _lib.PA_ERR_INVALID_ARG
    b2 = _lib.pa_balls(16, 10, 10)  # stride not a multiple of 4
    g4 = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 64, 5.0)
    assert lib.pa_forward(ctypes.byref(g4), ctypes.byref(b2), 1, None, 0, None, 0, None) == _lib.PA_ERR_INVALID_ARG


def test_invalid_loss_and_adam_args_rejected_on_host(lib):
    from paper_2412_03898_gb300 import _lib
    assert lib.pa_residual_loss(None, None, 6, 1, None, None, None, None, 0, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_adam_step(None, None, None, None, 8, 1e-3, 0.9, 0.999, 1e-8, 0, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_loss_workspace_size(0, 1) == 0


def test_imaging_and_chain_rule_args_rejected_on_host(lib):
    from paper_2412_03898_gb300 import _lib
    E = _lib.PA_ERR_INVALID_ARG
    P = ctypes.c_void_p
    fake = P(256)  # never dereferenced: every call below fails its host-side checks first
    # pa_ubp_filter: fewer than 2 samples, aliasing, non-positive fs
    assert lib.pa_ubp_filter(fake, 3, 1, 40.0, 0.0, P(512), None) == E
    assert lib.pa_ubp_filter(fake, 3, 64, 40.0, 0.0, fake, None) == E
    assert lib.pa_ubp_filter(fake, 3, 64, 0.0, 0.0, P(512), None) == E
    # pa_ubp / pa_splat / pa_map: bad grids, NULL buffers, non-positive kappa
    g = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 64, 5.0)
    good = _lib.pa_grid((ctypes.c_float * 3)(0, 0, 0), 0.5, 4, 4, 4)
    flat = _lib.pa_grid((ctypes.c_float * 3)(0, 0, 0), 0.0, 4, 4, 4)
    empty = _lib.pa_grid((ctypes.c_float * 3)(0, 0, 0), 0.5, 0, 4, 4)
    c3 = (ctypes.c_float * 3)(0, 0, 0)
    assert lib.pa_ubp(ctypes.byref(g), c3, fake, ctypes.byref(flat), fake, None) == E
    assert lib.pa_ubp(ctypes.byref(g), None, fake, ctypes.byref(good), fake, None) == E
    assert lib.pa_ubp(ctypes.byref(g), c3, None, ctypes.byref(good), fake, None) == E
    b = _lib.pa_balls(16, 4, 4)
    assert lib.pa_splat(ctypes.byref(b), 0.0, ctypes.byref(good), fake, None) == E
    assert lib.pa_splat(ctypes.byref(b), 5.0, ctypes.byref(empty), fake, None) == E
    assert lib.pa_map(None, ctypes.byref(good), fake, fake, fake, None) == E
    assert lib.pa_map(fake, ctypes.byref(flat), fake, fake, fake, None) == E
    # pa_ssim: images smaller than the window, unknown flags
    assert lib.pa_ssim_workspace_size(10, 80) == 0
    assert lib.pa_ssim(fake, fake, 10, 80, 1.0, 0, None, fake, fake, 4096, None) == E
    assert lib.pa_ssim(fake, fake, 64, 80, 1.0, 1 << 7, None, fake, fake, 4096, None) == E
    assert lib.pa_ssim(fake, fake, 64, 80, 0.0, 0, None, fake, fake, 4096, None) == E
    # pa_deform_backward: n_basis outside [1, 128], NULL gradient outputs, unknown flags
    canon = _lib.pa_canon(16, 16, 16, 16, 4, 4, 129)
    gr = _lib.pa_grads(16, 16, 16, 16)
    assert lib.pa_deform_backward(ctypes.byref(canon), fake, 2, fake, ctypes.byref(gr), 0, None) == E
    canon = _lib.pa_canon(16, 16, 16, 16, 4, 4, 65)
    null_gr = _lib.pa_grads(16, None, 16, 16)
    assert lib.pa_deform_backward(ctypes.byref(canon), fake, 2, fake, ctypes.byref(null_gr), 0, None) == E
    assert lib.pa_deform_backward(ctypes.byref(canon), fake, 2, fake, ctypes.byref(gr), 1 << 5, None) == E


def test_invalid_tile_plans_rejected_on_host(lib):
    from paper_2412_03898_gb300 import _lib
    g = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 64, 5.0)  # pointers never dereferenced
    b = _lib.pa_balls(16, 10, 12)
    out7 = (ctypes.c_int32 * 7)()
    for bad in ((17, 0, 0, 0, 0), (16, 6, 0, 0, 0), (16, 0, 8196, 0, 0), (16, 0, 6, 0, 0), (16, 0, 0, -1, 0),
                (16, 0, 0, 0, 17), (-1, 0, 0, 0, 0)):
        t = (ctypes.c_int32 * 5)(*bad)
        assert lib.pa_forward_plan_info(ctypes.byref(g), ctypes.byref(b), 1, t, out7) == _lib.PA_ERR_INVALID_ARG, bad
        assert lib.pa_forward_workspace_size_ex(ctypes.byref(g), ctypes.byref(b), 1, t) == 0, bad
        assert lib.pa_forward_ex(ctypes.byref(g), ctypes.byref(b), 1, None, 0, t, None, 0, None) == \
            _lib.PA_ERR_INVALID_ARG, bad


def test_plan_values_round_trip_and_checks_on_host(lib):
    """pa_plan_from_values / pa_plan_get / pa_plan_destroy need no device; bad
    values are rejected and leave *out NULL."""
    from paper_2412_03898_gb300 import _lib
    h = ctypes.c_void_p()
    v = (ctypes.c_int32 * 7)(12, 2048, 256, 3, 8, 4, 16)
    assert lib.pa_plan_from_values(v, ctypes.byref(h)) == _lib.PA_OK and h.value
    out = (ctypes.c_int32 * 7)()
    ms = (ctypes.c_float * 2)(9.0, 9.0)
    assert lib.pa_plan_get(h, out, ms) == _lib.PA_OK
    assert list(out) == [12, 2048, 256, 3, 8, 4, 16] and list(ms) == [0.0, 0.0]
    lib.pa_plan_destroy(h)
    lib.pa_plan_destroy(None)
    for bad in ((17, 0, 0, 0, 0, 0, 0), (0, 6, 0, 0, 0, 0, 0), (0, 0, 0, 0, 0, -1, 0), (0, 0, 0, 0, 0, 0, 2000)):
        h = ctypes.c_void_p(1234)
        assert lib.pa_plan_from_values((ctypes.c_int32 * 7)(*bad), ctypes.byref(h)) == _lib.PA_ERR_INVALID_ARG
        assert not h.value
    assert lib.pa_plan_from_values(None, None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_plan_get(None, out, None) == _lib.PA_ERR_INVALID_ARG
    # the heuristic plan of a valid scene list launches nothing (no device needed)
    g = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 64, 5.0)
    sc = (_lib.pa_scene * 1)(_lib.pa_scene(g, _lib.pa_balls(16, 10, 12), 1, 16, None, None))
    h = ctypes.c_void_p()
    assert lib.pa_plan_create(sc, 1, 0, None, 0, None, ctypes.byref(h)) == _lib.PA_OK and h.value
    lib.pa_plan_destroy(h)
    assert lib.pa_plan_create(sc, 0, 0, None, 0, None, ctypes.byref(h)) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_plan_create(sc, 1, 1 << 6, None, 0, None, ctypes.byref(h)) == _lib.PA_ERR_INVALID_ARG
    badg = (_lib.pa_scene * 1)(_lib.pa_scene(_lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 62, 5.0),
                                             _lib.pa_balls(16, 10, 12), 1, 16, None, None))
    assert lib.pa_plan_create(badg, 1, 0, None, 0, None, ctypes.byref(h)) == _lib.PA_ERR_INVALID_ARG


def test_4d_calls_and_probe_reject_bad_args_on_host(lib):
    from paper_2412_03898_gb300 import _lib
    E = _lib.PA_ERR_INVALID_ARG
    P = ctypes.c_void_p
    fake = P(256)  # never dereferenced: every call below fails its host-side checks first
    g = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 64, 5.0)
    good = _lib.pa_canon(16, 16, 16, 16, 4, 4, 3)
    bad_nb = _lib.pa_canon(16, 16, 16, 16, 4, 4, 0)
    bad_stride = _lib.pa_canon(16, 16, 16, 16, 6, 6, 3)
    gr = _lib.pa_grads(16, 16, 16, 16)
    null_gr = _lib.pa_grads(16, 16, None, 16)
    assert lib.pa_forward_4d(None, ctypes.byref(good), fake, 2, fake, 0, None, fake, 4096, None) == E
    assert lib.pa_forward_4d(ctypes.byref(g), ctypes.byref(bad_nb), fake, 2, fake, 0, None, fake, 4096, None) == E
    assert lib.pa_forward_4d(ctypes.byref(g), ctypes.byref(bad_stride), fake, 2, fake, 0, None, fake, 4096,
                             None) == E
    assert lib.pa_forward_4d(ctypes.byref(g), ctypes.byref(good), fake, 2, fake, 1 << 4, None, fake, 4096,
                             None) == E
    assert lib.pa_forward_4d(ctypes.byref(g), ctypes.byref(good), fake, 2, P(258), 0, None, fake, 4096, None) == E
    assert lib.pa_forward_4d(ctypes.byref(g), ctypes.byref(good), None, 2, fake, 0, None, fake, 4096, None) == E
    assert lib.pa_adjoint_4d(ctypes.byref(g), ctypes.byref(good), fake, 2, fake, None, None, 0, None, fake, 4096,
                             None) == E
    assert lib.pa_adjoint_4d(ctypes.byref(g), ctypes.byref(good), fake, 2, fake, None, ctypes.byref(null_gr), 0,
                             None, fake, 4096, None) == E
    assert lib.pa_adjoint_4d(ctypes.byref(g), ctypes.byref(good), fake, 2, P(260), None, ctypes.byref(gr), 0,
                             None, fake, 4096, None) == E
    assert lib.pa_adjoint_4d(ctypes.byref(g), ctypes.byref(good), fake, 2, fake, None, ctypes.byref(gr), 1 << 3,
                             None, fake, 4096, None) == E
    assert lib.pa_forward_4d_workspace_size(ctypes.byref(g), ctypes.byref(bad_nb), 2, None) == 0
    assert lib.pa_adjoint_4d_workspace_size(None, ctypes.byref(good), 2, None) == 0
    # work-queue counter (256) + one frame of states and one of gradients
    # (5 x stride 4 floats, rounded up to 256 bytes each)
    assert lib.pa_adjoint_4d_workspace_size(ctypes.byref(g), ctypes.byref(good), 2, None) == 256 + 2 * 256
    assert lib.pa_measure_unit_rates(None, None) == E


def test_spatial_order_and_gather_args_checked_on_host(lib):
    from paper_2412_03898_gb300 import _lib
    E, W = _lib.PA_ERR_INVALID_ARG, _lib.PA_ERR_WORKSPACE
    P = ctypes.c_void_p
    fake = P(256)  # never dereferenced: every call below fails its host-side checks first
    b = _lib.pa_balls(16, 1000, 1000)
    assert lib.pa_spatial_order(None, fake, fake, 1 << 20, None) == E
    assert lib.pa_spatial_order(ctypes.byref(_lib.pa_balls(16, 1000, 998)), fake, fake, 1 << 20, None) == E
    assert lib.pa_spatial_order(ctypes.byref(b), None, fake, 1 << 20, None) == E
    assert lib.pa_spatial_order(ctypes.byref(b), fake, fake, 16, None) == W
    assert lib.pa_spatial_order(ctypes.byref(b), fake, P(256 + 16), 1 << 20, None) == W
    assert lib.pa_spatial_order_workspace_size(0) == 0
    assert lib.pa_spatial_order_workspace_size(1000) > 16 * 1000
    assert lib.pa_gather_rows(fake, P(512), 10, 8, 5, fake, None) == E  # stride < n
    assert lib.pa_gather_rows(fake, fake, 10, 12, 5, fake, None) == E   # in == out
    assert lib.pa_gather_rows(None, P(512), 10, 12, 5, fake, None) == E


def test_adjoint_workspace_checked_on_host(lib):
    from paper_2412_03898_gb300 import _lib
    W = _lib.PA_ERR_WORKSPACE
    P = ctypes.c_void_p
    fake = P(256)  # never dereferenced: the workspace check fails first
    g = _lib.pa_geom(16, 4, 4, 1.5, 40.0, 0.0, 64, 5.0)
    b = _lib.pa_balls(16, 4, 4)
    gr = _lib.pa_grads(16, None, None, None)
    args = (ctypes.byref(g), ctypes.byref(b), None, None, 1, fake, None, ctypes.byref(gr), 0)
    assert lib.pa_adjoint(*args, P(256 + 16), 256, None) == W  # not 256-byte aligned
    assert lib.pa_adjoint(*args, fake, 128, None) == W  # smaller than PA_ADJOINT_WORKSPACE_BYTES
    hdr = open(os.path.join(ROOT, "include", "pa.h")).read()
    assert int(re.search(r"#define PA_ADJOINT_WORKSPACE_BYTES (\d+)u", hdr).group(1)) == _lib.PA_ADJOINT_WORKSPACE_BYTES


def test_noalloc_loss_rejects_problems_beyond_its_scratch_on_host(lib):
    """pa_residual_loss_noalloc checks its fixed scratch's capacity on the host
    before anything else touches the device: 17 frames of 1024 blocks need
    17408 partials, more than the 16384 it holds.  The pointers are never
    dereferenced, and this runs where no GPU is visible, so a regression of
    the check fails the test instead of launching anything."""
    from paper_2412_03898_gb300 import _lib
    fake = ctypes.c_void_p(256)
    assert lib.pa_residual_loss_noalloc(fake, fake, 1024 * 32768, 17, None, fake, None, None) == \
        _lib.PA_ERR_WORKSPACE
    # 16384 single-block frames fit; 16385 do not (checked before the device is asked for the scratch)
    assert lib.pa_residual_loss_noalloc(fake, fake, 4, 16385, None, fake, None, None) == _lib.PA_ERR_WORKSPACE
