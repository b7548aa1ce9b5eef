"""The C ABI library loads and exports every function vdf.h declares; host-side
argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def L():
    from paper_1009_0958_gb300 import build, vdf
    build.build()
    return vdf.lib()


@pytest.fixture(scope="module")
def B():
    """Two 1 MiB buffers for calls that must fail their host-side checks.  On a
    machine with a GPU they are device memory, so a check that regressed and
    let a call through would launch on valid memory; without a GPU they are
    host memory (nothing can be launched there)."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        keep = [torch.zeros(1 << 20, dtype=torch.uint8, device="cuda") for _ in range(2)]
        ptrs = [t.data_ptr() for t in keep]
    else:
        keep = [np.zeros(1 << 20, np.uint8) for _ in range(2)]
        ptrs = [a.ctypes.data for a in keep]
    yield [ctypes.c_void_p(v) for v in ptrs]
    del keep


@pytest.fixture(scope="module")
def H():
    """A 1 MiB host buffer (host frame arguments)."""
    import numpy as np
    a = np.zeros(1 << 20, np.uint8)
    yield ctypes.c_void_p(a.ctypes.data)
    del a


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vdf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vdf_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 8
    for n in names:
        assert hasattr(L, n), n


def test_strerror_and_sizes(L):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.vdf_strerror(code)
    assert L.vdf_workspace_bytes(1080, 1920, 0) == 0
    assert L.vdf_workspace_bytes(1080, 1920, 1) >= 4 * 1080 * 1920
    assert L.vdf_workspace_bytes(0, 10, 1) == 0
    assert L.vdf_host_buffer_bytes(10, 10, 1) >= 700


@pytest.mark.parametrize("args", [
    dict(img=None), dict(M=0), dict(N=-1), dict(win=4), dict(win=9), dict(win=1), dict(filter=3), dict(filter=-1),
    dict(filter=1, p=1.5), dict(filter=1, p=-0.1),
    dict(dist=3), dict(dist=1, q=5), dict(precision=2),
])
def test_invalid_arguments_rejected_on_host(L, B, args):
    a = dict(img=B[0], M=8, N=8, win=3, filter=0, p=0.5, dist=0, q=4, precision=0, out=B[1])
    a.update(args)
    rc = L.vdf_filter(a["img"], a["M"], a["N"], a["win"], a["filter"], a["p"], a["dist"], a["q"], a["precision"],
                      a["out"], None, None, None, 0, None)
    assert rc == -1


def test_minkowski_order_checked_on_host(L, B):
    """vdf_filter_lp: orders 1, 2 and infinity (0) only; the DDF at order 1 or
    infinity needs the exact angle; the VMF ignores p and dist_mode."""
    img, out = B

    def call(filter, p, order, dist, precision=0, M=8):
        return L.vdf_filter_lp(img, M, 8, 3, filter, p, order, dist, 4, precision, out, None, None, None, 0, None)
    for order in (3, -1, 4):
        assert call(2, 0.5, order, 0) == -1
    assert call(1, 0.25, 1, 2) == -6                     # DDF, order 1, Method 2
    assert call(1, 0.25, 0, 1) == -6                     # DDF, order infinity, Method 1
    assert call(2, 0.25, 1, 0, M=0) == -1                # sizes still checked
    assert call(2, 7.0, 1, 0, precision=1) == -5         # VMF: p ignored, reaches the workspace check
    assert call(1, 7.0, 1, 0, precision=1) == -1         # DDF: p checked
    f32 = L.vdf_filter_f32(img, 1, 8, 8, 3, 2, 0.5, 0, 4, 0, out, None, None, 0, None)
    assert f32 == -6                                     # no VMF on the float path


def test_acwddf_arguments_checked_on_host(L, B):
    """vdf_filter_acwddf: lambda in [1, d - 2], finite T, the usual checks."""
    img, out = B

    def call(win, lam, T, dist=0, q=4, precision=0):
        return L.vdf_filter_acwddf(img, 8, 8, win, dist, q, lam, T, precision, out, None, None, 0, None)
    assert call(3, 0, 10.8) == -1 and call(3, 4, 10.8) == -1 and call(5, 12, 10.8) == -1
    assert call(3, 2, float("inf")) == -1 and call(3, 2, float("nan")) == -1
    assert call(4, 2, 10.8) == -1 and call(3, 2, 10.8, dist=1, q=5) == -1
    assert call(3, 2, 10.8, precision=1) == -5    # valid, but no workspace
    assert call(7, 2, 10.8) == -6                  # the 7x7 window is not offered for the ACWDDF


def test_window_7_limits_on_host(L, B):
    """The 7x7 window is accepted by the uint8 filters, not by the float path,
    the backward pass, the autotuner or the tuned-shape table."""
    img, out = B
    assert L.vdf_filter(img, 8, 8, 7, 1, 0.25, 0, 4, 1, out, None, None, None, 0, None) == -5   # needs a workspace
    assert L.vdf_filter_f32(img, 1, 8, 8, 7, 1, 0.25, 0, 4, 0, out, None, None, 0, None) == -6
    assert L.vdf_backward_f32(img, img, 1, 8, 8, 7, out, None) == -1
    assert L.vdf_set_tuned_shape(7, 1, 0, 0) == -1 and L.vdf_get_tuned_shape(7, 1, 0) == -1


def test_tuned_shape_table_kinds(L):
    """The DDF 5x5 at p = 1/4 (exact, Method 2) has its own table entry (score
    slots); vdf_set_tuned_shape writes both entries; Method 1, other
    exponents, 3x3 and the BVDF read the raw-slot entry."""
    L.vdf_get_tuned_shape_p.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.vdf_get_tuned_shape_p.restype = ctypes.c_int
    try:
        for dist in (0, 1, 2):
            assert L.vdf_set_tuned_shape(5, 1, dist, 3) == 0
            assert L.vdf_get_tuned_shape(5, 1, dist) == 3
            for p in (0.25, 0.3, 0.5):
                assert L.vdf_get_tuned_shape_p(5, 1, dist, p) == 3
        assert L.vdf_get_tuned_shape_p(7, 1, 0, 0.25) == -1 and L.vdf_get_tuned_shape_p(5, 3, 0, 0.25) == -1
    finally:
        for dist in (0, 1, 2):
            L.vdf_set_tuned_shape(5, 1, dist, 0)


def test_autotune_acwddf_argument_checks(L, B):
    """Rejected before any launch: a null image, a missing workspace, a bad
    smoothing level."""
    P = ctypes.c_void_p
    L.vdf_autotune_acwddf.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_double, P, P, P, ctypes.c_size_t, ctypes.c_int, P, P, P]
    L.vdf_autotune_acwddf.restype = ctypes.c_int
    img, out = B
    assert L.vdf_autotune_acwddf(None, 8, 8, 3, 0, 4, 2, 10.8, out, None, None, 0, 1, None, None, None) == -1
    assert L.vdf_autotune_acwddf(img, 8, 8, 3, 0, 4, 2, 10.8, out, None, None, 0, 1, None, None, None) == -5


def test_aliasing_and_workspace_checks(L, B):
    p = B[0]
    assert L.vdf_filter(p, 8, 8, 3, 0, 0.5, 0, 4, 0, p, None, None, None, 0, None) == -1      # out == img
    assert L.vdf_filter(p, 8, 8, 3, 0, 0.5, 0, 4, 1, B[1], None, None, None, 0, None) == -5


def test_debug_terms_arguments_checked_on_host(L, B):
    p = B[0]
    assert L.vdf_debug_fp32_terms(None, 4, 0, 4, None, None, None) == -1
    assert L.vdf_debug_fp32_terms(p, -1, 0, 4, None, None, None) == -1
    assert L.vdf_debug_fp32_terms(p, 4, 3, 4, None, None, None) == -1
    assert L.vdf_debug_fp32_terms(p, 4, 1, 5, None, None, None) == -1
    assert L.vdf_debug_fp32_terms(p, 0, 0, 4, None, None, None) == 0    # nothing to launch


def test_host_frames_arguments_checked_on_host(L, B, H):
    p = B[0]
    arr = (ctypes.c_void_p * 1)(H)
    nul = (ctypes.c_void_p * 1)(None)
    assert L.vdf_filter_host_frames(None, arr, None, 1, 8, 8, 3, 0, 0.5, 0, 4, 1, p, 1 << 20, None) == -1
    assert L.vdf_filter_host_frames(arr, nul, None, 1, 8, 8, 3, 0, 0.5, 0, 4, 1, p, 1 << 20, None) == -1
    assert L.vdf_filter_host_frames(arr, arr, None, -1, 8, 8, 3, 0, 0.5, 0, 4, 1, p, 1 << 20, None) == -1
    assert L.vdf_filter_host_frames(arr, arr, None, 1, 0, 8, 3, 0, 0.5, 0, 4, 1, p, 1 << 20, None) == -1
    assert L.vdf_filter_host_frames(arr, arr, None, 1, 8, 8, 3, 0, 0.5, 0, 4, 1, p, 16, None) == -5
    assert L.vdf_filter_host_frames(arr, arr, None, 0, 8, 8, 3, 0, 0.5, 0, 4, 1, None, 0, None) == 0
    one = L.vdf_host_buffer_bytes(8, 8, 1)
    assert L.vdf_host_frames_buffer_bytes(8, 8, 1) == 3 * ((one + 255) // 256 * 256)


def test_float_debug_entries_checked_on_host(L, B):
    assert L.vdf_debug_fp32_terms_f32(None, 4, None, None, None) == -1
    assert L.vdf_debug_fp32_terms_f32(B[0], -1, None, None, None) == -1
    assert L.vdf_debug_sqrt_error(None, None) == -1


def test_plan_host_logic(L):
    """vdf_plan_create validates descriptors and sizes the workspace on the
    host: counters (256 B), descriptors (56 B each, 16-byte rounded), one int
    per work item (tiles of the tuned shape, 32x16 by default) and one
    recheck entry (8 B) per pixel.  No device memory is touched."""
    from paper_1009_0958_gb300 import vdf
    P = ctypes.c_void_p
    L.vdf_plan_create.argtypes = [ctypes.POINTER(P), P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.vdf_plan_create.restype = ctypes.c_int
    L.vdf_plan_workspace_bytes.argtypes, L.vdf_plan_workspace_bytes.restype = [P], ctypes.c_size_t
    L.vdf_plan_set_persistent.argtypes, L.vdf_plan_set_persistent.restype = [P, ctypes.c_int], ctypes.c_int
    L.vdf_plan_destroy.argtypes, L.vdf_plan_destroy.restype = [P], None
    for win in (3, 5):
        for f in (0, 1):
            assert L.vdf_set_tuned_shape(win, f, 0, 0) == 0
    dims = [(40, 70, 3, 0), (1, 1, 5, 1), (100, 33, 5, 0), (17, 200, 3, 1), (64, 64, 5, 1)]

    def descs(items, base=0x100000):
        arr = (vdf.ImageDesc * len(items))()
        for k, (M, N, win, f) in enumerate(items):
            a = base + k * (1 << 24)
            arr[k] = vdf.ImageDesc(a, a + (1 << 23), 0, M, N, win, f, 0.25)
        return arr

    h = P()
    arr = descs(dims)
    assert L.vdf_plan_create(ctypes.byref(h), ctypes.cast(arr, P), len(dims), 0, 4) == 0
    tiles = sum(-(-M // 16) * -(-N // 32) for M, N, _, _ in dims)
    pixels = sum(M * N for M, N, _, _ in dims)
    up16 = lambda v: (v + 15) // 16 * 16
    assert L.vdf_plan_workspace_bytes(h) == 256 + up16(56 * len(dims)) + up16(4 * tiles) + 8 * pixels
    assert L.vdf_plan_set_persistent(h, 1) == 0 and L.vdf_plan_set_persistent(h, 0) == 0
    L.vdf_plan_destroy(h)
    bad = [[(0, 5, 3, 0)], [(5, 5, 4, 0)], [(5, 5, 3, 2)], [(5, 5, 3, 7)]]
    for items in bad:
        h = P()
        assert L.vdf_plan_create(ctypes.byref(h), ctypes.cast(descs(items), P), 1, 0, 4) == -1
    h = P()
    assert L.vdf_plan_create(ctypes.byref(h), ctypes.cast(descs(dims[:1]), P), 1, 1, 5) == -1   # Method 1 needs q in 2..4
    assert L.vdf_plan_create(ctypes.byref(h), ctypes.cast(descs(dims[:1]), P), 1, 3, 4) == -1   # no such mode
    for dist in (1, 2):                                                                            # Methods 1 and 2
        h2 = P()
        assert L.vdf_plan_create(ctypes.byref(h2), ctypes.cast(descs(dims[:1]), P), 1, dist, 4) == 0
        L.vdf_plan_destroy(h2)
    assert L.vdf_plan_create(ctypes.byref(h), None, 1, 0, 4) == -1
    over = (vdf.ImageDesc * 1)()
    over[0] = vdf.ImageDesc(0x100000, 0x100010, 0, 8, 8, 3, 0, 0.5)   # out overlaps img
    assert L.vdf_plan_create(ctypes.byref(h), ctypes.cast(over, P), 1, 0, 4) == -1
