"""vdf_filter_noalloc: the allocation-free entry point.

It serves callers that cannot allocate device memory: its scratch lives in a
fixed device array inside the library instead of a caller workspace.  Its
output must equal vdf_filter's FP32 path bit for bit, on consecutive calls
(the shared array keeps the previous call's contents), and images above its
2^21-pixel capacity must be refused before anything is launched.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0958_gb300 import build, vdf
    build.build()
    return vdf


@pytest.mark.parametrize("win,filter,p", [(5, "ddf", 0.25), (3, "bvdf", 0.5)])
def test_noalloc_equals_workspace_path_on_consecutive_calls(V, win, filter, p):
    from paper_1009_0958_gb300 import synth
    imgs = [synth.make_image(512, 640, 31, 0.20, rectangles=12)[1], synth.make_image(1080, 1920, 32, 0.10, rectangles=12)[1]]
    for img in imgs:                      # two calls in a row through the same static scratch
        x = torch.from_numpy(img).cuda()
        ws = V.alloc_workspace(*img.shape[:2], "fp32")
        o_ref, i_ref = V.filter(x, win, filter, p, "exact", 4, precision="fp32", workspace=ws)
        o, i = V.filter_noalloc(x, win, filter, p, "exact", 4)
        torch.cuda.synchronize()
        assert V.workspace_stats(ws)[0] > 0     # the case exercises the recheck list
        assert torch.equal(o, o_ref) and torch.equal(i, i_ref)


def test_noalloc_rejects_images_above_capacity(V):
    """An image one row above the limit gets VDF_E_WORKSPACE.  Its buffers are
    real device memory of the full size, so even a size check that regressed
    would filter valid memory instead of faulting."""
    M, N = 2049, 1024
    assert V.NOALLOC_MAX_PIXELS < M * N
    L = V.lib()
    V.filter_noalloc(torch.zeros((4, 4, 3), dtype=torch.uint8, device="cuda"))   # sets argtypes
    img = torch.zeros((M, N, 3), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(img)
    idx = torch.empty((M, N), dtype=torch.int8, device="cuda")
    rc = L.vdf_filter_noalloc(ctypes.c_void_p(img.data_ptr()), M, N, 3, 0, 0.5, 0, 4, ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(idx.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == -5
    # argument errors come before the size check
    rc = L.vdf_filter_noalloc(None, M, N, 3, 0, 0.5, 0, 4, ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == -1
