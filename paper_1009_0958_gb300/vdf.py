"""ctypes binding of libvdf (C ABI in include/vdf.h).

Argument marshalling only: tensors are passed as raw device pointers with
their sizes, the stream is torch's current CUDA stream, and every step of the
filter runs in the library's CUDA kernels.  There is no CPU fallback: if the
library or a GPU is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

FILTERS = {"bvdf": 0, "ddf": 1, "vmf": 2}
# Minkowski order of the distance term (Eq. (1)): 1, 2, or "inf"
ORDERS = {1: 1, 2: 2, "inf": 0}
DISTS = {"exact": 0, "minimax": 1, "rgb": 2}
PRECISIONS = {"fp64": 0, "fp32": 1}

_lock = threading.Lock()
_lib = None


class VdfError(RuntimeError):
    pass


def lib():
    """Load libvdf.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise VdfError(f"libvdf.so not built ({_build.LIB}); run paper_1009_0958_gb300.build.build()")
            L = ctypes.CDLL(_build.LIB)
            P, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
            L.vdf_strerror.argtypes, L.vdf_strerror.restype = [i], ctypes.c_char_p
            L.vdf_last_cuda_error.argtypes, L.vdf_last_cuda_error.restype = [], ctypes.c_char_p
            L.vdf_workspace_bytes.argtypes, L.vdf_workspace_bytes.restype = [i, i, i], sz
            L.vdf_host_buffer_bytes.argtypes, L.vdf_host_buffer_bytes.restype = [i, i, i], sz
            L.vdf_filter.argtypes = [P, i, i, i, i, d, i, i, i, P, P, P, P, sz, P]
            L.vdf_filter_lp.argtypes = [P, i, i, i, i, d, i, i, i, i, P, P, P, P, sz, P]
            L.vdf_filter_acwddf.argtypes = [P, i, i, i, i, i, i, d, i, P, P, P, sz, P]
            L.vdf_filter_host.argtypes = [P, i, i, i, i, d, i, i, i, P, P, P, sz, P]
            L.vdf_filter_f32.argtypes = [P, i, i, i, i, i, d, i, i, i, P, P, P, sz, P]
            L.vdf_backward_f32.argtypes = [P, P, i, i, i, i, P, P]
            L.vdf_fp32_pass.argtypes = [P, i, i, i, i, d, i, i, P, P, P, sz, P]
            L.vdf_fp64_recheck.argtypes = [P, i, i, i, i, d, i, i, P, P, P, sz, P]
            L.vdf_workspace_stats.argtypes = [P, P, P, P]
            L.vdf_read_stats.argtypes = [P, P, P]
            L.vdf_debug_fp32_scores.argtypes = [P, i, i, i, i, d, i, i, P, P]
            L.vdf_debug_fp32_terms.argtypes = [P, i, i, i, P, P, P]
            L.vdf_debug_fp32_terms_f32.argtypes = [P, i, P, P, P]
            L.vdf_debug_sqrt_error.argtypes = [P, P]
            L.vdf_host_frames_buffer_bytes.argtypes, L.vdf_host_frames_buffer_bytes.restype = [i, i, i], sz
            L.vdf_filter_host_frames.argtypes = [P, P, P, i, i, i, i, i, d, i, i, i, P, sz, P]
            for f in ("vdf_filter", "vdf_filter_lp", "vdf_filter_acwddf", "vdf_filter_host", "vdf_workspace_stats", "vdf_debug_fp32_scores",
                      "vdf_debug_fp32_terms", "vdf_filter_host_frames", "vdf_debug_fp32_terms_f32",
                      "vdf_debug_sqrt_error",
                      "vdf_fp32_pass", "vdf_fp64_recheck", "vdf_filter_f32", "vdf_backward_f32"):
                getattr(L, f).restype = i
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        L = lib()
        msg = L.vdf_strerror(rc).decode()
        if rc == -2:
            msg += ": " + L.vdf_last_cuda_error().decode()
        raise VdfError(f"libvdf error {rc}: {msg}")


def _code(table, v):
    return table[v] if isinstance(v, str) else int(v)


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def workspace_bytes(M: int, N: int, precision="fp32") -> int:
    return int(lib().vdf_workspace_bytes(M, N, _code(PRECISIONS, precision)))


def alloc_workspace(M: int, N: int, precision="fp32", device=None) -> torch.Tensor | None:
    n = workspace_bytes(M, N, precision)
    if n == 0:
        return None
    return torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")


def _aligned(ws: torch.Tensor | None):
    if ws is None:
        return None, 0
    p = ws.data_ptr()
    off = (-p) % 256
    return ctypes.c_void_p(p + off), ws.numel() - off


def filter(img: torch.Tensor, win: int = 3, filter="bvdf", p: float = 0.5, dist="exact", q: int = 4,
           precision="fp32", out: torch.Tensor | None = None, index: torch.Tensor | None = None,
           want_index: bool = True, agg: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
           stream=None, order=2):
    """Filter an M x N x 3 uint8 CUDA image.  Returns ``(out, index)``.

    ``filter``: "bvdf", "ddf" or "vmf"; ``order``: Minkowski order of the
    distance term of the DDF and the VMF (1, 2 or "inf")."""
    if not (img.is_cuda and img.dtype == torch.uint8 and img.dim() == 3 and img.shape[2] == 3):
        raise VdfError("img must be a CUDA uint8 tensor of shape (M, N, 3)")
    img = img.contiguous()
    M, N = int(img.shape[0]), int(img.shape[1])
    if out is None:
        out = torch.empty_like(img)
    if index is None and want_index:
        index = torch.empty((M, N), dtype=torch.int8, device=img.device)
    prec = _code(PRECISIONS, precision)
    if workspace is None:
        workspace = alloc_workspace(M, N, prec, img.device)
    wp, wn = _aligned(workspace)
    if order not in ORDERS:
        raise VdfError("order must be 1, 2 or 'inf'")
    _check(lib().vdf_filter_lp(_ptr(img), M, N, win, _code(FILTERS, filter), float(p), ORDERS[order],
                               _code(DISTS, dist), q, prec, _ptr(out), _ptr(index), _ptr(agg), wp, wn,
                               _stream(stream)))
    return out, index


def filter_acwddf(img: torch.Tensor, win: int = 3, dist="exact", q: int = 4, lam: int = 2, T: float = 10.8,
                  precision="fp32", out: torch.Tensor | None = None, index: torch.Tensor | None = None,
                  want_index: bool = True, workspace: torch.Tensor | None = None, stream=None):
    """ACWDDF (Eq. (9)) of an M x N x 3 uint8 CUDA image: the DDF output
    where the centre-weighted VMF levels lam .. lam+2 differ enough from the
    centre (switching sum above T), else the centre.  Returns ``(out, index)``."""
    if not (img.is_cuda and img.dtype == torch.uint8 and img.dim() == 3 and img.shape[2] == 3):
        raise VdfError("img must be a CUDA uint8 tensor of shape (M, N, 3)")
    img = img.contiguous()
    M, N = int(img.shape[0]), int(img.shape[1])
    if out is None:
        out = torch.empty_like(img)
    if index is None and want_index:
        index = torch.empty((M, N), dtype=torch.int8, device=img.device)
    prec = _code(PRECISIONS, precision)
    if workspace is None:
        workspace = alloc_workspace(M, N, prec, img.device)
    wp, wn = _aligned(workspace)
    _check(lib().vdf_filter_acwddf(_ptr(img), M, N, win, _code(DISTS, dist), q, int(lam), float(T), prec, _ptr(out),
                                   _ptr(index), wp, wn, _stream(stream)))
    return out, index


def workspace_stats(workspace: torch.Tensor, stream=None):
    """(pixels rechecked in FP64, overflow flag) of the last call using it."""
    r = ctypes.c_int64(0)
    o = ctypes.c_int32(0)
    wp, _ = _aligned(workspace)
    _check(lib().vdf_workspace_stats(wp, ctypes.byref(r), ctypes.byref(o), _stream(stream)))
    return int(r.value), int(o.value)


class Stats(ctypes.Structure):
    """vdf_stats of vdf.h."""
    _fields_ = [("rechecked", ctypes.c_int64), ("structural_ties", ctypes.c_int64), ("overflow", ctypes.c_int32)]


def read_stats(workspace: torch.Tensor, stream=None) -> dict:
    """Counters of the last FP32 call using ``workspace``: pixels rechecked in
    FP64, pixels settled as structural ties, overflow flag."""
    st = Stats()
    wp, _ = _aligned(workspace)
    _check(lib().vdf_read_stats(wp, ctypes.byref(st), _stream(stream)))
    return {"rechecked": int(st.rechecked), "structural_ties": int(st.structural_ties), "overflow": int(st.overflow)}


def host_buffer_bytes(M: int, N: int, precision="fp32") -> int:
    return int(lib().vdf_host_buffer_bytes(M, N, _code(PRECISIONS, precision)))


def filter_host(img_host: torch.Tensor, win=3, filter="bvdf", p=0.5, dist="exact", q=4, precision="fp32",
                out_host: torch.Tensor | None = None, index_host: torch.Tensor | None = None,
                dev_buffer: torch.Tensor | None = None, stream=None):
    """Filter a host (ideally pinned) uint8 M x N x 3 image end to end: the
    library copies it in, filters and copies the result back, then waits."""
    M, N = int(img_host.shape[0]), int(img_host.shape[1])
    prec = _code(PRECISIONS, precision)
    if out_host is None:
        out_host = torch.empty_like(img_host)
    if dev_buffer is None:
        dev_buffer = torch.empty(host_buffer_bytes(M, N, prec) + 256, dtype=torch.uint8, device="cuda")
    bp, bn = _aligned(dev_buffer)
    _check(lib().vdf_filter_host(_ptr(img_host), M, N, win, _code(FILTERS, filter), float(p), _code(DISTS, dist), q,
                                 prec, _ptr(out_host), _ptr(index_host), bp, bn, _stream(stream)))
    return out_host, index_host


def host_frames_buffer_bytes(M: int, N: int, precision="fp32") -> int:
    return int(lib().vdf_host_frames_buffer_bytes(M, N, _code(PRECISIONS, precision)))


def filter_host_frames(frames, win=5, filter="ddf", p=0.25, dist="exact", q=4, precision="fp32", outs=None,
                       indices=None, dev_buffer: torch.Tensor | None = None, stream=None):
    """Filter a list of M x N x 3 uint8 host tensors (pinned for overlap)
    with the copies of each frame overlapping the filtering of the others.
    Returns ``(outs, indices)`` as lists of host tensors."""
    if not frames:
        return [], []
    M, N = int(frames[0].shape[0]), int(frames[0].shape[1])
    for f in frames:
        if f.is_cuda or f.dtype != torch.uint8 or tuple(f.shape) != (M, N, 3) or not f.is_contiguous():
            raise VdfError("frames must be contiguous host uint8 tensors of one shape (M, N, 3)")
    n = len(frames)
    if outs is None:
        outs = [torch.empty((M, N, 3), dtype=torch.uint8).pin_memory() for _ in range(n)]
    if indices is None:
        indices = [torch.empty((M, N), dtype=torch.int8).pin_memory() for _ in range(n)]
    prec = _code(PRECISIONS, precision)
    need = int(lib().vdf_host_frames_buffer_bytes(M, N, prec))
    if dev_buffer is None:
        dev_buffer = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    bp, bn = _aligned(dev_buffer)
    P = ctypes.c_void_p
    ins = (P * n)(*[f.data_ptr() for f in frames])
    ous = (P * n)(*[o.data_ptr() for o in outs])
    ixs = (P * n)(*[(x.data_ptr() if x is not None else None) for x in indices])
    _check(lib().vdf_filter_host_frames(ins, ous, ixs, n, M, N, win, _code(FILTERS, filter), float(p),
                                        _code(DISTS, dist), q, prec, bp, bn, _stream(stream)))
    return outs, indices


def debug_fp32_scores(img: torch.Tensor, win=3, filter="bvdf", p=0.5, dist="exact", q=4, stream=None):
    """Per-member FP32 scores and certified bounds, shape (M, N, n, 2)."""
    M, N = int(img.shape[0]), int(img.shape[1])
    fe = torch.full((M, N, win * win, 2), float("nan"), dtype=torch.float32, device=img.device)
    _check(lib().vdf_debug_fp32_scores(_ptr(img.contiguous()), M, N, win, _code(FILTERS, filter), float(p),
                                       _code(DISTS, dist), q, _ptr(fe), _stream(stream)))
    return fe


def debug_fp32_terms(pairs: torch.Tensor, dist="exact", q=4, stream=None):
    """FP32 pair terms of the tile kernel for an (n, 6) int32 CUDA tensor of
    pixel pairs (R, G, B of x then y).  Returns ``(angle, l2)`` float32."""
    if not (pairs.is_cuda and pairs.dtype == torch.int32 and pairs.dim() == 2 and pairs.shape[1] == 6):
        raise VdfError("pairs must be a CUDA int32 tensor of shape (n, 6)")
    pairs = pairs.contiguous()
    n = int(pairs.shape[0])
    ang = torch.empty(n, dtype=torch.float32, device=pairs.device)
    l2 = torch.empty(n, dtype=torch.float32, device=pairs.device)
    _check(lib().vdf_debug_fp32_terms(_ptr(pairs), n, _code(DISTS, dist), q, _ptr(ang), _ptr(l2), _stream(stream)))
    return ang, l2


def debug_fp32_terms_f32(pairs: torch.Tensor, stream=None):
    """FP32 terms of the float-input tile kernel for an (n, 6) float32 CUDA
    tensor of pixel pairs.  Returns ``(angle, l2)`` (NaN for unsafe pixels)."""
    if not (pairs.is_cuda and pairs.dtype == torch.float32 and pairs.dim() == 2 and pairs.shape[1] == 6):
        raise VdfError("pairs must be a CUDA float32 tensor of shape (n, 6)")
    pairs = pairs.contiguous()
    n = int(pairs.shape[0])
    ang = torch.empty(n, dtype=torch.float32, device=pairs.device)
    l2 = torch.empty(n, dtype=torch.float32, device=pairs.device)
    _check(lib().vdf_debug_fp32_terms_f32(_ptr(pairs), n, _ptr(ang), _ptr(l2), _stream(stream)))
    return ang, l2


def debug_sqrt_error(stream=None) -> float:
    """Largest relative error (units of 2^-24) of the approximate square root
    over every positive normal float."""
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    _check(lib().vdf_debug_sqrt_error(_ptr(out), _stream(stream)))
    return float(out.item())


def filter_f32(img: torch.Tensor, win: int = 3, filter="ddf", p: float = 0.5, dist="exact", q: int = 4,
               precision="fp32", out: torch.Tensor | None = None, index: torch.Tensor | None = None,
               workspace: torch.Tensor | None = None, stream=None):
    """Filter a B x 3 x M x N float32 CUDA batch.  Returns ``(out, index)``."""
    if not (img.is_cuda and img.dtype == torch.float32 and img.dim() == 4 and img.shape[1] == 3):
        raise VdfError("img must be a CUDA float32 tensor of shape (B, 3, M, N)")
    img = img.contiguous()
    B, _, M, N = (int(v) for v in img.shape)
    if out is None:
        out = torch.empty_like(img)
    if index is None:
        index = torch.empty((B, M, N), dtype=torch.int8, device=img.device)
    prec = _code(PRECISIONS, precision)
    if workspace is None:
        workspace = alloc_workspace(B * M, N, prec, img.device)
    wp, wn = _aligned(workspace)
    _check(lib().vdf_filter_f32(_ptr(img), B, M, N, win, _code(FILTERS, filter), float(p), _code(DISTS, dist), q,
                                prec, _ptr(out), _ptr(index), wp, wn, _stream(stream)))
    return out, index


def backward_f32(grad_y: torch.Tensor, index: torch.Tensor, win: int, grad_x: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """Gradient of :func:`filter_f32` w.r.t. its input (deterministic gather)."""
    grad_y = grad_y.contiguous()
    B, _, M, N = (int(v) for v in grad_y.shape)
    if grad_x is None:
        grad_x = torch.empty_like(grad_y)
    _check(lib().vdf_backward_f32(_ptr(grad_y), _ptr(index.contiguous()), B, M, N, win, _ptr(grad_x),
                                  _stream(stream)))
    return grad_x


NOALLOC_MAX_PIXELS = 1 << 21


def filter_noalloc(img: torch.Tensor, win: int = 3, filter="bvdf", p: float = 0.5, dist="exact", q: int = 4,
                   out: torch.Tensor | None = None, index: torch.Tensor | None = None, stream=None):
    """The FP32 certified filter through ``vdf_filter_noalloc``: no workspace,
    the library's fixed device scratch (at most 2^21 pixels) is used instead."""
    L = lib()
    fn = L.vdf_filter_noalloc
    if fn.argtypes is None:
        P, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        fn.argtypes = [P, i, i, i, i, d, i, i, P, P, P]
        fn.restype = i
    img = img.contiguous()
    M, N = int(img.shape[0]), int(img.shape[1])
    if out is None:
        out = torch.empty_like(img)
    if index is None:
        index = torch.empty((M, N), dtype=torch.int8, device=img.device)
    _check(fn(_ptr(img), M, N, win, _code(FILTERS, filter), float(p), _code(DISTS, dist), q, _ptr(out), _ptr(index),
              _stream(stream)))
    return out, index


# ---------------------------------------------------------------- autotune

def _tune_fns(L):
    P, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    if L.vdf_autotune.argtypes is None:
        L.vdf_autotune.argtypes = [P, i, i, i, i, d, i, i, P, P, P, sz, i, P, P, P]
        L.vdf_autotune_acwddf.argtypes = [P, i, i, i, i, i, i, d, P, P, P, sz, i, P, P, P]
        L.vdf_tile_shape.argtypes = [i, P, P]
        L.vdf_get_tuned_shape.argtypes = [i, i, i]
        L.vdf_get_tuned_shape_p.argtypes = [i, i, i, d]
        L.vdf_set_tuned_shape.argtypes = [i, i, i, i]
        for f in ("vdf_autotune", "vdf_autotune_acwddf", "vdf_tile_shape", "vdf_get_tuned_shape", "vdf_get_tuned_shape_p",
                  "vdf_set_tuned_shape", "vdf_num_tile_shapes"):
            getattr(L, f).restype = i
    return L


def tile_shapes():
    """[(tile_w, tile_h)] of the FP32 kernel's shapes, by shape id."""
    L = _tune_fns(lib())
    out = []
    for s in range(L.vdf_num_tile_shapes()):
        w, h = ctypes.c_int(), ctypes.c_int()
        _check(L.vdf_tile_shape(s, ctypes.byref(w), ctypes.byref(h)))
        out.append((w.value, h.value))
    return out


def autotune(img: torch.Tensor, win=5, filter="ddf", p=0.25, dist="exact", q=4, reps=5, stream=None):
    """Time every tile shape on `img`; the fastest is recorded for (win,
    filter, dist) and used by later calls.  Returns (shape_id, ms)."""
    L = _tune_fns(lib())
    img = img.contiguous()
    M, N = int(img.shape[0]), int(img.shape[1])
    out = torch.empty_like(img)
    idx = torch.empty((M, N), dtype=torch.int8, device=img.device)
    ws = alloc_workspace(M, N, "fp32", img.device)
    wp, wn = _aligned(ws)
    s, ms = ctypes.c_int(), ctypes.c_float()
    _check(L.vdf_autotune(_ptr(img), M, N, win, _code(FILTERS, filter), float(p), _code(DISTS, dist), q, _ptr(out),
                          _ptr(idx), wp, wn, reps, _stream(stream), ctypes.byref(s), ctypes.byref(ms)))
    return s.value, ms.value


def autotune_acwddf(img: torch.Tensor, win: int, dist: str = "exact", q: int = 4, lam: int = 2, T: float = 10.8,
                    reps: int = 3, workspace=None, stream=None):
    """Times the FP32 ACWDDF (Eq. (9)) in every tile shape on ``img`` and records the
    fastest for vdf_filter_acwddf.  Returns (shape, ms)."""
    L = _tune_fns(lib())
    img = img.contiguous()
    M, N = int(img.shape[0]), int(img.shape[1])
    out = torch.empty_like(img)
    idx = torch.empty((M, N), dtype=torch.int8, device=img.device)
    ws = workspace if workspace is not None else alloc_workspace(M, N, "fp32", img.device)
    wp, wn = _aligned(ws)
    s, ms = ctypes.c_int(), ctypes.c_float()
    _check(L.vdf_autotune_acwddf(_ptr(img), M, N, win, _code(DISTS, dist), q, int(lam), float(T), _ptr(out), _ptr(idx),
                                 wp, wn, reps, _stream(stream), ctypes.byref(s), ctypes.byref(ms)))
    return s.value, ms.value


def tuned_shape(win, filter="ddf", dist="exact", p=None) -> int:
    """The tuned tile shape; with p, the entry used at that DDF exponent."""
    L = _tune_fns(lib())
    if p is None:
        return int(L.vdf_get_tuned_shape(win, _code(FILTERS, filter), _code(DISTS, dist)))
    return int(L.vdf_get_tuned_shape_p(win, _code(FILTERS, filter), _code(DISTS, dist), float(p)))


def set_tuned_shape(win, filter, dist, shape: int):
    _check(_tune_fns(lib()).vdf_set_tuned_shape(win, _code(FILTERS, filter), _code(DISTS, dist), shape))


# ------------------------------------------------------------------- batch

class ImageDesc(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("out", ctypes.c_void_p), ("index_out", ctypes.c_void_p),
                ("M", ctypes.c_int), ("N", ctypes.c_int), ("win", ctypes.c_int), ("filter", ctypes.c_int),
                ("p", ctypes.c_double)]


class Plan:
    """A batch of uneven uint8 images: one tile-kernel launch per
    configuration present, then one FP64 recheck launch.

    ``items``: list of dicts with keys ``img`` (CUDA uint8 M x N x 3), and
    optionally ``win`` (3), ``filter`` ("bvdf"), ``p`` (0.5), ``out`` and
    ``index``.  Outputs are allocated when absent.  The workspace is
    allocated here (torch), uploaded once, and reused by every launch.
    ``persistent`` selects the persistent work-queue form of the tile kernels
    instead of one CTA per work item (same results, slower).
    """

    def __init__(self, items, dist="exact", q=4, device=None, persistent=False):
        L = lib()
        if L.vdf_plan_create.argtypes is None:
            P, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            L.vdf_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), P, i, i, i]
            L.vdf_plan_workspace_bytes.argtypes, L.vdf_plan_workspace_bytes.restype = [P], sz
            for f in ("vdf_plan_upload", "vdf_filter_batch", "vdf_plan_graph_launch"):
                getattr(L, f).argtypes = [P, P, sz, P]
                getattr(L, f).restype = i
            L.vdf_plan_create.restype = i
            L.vdf_plan_destroy.argtypes, L.vdf_plan_destroy.restype = [P], None
            L.vdf_plan_set_persistent.argtypes, L.vdf_plan_set_persistent.restype = [P, i], i
        self._L = L
        self.items = []
        descs = (ImageDesc * len(items))()
        for k, it in enumerate(items):
            img = it["img"].contiguous()
            M, N = int(img.shape[0]), int(img.shape[1])
            out = it.get("out")
            if out is None:
                out = torch.empty_like(img)
            idx = it.get("index")
            if idx is None:
                idx = torch.empty((M, N), dtype=torch.int8, device=img.device)
            rec = dict(img=img, out=out, index=idx, win=int(it.get("win", 3)), filter=it.get("filter", "bvdf"),
                       p=float(it.get("p", 0.5)))
            self.items.append(rec)
            descs[k] = ImageDesc(img.data_ptr(), out.data_ptr(), idx.data_ptr(), M, N, rec["win"],
                                 _code(FILTERS, rec["filter"]), rec["p"])
        self._handle = ctypes.c_void_p()
        _check(L.vdf_plan_create(ctypes.byref(self._handle), ctypes.cast(descs, ctypes.c_void_p), len(items),
                                 _code(DISTS, dist), q))
        _check(L.vdf_plan_set_persistent(self._handle, int(bool(persistent))))
        nbytes = int(L.vdf_plan_workspace_bytes(self._handle))
        dev = device or self.items[0]["img"].device
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        self._wp, self._wn = _aligned(self.workspace)
        _check(L.vdf_plan_upload(self._handle, self._wp, self._wn, _stream(None)))

    def run(self, stream=None):
        _check(self._L.vdf_filter_batch(self._handle, self._wp, self._wn, _stream(stream)))

    def set_persistent(self, persistent: bool):
        _check(self._L.vdf_plan_set_persistent(self._handle, int(bool(persistent))))

    def graph_launch(self, stream=None):
        _check(self._L.vdf_plan_graph_launch(self._handle, self._wp, self._wn, _stream(stream)))

    def stats(self, stream=None):
        return workspace_stats(self.workspace, stream)

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            self._L.vdf_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_pass(img: torch.Tensor, out: torch.Tensor, index: torch.Tensor, workspace: torch.Tensor, win=5,
              filter="ddf", p=0.25, dist="exact", q=4, stream=None):
    """Stage 1 of the FP32 path (certified pass + recheck list in `workspace`)."""
    M, N = int(img.shape[0]), int(img.shape[1])
    wp, wn = _aligned(workspace)
    _check(lib().vdf_fp32_pass(_ptr(img), M, N, win, _code(FILTERS, filter), float(p), _code(DISTS, dist), q,
                               _ptr(out), _ptr(index), wp, wn, _stream(stream)))


def fp64_recheck(img: torch.Tensor, out: torch.Tensor, index: torch.Tensor, workspace: torch.Tensor, win=5,
                 filter="ddf", p=0.25, dist="exact", q=4, stream=None):
    """Stage 2 of the FP32 path (FP64 recheck of the listed pixels); may run
    on another stream than stage 1 once it has finished."""
    M, N = int(img.shape[0]), int(img.shape[1])
    wp, wn = _aligned(workspace)
    _check(lib().vdf_fp64_recheck(_ptr(img), M, N, win, _code(FILTERS, filter), float(p), _code(DISTS, dist), q,
                                  _ptr(out), _ptr(index), wp, wn, _stream(stream)))
