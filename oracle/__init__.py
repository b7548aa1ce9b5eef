"""CPU oracle for the directional vector filters -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library (``paper_1009_0958_gb300``) never
imports it, and it imports nothing from the library.

``build()`` compiles ``vdf_oracle.c`` (plain C, double + binary128) into
``liboracle.so`` next to this file; the wrappers below load it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vdf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FILTERS = {"bvdf": 0, "ddf": 1, "vmf": 2}
# Minkowski order of Eq. (1): 1, 2, or "inf" (the maximum component difference)
ORDERS = {1: 1, 2: 2, "inf": 0}
DISTS = {"exact": 0, "minimax": 1, "rgb": 2}
FLAG_ESCALATED, FLAG_TIE, FLAG_GRAY = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
            L.vdf_oracle_filter_u8.argtypes = [P, i, i, i, i, d, i, i, P, i64, P, P, P, P, i]
            L.vdf_oracle_filter_u8_lp.argtypes = [P, i, i, i, i, d, i, i, i, P, i64, P, P, P, P, i]
            L.vdf_oracle_window_lp.argtypes = [P, i, i, d, i, i, i, P, P, P]
            L.vdf_oracle_filter_acwddf.argtypes = [P, i, i, i, i, i, i, d, P, i64, P, P, P, i]
            L.vdf_oracle_window_acwddf.argtypes = [P, i, i, i, i, d, P, P, P]
            L.vdf_oracle_window_cwvmf.argtypes = [P, i, i, P]
            L.vdf_oracle_filter_f32.argtypes = [P, i, i, i, i, i, d, i, i, P, i64, P, P, P, P, i]
            L.vdf_oracle_window.argtypes = [P, i, i, d, i, i, P, P, P]
            L.vdf_oracle_term.argtypes = [P, P, i, i, i, P, P, P]
            L.vdf_oracle_poly.argtypes = [i, i, d, P, P]
            L.vdf_oracle_max_threads.argtypes = []
            for f in ("vdf_oracle_filter_u8", "vdf_oracle_filter_u8_lp", "vdf_oracle_window_lp",
                      "vdf_oracle_filter_acwddf", "vdf_oracle_window_acwddf", "vdf_oracle_window_cwvmf",
                      "vdf_oracle_filter_f32", "vdf_oracle_window",
                      "vdf_oracle_term", "vdf_oracle_poly", "vdf_oracle_max_threads"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cfg(filter, dist):
    return FILTERS[filter] if isinstance(filter, str) else int(filter), DISTS[dist] if isinstance(dist, str) else int(dist)


def filter_u8(img, win=3, filter="bvdf", p=0.5, dist="exact", q=4, pixels=None, want_agg=False, threads=0,
              order=2):
    """Run the oracle on an M x N x 3 uint8 image.

    ``order`` is the Minkowski order of the distance term (DDF, VMF): 1, 2
    or "inf".  Returns a dict with ``out`` (uint8, M x N x 3, or count x 3
    for a pixel subset), ``idx`` (int8), ``flags`` (int32) and, if requested,
    ``agg`` (float64, [..., n, 2]: sum of angular terms, sum of distance
    terms).
    """
    img = np.ascontiguousarray(img, dtype=np.uint8)
    M, N = img.shape[:2]
    f, dm = _cfg(filter, dist)
    n = win * win
    if pixels is None:
        shape, count, pix = (M, N), M * N, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        shape, count = (pix.shape[0],), pix.shape[0]
    out = np.zeros(shape + (3,), np.uint8)
    idx = np.zeros(shape, np.int8)
    flags = np.zeros(shape, np.int32)
    agg = np.zeros(shape + (n, 2), np.float64) if want_agg else None
    rc = lib().vdf_oracle_filter_u8_lp(_ptr(img), M, N, win, f, float(p), ORDERS[order], dm, q, _ptr(pix), count,
                                      _ptr(out), _ptr(idx), _ptr(flags), _ptr(agg), threads)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return {"out": out, "idx": idx, "flags": flags, "agg": agg}


def filter_f32(img_nchw, win=3, filter="ddf", p=0.5, dist="exact", q=4, pixels=None, want_agg=False, threads=0):
    """Run the oracle on a B x 3 x M x N float32 batch (same outputs as
    :func:`filter_u8`; ``out`` is B x 3 x M x N float32 for the full batch,
    count x 3 for a subset)."""
    img = np.ascontiguousarray(img_nchw, dtype=np.float32)
    B, C, M, N = img.shape
    assert C == 3
    f, dm = _cfg(filter, dist)
    n = win * win
    if pixels is None:
        count, pix = B * M * N, None
        out = np.zeros((B, 3, M, N), np.float32)
        shape = (B, M, N)
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        count = pix.shape[0]
        out = np.zeros((count, 3), np.float32)
        shape = (count,)
    idx = np.zeros(shape, np.int8)
    flags = np.zeros(shape, np.int32)
    agg = np.zeros(shape + (n, 2), np.float64) if want_agg else None
    rc = lib().vdf_oracle_filter_f32(_ptr(img), B, M, N, win, f, float(p), dm, q, _ptr(pix), count,
                                    _ptr(out), _ptr(idx), _ptr(flags), _ptr(agg), threads)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return {"out": out, "idx": idx, "flags": flags, "agg": agg}


def window(vecs, filter="bvdf", p=0.5, dist="exact", q=4, order=2):
    """Select within one window given as an n x 3 array (raster order).

    Returns ``(index, scores, agg, flags)``."""
    v = np.ascontiguousarray(vecs, dtype=np.float64)
    n = v.shape[0]
    f, dm = _cfg(filter, dist)
    score = np.zeros(n, np.float64)
    agg = np.zeros((n, 2), np.float64)
    fl = np.zeros(1, np.int32)
    sel = lib().vdf_oracle_window_lp(_ptr(v), n, f, float(p), ORDERS[order], dm, q, _ptr(score), _ptr(agg),
                                     _ptr(fl))
    if sel < 0:
        raise ValueError("oracle rejected the arguments")
    return sel, score, agg, int(fl[0])


def filter_acwddf(img, win=3, dist="exact", q=4, lam=2, T=10.8, pixels=None, threads=0):
    """ACWDDF (Eq. (9)) of an M x N x 3 uint8 image: dict with ``out``,
    ``idx`` and ``flags`` as :func:`filter_u8`."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    M, N = img.shape[:2]
    _, dm = _cfg(0, dist)
    if pixels is None:
        shape, count, pix = (M, N), M * N, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        shape, count = (pix.shape[0],), pix.shape[0]
    out = np.zeros(shape + (3,), np.uint8)
    idx = np.zeros(shape, np.int8)
    flags = np.zeros(shape, np.int32)
    rc = lib().vdf_oracle_filter_acwddf(_ptr(img), M, N, win, dm, q, lam, float(T), _ptr(pix), count, _ptr(out),
                                        _ptr(idx), _ptr(flags), threads)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return {"out": out, "idx": idx, "flags": flags}


def window_acwddf(vecs, dist="exact", q=4, lam=2, T=10.8):
    """ACWDDF of one window (n x 3, raster order): ``(index, cwvmf_indices,
    switching_sum, flags)``."""
    v = np.ascontiguousarray(vecs, dtype=np.float64)
    _, dm = _cfg(0, dist)
    cw = np.zeros(3, np.int32)
    sm = np.zeros(1)
    fl = np.zeros(1, np.int32)
    sel = lib().vdf_oracle_window_acwddf(_ptr(v), v.shape[0], dm, q, lam, float(T), _ptr(cw), _ptr(sm), _ptr(fl))
    if sel < 0:
        raise ValueError("oracle rejected the arguments")
    return sel, [int(c) for c in cw], float(sm[0]), int(fl[0])


def window_cwvmf(vecs, k):
    """Centre-weighted VMF of Eq. (9) of one window at smoothing level k:
    ``(index, flags)``."""
    v = np.ascontiguousarray(vecs, dtype=np.float64)
    fl = np.zeros(1, np.int32)
    sel = lib().vdf_oracle_window_cwvmf(_ptr(v), v.shape[0], k, _ptr(fl))
    if sel < 0:
        raise ValueError("oracle rejected the arguments")
    return sel, int(fl[0])


def term(x, y, which="angle", dist="exact", q=4):
    """One pair term (``which``: "angle", "l2", "l1" or "linf"): returns
    ``(double_value, binary128_hi, binary128_lo)``."""
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    d, hi, lo = (np.zeros(1) for _ in range(3))
    _, dm = _cfg(0, dist)
    code = {"angle": 0, "l2": 1, "l1": 2, "linf": 3}[which]
    rc = lib().vdf_oracle_term(_ptr(xa), _ptr(ya), code, dm, q, _ptr(d), _ptr(hi), _ptr(lo))
    if rc != 0:
        raise ValueError("bad term arguments")
    return float(d[0]), float(hi[0]), float(lo[0])


def poly(branch: str, q: int, t: float):
    """Table 1 polynomial (branch 'acos' in z or 'asin' in tau) at t, binary128 as (hi, lo)."""
    hi, lo = np.zeros(1), np.zeros(1)
    rc = lib().vdf_oracle_poly(1 if branch == "asin" else 0, q, float(t), _ptr(hi), _ptr(lo))
    if rc != 0:
        raise ValueError("bad poly arguments")
    return float(hi[0]), float(lo[0])


def max_threads() -> int:
    return int(lib().vdf_oracle_max_threads())
