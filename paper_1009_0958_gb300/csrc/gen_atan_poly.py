"""Fit the float32 polynomial atan(t) = t * Q(t^2), t in [0, 1], used by the
FP32 exact-angle term in vdf_internal.cuh (atan_q; 7 coefficients, Q of
degree 6).

Lawson's iteration (iteratively reweighted least squares) on a dense grid
drives the maximum *relative* error to its minimax value; the coefficients
are then rounded to float32 and the float32 Horner evaluation (with FMA) is
checked on 2 million points.  Run: python gen_atan_poly.py [ncoef]
"""
import sys

import numpy as np


def fit(ncoef, iters=80):
    t = np.unique(np.concatenate([np.cos(np.linspace(0, np.pi / 2, 40001)), np.linspace(0, 1, 40001)]))[1:]
    s = t * t
    f = np.arctan(t) / t
    V = np.vander(s, ncoef, increasing=True)
    w = np.ones_like(s)
    for _ in range(iters):
        W = np.sqrt(w) / f
        c, *_ = np.linalg.lstsq(V * W[:, None], f * W, rcond=None)
        e = np.abs(V @ c - f) / f
        w = w * e
        w /= w.sum()
    return c


def float32_eval_error(c32):
    t = np.linspace(0, 1, 2000001, dtype=np.float32)[1:]
    s = (t * t).astype(np.float32)
    acc = np.full_like(s, c32[-1])
    for k in range(len(c32) - 2, -1, -1):   # fma: exact product + add, one rounding
        acc = (acc.astype(np.float64) * s.astype(np.float64) + np.float64(c32[k])).astype(np.float32)
    a = (acc.astype(np.float64) * t.astype(np.float64)).astype(np.float32)
    ref = np.arctan(t.astype(np.float64))
    return (np.abs(a.astype(np.float64) - ref) / ref).max() / 2.0 ** -24


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 7
    c32 = fit(n).astype(np.float32)
    print("constexpr float kAtanQ[%d] = {%s};" % (n, ", ".join("%.8gf" % v for v in c32)))
    print("max relative error of the float32 evaluation: %.2f ulp (u = 2^-24)" % float32_eval_error(c32))
