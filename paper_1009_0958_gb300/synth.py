"""Seeded synthetic colour images for the directional vector filters.

This module is the only code shared by the CUDA path's tests/bench and the CPU
oracle's tests.  It holds no filter arithmetic: it only draws images.

The paper's own test images (Section III, Figure 2) are not available, so the
workloads are stand-ins with the same structure: smooth colour fields, flat
regions with sharp edges (which produce exact duplicates and hence ties), and
the impulsive noise of Section III, Eq. (8).

All generators use numpy's PCG64 through ``np.random.default_rng(seed)`` and
return HWC ``uint8`` arrays (rows M, columns N, 3 channels) unless stated.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "sinusoid_field",
    "add_rectangles",
    "impulsive_noise",
    "make_image",
    "to_float_nchw",
    "batch_shapes",
]


def sinusoid_field(M: int, N: int, seed: int, terms: int = 4) -> np.ndarray:
    """Smooth RGB field: per channel, 127.5 plus ``terms`` random plane waves.

    Each wave has amplitude U(10, 30), spatial frequencies U(-3, 3) cycles per
    image along each axis and phase U(0, 2*pi).  With four waves the amplitude
    sum stays below 120, so nothing clips and no pixel is black.
    """
    rng = np.random.default_rng(seed)
    r = np.arange(M, dtype=np.float64)[:, None]
    c = np.arange(N, dtype=np.float64)[None, :]
    out = np.empty((M, N, 3), dtype=np.float64)
    for k in range(3):
        a = rng.uniform(10.0, 30.0, terms)
        u = rng.uniform(-3.0, 3.0, terms)
        v = rng.uniform(-3.0, 3.0, terms)
        ph = rng.uniform(0.0, 2.0 * np.pi, terms)
        acc = np.full((M, N), 127.5)
        for m in range(terms):
            acc += a[m] * np.sin(2.0 * np.pi * (u[m] * c / max(N, 1) + v[m] * r / max(M, 1)) + ph[m])
        out[:, :, k] = acc
    return np.clip(np.rint(out), 0, 255).astype(np.uint8)


def add_rectangles(img: np.ndarray, seed: int, count: int = 12) -> np.ndarray:
    """Overwrite ``count`` axis-aligned flat rectangles of random colour.

    Sides are U(5%, 30%) of each image dimension; colours are uniform 0..255
    per channel.  Flat regions give windows full of identical vectors.
    """
    rng = np.random.default_rng(seed)
    out = img.copy()
    M, N = out.shape[:2]
    for _ in range(count):
        h = max(1, int(round(rng.uniform(0.05, 0.30) * M)))
        w = max(1, int(round(rng.uniform(0.05, 0.30) * N)))
        r0 = int(rng.integers(0, max(1, M - h + 1)))
        c0 = int(rng.integers(0, max(1, N - w + 1)))
        out[r0:r0 + h, c0:c0 + w, :] = rng.integers(0, 256, 3, dtype=np.int64).astype(np.uint8)
    return out


def impulsive_noise(img: np.ndarray, phi: float, seed: int,
                    channel_probs: tuple[float, float, float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """Correlated impulsive noise model, Section III, Eq. (8).

    With probability ``phi`` a pixel is corrupted.  A corrupted pixel has only
    channel k replaced with probability ``channel_probs[k]``, and all three
    channels replaced otherwise.  Replacement values are uniform 0..255.  The
    default (all-channel impulses) is the variant with phi_1 = phi_2 = phi_3 =
    0; the paper's own experiments use 0.25 for each channel.
    """
    rng = np.random.default_rng(seed)
    out = img.copy()
    M, N = out.shape[:2]
    hit = rng.random((M, N)) < phi
    choice = rng.random((M, N))
    repl = rng.integers(0, 256, (M, N, 3), dtype=np.int64).astype(np.uint8)
    p1, p2, p3 = channel_probs
    edges = np.cumsum([p1, p2, p3])
    which = np.searchsorted(edges, choice, side="right")  # 0,1,2 single channel; 3 all
    for k in range(3):
        mask = hit & ((which == k) | (which == 3))
        out[:, :, k][mask] = repl[:, :, k][mask]
    return out


def make_image(M: int, N: int, seed: int, noise: float = 0.10, rectangles: int = 0,
               channel_probs: tuple[float, float, float] = (0.0, 0.0, 0.0)):
    """Return ``(clean, noisy)`` uint8 HWC images of the standard recipe.

    ``clean`` is the sinusoid field, optionally with ``rectangles`` flat
    rectangles; ``noisy`` adds impulsive noise of probability ``noise``.
    Sub-seeds are derived from ``seed`` so every part is reproducible.
    """
    clean = sinusoid_field(M, N, seed)
    if rectangles:
        clean = add_rectangles(clean, seed + 1_000_003, rectangles)
    noisy = impulsive_noise(clean, noise, seed + 2_000_003, channel_probs)
    return clean, noisy


def to_float_nchw(imgs: np.ndarray) -> np.ndarray:
    """uint8 B x M x N x 3 (or M x N x 3) to float32 B x 3 x M x N in [0, 1]."""
    a = np.asarray(imgs)
    if a.ndim == 3:
        a = a[None]
    return np.ascontiguousarray(np.transpose(a.astype(np.float32) / np.float32(255.0), (0, 3, 1, 2)))


def batch_shapes(count: int, seed: int, lo: int = 64, hi: int = 2048,
                 aspect_lo: float = 0.5, aspect_hi: float = 2.0):
    """Image sizes for the uneven batch workload.

    The side s is log-uniform in [lo, hi] and the aspect ratio a log-uniform
    in [aspect_lo, aspect_hi]; the image is round(s * sqrt(a)) wide and
    round(s / sqrt(a)) high, each clipped to [1, 2 * hi].
    """
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(np.log(lo), np.log(hi), count))
    a = np.exp(rng.uniform(np.log(aspect_lo), np.log(aspect_hi), count))
    N = np.clip(np.rint(s * np.sqrt(a)), 1, 2 * hi).astype(np.int64)
    M = np.clip(np.rint(s / np.sqrt(a)), 1, 2 * hi).astype(np.int64)
    return [(int(m), int(n)) for m, n in zip(M, N)]
