"""Quality report in the layout of the paper's Experiment 1 (Section III,
Tables 2 and 3), on synthetic stand-ins for its test images.

For each image size, filter, window, distance mode and noise level it gives
the fraction of pixels where the mode (Method 1, Table 1 with degree q; or
Method 2, Eq. (7)) selects a different member than the exact arccos form of
Eq. (2), and the PSNR and MAE of the filtered image against the clean one
(textbook definitions over the three channels), next to those of the noisy
input.  Images: the sinusoid field with 12 flat rectangles, corrupted by the
impulsive noise of Eq. (8) with all three channel probabilities equal.

Run on a CUDA device:  python -m paper_1009_0958_gb300.report [--json]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import synth, vdf

SIZES = [(512, 512), (1080, 1920)]
FILTERS = [("bvdf", 0.5), ("ddf", 0.25)]
WINDOWS = [3, 5]
MODES = [("exact", 4), ("minimax", 4), ("rgb", 4)]
NOISE = [0.05, 0.10, 0.20]


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2)
    return math.inf if mse == 0 else 10.0 * math.log10(255.0 ** 2 / mse)


def mae(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.mean(np.abs(a.astype(np.float64) - b.astype(np.float64))))


def evaluate(sizes=SIZES, filters=FILTERS, windows=WINDOWS, modes=MODES, noise=NOISE, seed=2024):
    """One row per (size, filter, window, noise, mode)."""
    rows = []
    for (M, N) in sizes:
        for k, phi in enumerate(noise):
            clean, noisy = synth.make_image(M, N, seed + 17 * k, phi, rectangles=12)
            x = torch.from_numpy(noisy).cuda()
            for filt, p in filters:
                for win in windows:
                    exact_idx = None
                    for dist, q in modes:
                        out, idx = vdf.filter(x, win, filt, p, dist, q, precision="fp32")
                        out, idx = out.cpu().numpy(), idx.cpu().numpy()
                        if dist == "exact":
                            exact_idx = idx
                        rows.append(dict(
                            size=f"{N}x{M}", filter=filt, p=p if filt == "ddf" else None, win=win, noise=phi,
                            dist=dist, q=q if dist == "minimax" else None,
                            mismatch_vs_exact=float(np.mean(idx != exact_idx)),
                            psnr=psnr(out, clean), mae=mae(out, clean),
                            psnr_noisy=psnr(noisy, clean), mae_noisy=mae(noisy, clean)))
    return rows


def markdown(rows) -> str:
    head = ("| size | filter | window | noise | mode | mismatch vs exact | PSNR dB (noisy) | MAE (noisy) |\n"
            "|---|---|---|---|---|---|---|---|")
    lines = [head]
    for r in rows:
        mode = r["dist"] + (f" q={r['q']}" if r["q"] else "")
        filt = r["filter"].upper() + (f" p={r['p']}" if r["p"] is not None else "")
        lines.append(f"| {r['size']} | {filt} | {r['win']}x{r['win']} | {int(round(100 * r['noise']))}% | {mode} "
                     f"| {100 * r['mismatch_vs_exact']:.2f}% | {r['psnr']:.2f} ({r['psnr_noisy']:.2f}) "
                     f"| {r['mae']:.2f} ({r['mae_noisy']:.2f}) |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--json", action="store_true", help="print the rows as JSON instead of a table")
    args = ap.parse_args()
    rows = evaluate()
    print(json.dumps(rows) if args.json else markdown(rows))


if __name__ == "__main__":
    main()
