"""Quality report in the layout of the paper's experiments (Section III):
Experiment 1 (Tables 2 and 3: the BVDF and its two speed-up methods) and
Experiment 2 (Tables 4 and 5: the ACWDDF of Eq. (9), lambda = 2, T = 10.8),
plus the DDF, on synthetic stand-ins for the paper's test images.

For each image size, filter, window, noise model and level, and distance mode
it gives:
  * the fraction of pixels where the mode (Method 1, Table 1 with degree q;
    Method 2, Eq. (7), through Eq. (10) inside the DDF and the ACWDDF)
    selects another member than the exact arccos form of Eq. (2);
  * MAE and PSNR of the filtered image against the clean one (textbook
    definitions over the three channels), next to those of the noisy input
    (the tables' "none" row);
  * the GPU time of the FP32 certified path (CUDA events, mean of three
    calls), in the place of the tables' TIME column.
NCD is not reported: it needs a colour-space conversion the paper does not
give.

Noise (Section III, Eq. (8)): a pixel is corrupted with probability phi; a
corrupted pixel has one channel k replaced with probability phi_k and all
three replaced otherwise.  "eq8" is the paper's setting, phi_k = 0.25 for
every channel, at its two levels 10% and 15%; "all" replaces all three
channels (phi_k = 0), the model the benchmark configurations name, at 5, 10,
15 and 20%.  Images: the sinusoid field with 12 flat rectangles.

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
FILTERS = [("bvdf", 0.5), ("ddf", 0.25), ("acwddf", None)]
WINDOWS = [3, 5]
MODES = [("exact", 4), ("minimax", 4), ("rgb", 4)]
NOISE_MODELS = {"eq8": (0.25, 0.25, 0.25), "all": (0.0, 0.0, 0.0)}
NOISE = [("eq8", 0.10), ("eq8", 0.15), ("all", 0.05), ("all", 0.10), ("all", 0.15), ("all", 0.20)]
ACW_LAMBDA, ACW_T = 2, 10.8


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2)
    return math.inf if mse == 0 else 10.0 * math.log10(255.0 ** 2 / mse)


def mae(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.mean(np.abs(a.astype(np.float64) - b.astype(np.float64))))


def noisy_image(M: int, N: int, seed: int, model: str, phi: float):
    """(clean, noisy) for one noise model and level."""
    return synth.make_image(M, N, seed, phi, rectangles=12, channel_probs=NOISE_MODELS[model])


def run_filter(x, filt, p, win, dist, q):
    if filt == "acwddf":
        return vdf.filter_acwddf(x, win, dist, q, ACW_LAMBDA, ACW_T, precision="fp32")
    return vdf.filter(x, win, filt, p, dist, q, precision="fp32")


def timed_ms(fn, reps: int = 3) -> float:
    fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def evaluate(sizes=SIZES, filters=FILTERS, windows=WINDOWS, modes=MODES, noise=NOISE, seed=2024, timing=True):
    """One row per (size, noise model and level, filter, window, mode)."""
    rows = []
    for (M, N) in sizes:
        for k, (model, phi) in enumerate(noise):
            clean, noisy = noisy_image(M, N, seed + 17 * k, model, phi)
            x = torch.from_numpy(noisy).cuda()
            for filt, p in filters:
                for win in windows:
                    exact_idx = None
                    for dist, q in modes:
                        out, idx = run_filter(x, filt, p, win, dist, q)
                        ms = timed_ms(lambda: run_filter(x, filt, p, win, dist, q)) if timing else None
                        out, idx = out.cpu().numpy(), idx.cpu().numpy()
                        if dist == "exact":
                            exact_idx = idx
                        rows.append(dict(
                            size=f"{N}x{M}", filter=filt, p=p if filt == "ddf" else None, win=win, noise=phi,
                            noise_model=model, dist=dist, q=q if dist == "minimax" else None,
                            mismatch_vs_exact=float(np.mean(idx != exact_idx)),
                            psnr=psnr(out, clean), mae=mae(out, clean),
                            psnr_noisy=psnr(noisy, clean), mae_noisy=mae(noisy, clean), gpu_ms=ms))
    return rows


def markdown(rows) -> str:
    head = ("| size | filter | window | noise | mode | mismatch vs exact | MAE (noisy) | PSNR dB (noisy) | GPU ms |\n"
            "|---|---|---|---|---|---|---|---|---|")
    lines = [head]
    for r in rows:
        mode = r["dist"] + (f" q={r['q']}" if r["q"] else "")
        filt = r["filter"].upper() + (f" p={r['p']}" if r["p"] is not None else "")
        model = r.get("noise_model", "all")
        noise = f"{int(round(100 * r['noise']))}% {model}"
        ms = "-" if r.get("gpu_ms") is None else f"{r['gpu_ms']:.3f}"
        lines.append(f"| {r['size']} | {filt} | {r['win']}x{r['win']} | {noise} | {mode} "
                     f"| {100 * r['mismatch_vs_exact']:.2f}% | {r['mae']:.3f} ({r['mae_noisy']:.3f}) "
                     f"| {r['psnr']:.2f} ({r['psnr_noisy']:.2f}) | {ms} |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--json", action="store_true", help="print the rows as JSON instead of a table")
    args = ap.parse_args()
    rows = evaluate()
    print(json.dumps(rows) if args.json else markdown(rows))


if __name__ == "__main__":
    main()
