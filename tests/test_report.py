"""Host-side definitions of the quality report (PSNR, MAE, table layout)."""
import math

import numpy as np


def test_psnr_mae_definitions():
    from paper_1009_0958_gb300 import report
    a = np.zeros((4, 4, 3), dtype=np.uint8)
    b = a.copy()
    assert report.psnr(a, b) == math.inf and report.mae(a, b) == 0.0
    b[0, 0, 0] = 255                      # one error of 255 in 48 values
    assert abs(report.psnr(a, b) - 10 * math.log10(48)) < 1e-12
    assert abs(report.mae(a, b) - 255 / 48) < 1e-12


def test_markdown_rows():
    from paper_1009_0958_gb300 import report
    rows = [dict(size="8x8", filter="ddf", p=0.25, win=5, noise=0.1, noise_model="eq8", dist="minimax", q=4,
                 mismatch_vs_exact=0.125, psnr=30.0, mae=1.5, psnr_noisy=18.0, mae_noisy=12.0, gpu_ms=0.25)]
    t = report.markdown(rows)
    assert "| 8x8 | DDF p=0.25 | 5x5 | 10% eq8 | minimax q=4 | 12.50% | 1.500 (12.000) | 30.00 (18.00) | 0.250 |" in t


def test_noise_models_follow_eq8():
    """The paper's setting of Eq. (8): a corrupted pixel has one channel
    replaced with probability 0.25 each and all three with probability 0.25;
    the 'all' model always replaces all three."""
    from paper_1009_0958_gb300 import report
    assert report.NOISE_MODELS["eq8"] == (0.25, 0.25, 0.25) and report.NOISE_MODELS["all"] == (0.0, 0.0, 0.0)
    assert {lvl for m, lvl in report.NOISE if m == "eq8"} == {0.10, 0.15}
    clean, noisy = report.noisy_image(400, 500, 3, "eq8", 0.15)
    changed = (clean != noisy)
    frac = changed.any(axis=2).mean()
    # a corrupted channel keeps its value with probability 1/256
    assert abs(frac - 0.15) < 0.01
    nchan = changed.sum(axis=2)[changed.any(axis=2)]
    single = (nchan == 1).mean()
    # single-channel corruptions are 3/4 of the corrupted pixels (plus the rare
    # all-channel replacement that keeps two values)
    assert abs(single - 0.75) < 0.03
