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
    rows = [dict(size="8x8", filter="ddf", p=0.25, win=5, noise=0.1, dist="minimax", q=4, mismatch_vs_exact=0.125,
                 psnr=30.0, mae=1.5, psnr_noisy=18.0, mae_noisy=12.0)]
    t = report.markdown(rows)
    assert "| 8x8 | DDF p=0.25 | 5x5 | 10% | minimax q=4 | 12.50% | 30.00 (18.00) | 1.50 (12.00) |" in t
