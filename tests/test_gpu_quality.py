"""Image quality of the filters under the paper's protocol (Section III,
Experiments 1 and 2) on synthetic images: filtering impulsive noise of either
model (Eq. (8) with phi_k = 0.25, or all three channels replaced) at the
paper's 10% and 15% levels raises the PSNR against the clean image well above
the noisy input's, for the BVDF, the DDF and the ACWDDF; the exact mode has no
mismatch against itself and the speed-up modes select the exact mode's member
on most pixels; the ACWDDF's exact mode equals the oracle's on the report's
image."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NOISE = [("eq8", 0.10), ("eq8", 0.15), ("all", 0.10), ("all", 0.15)]


@pytest.fixture(scope="module")
def rows():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0958_gb300 import build, report
    build.build()
    return report.evaluate(sizes=[(256, 320)], noise=NOISE, timing=False)


def test_filtering_raises_psnr(rows):
    for r in rows:
        assert r["psnr"] > r["psnr_noisy"] + 5.0, r
        assert r["mae"] < r["mae_noisy"], r


def test_mismatch_fractions(rows):
    for r in rows:
        if r["dist"] == "exact":
            assert r["mismatch_vs_exact"] == 0.0
        else:
            assert 0.0 <= r["mismatch_vs_exact"] < 0.5, r
    assert len(rows) == len(NOISE) * 3 * 2 * 3
    assert {r["filter"] for r in rows} == {"bvdf", "ddf", "acwddf"}
    assert {(r["noise_model"], r["noise"]) for r in rows} == set(NOISE)


def test_markdown_table(rows):
    from paper_1009_0958_gb300 import report
    table = report.markdown(rows)
    assert table.count("\n") == len(rows) + 1 and "mismatch vs exact" in table
    assert "15% eq8" in table and "ACWDDF" in table


@pytest.mark.parametrize("model,phi", NOISE)
@pytest.mark.parametrize("win", [3, 5])
def test_acwddf_exact_equals_oracle_on_report_image(model, phi, win):
    import oracle
    from paper_1009_0958_gb300 import report, vdf
    oracle.build()
    k = NOISE.index((model, phi))
    _, noisy = report.noisy_image(256, 320, 2024 + 17 * k, model, phi)
    ref = oracle.filter_acwddf(noisy, win, "exact", 4, report.ACW_LAMBDA, report.ACW_T)
    out, idx = vdf.filter_acwddf(torch.from_numpy(noisy).cuda(), win, "exact", 4, report.ACW_LAMBDA, report.ACW_T,
                                 precision="fp32")
    torch.cuda.synchronize()
    assert np.array_equal(idx.cpu().numpy(), ref["idx"]) and np.array_equal(out.cpu().numpy(), ref["out"])
