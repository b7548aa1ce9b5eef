"""Image-quality sanity of the filters (Section III's protocol on synthetic
images): filtering impulsive noise raises the PSNR against the clean image
well above the noisy input's, the exact mode has no mismatch against itself,
and the speed-up modes select the exact mode's member on most pixels."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rows():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0958_gb300 import build, report
    build.build()
    return report.evaluate(sizes=[(256, 320)], noise=[0.10, 0.20])


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
    assert len(rows) == 2 * 2 * 2 * 3


def test_markdown_table(rows):
    from paper_1009_0958_gb300 import report
    table = report.markdown(rows)
    assert table.count("\n") == len(rows) + 1 and "mismatch vs exact" in table
