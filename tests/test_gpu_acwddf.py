"""ACWDDF (Eq. (9)) through vdf_filter_acwddf: the CUDA selections equal the
CPU oracle's bit for bit in both precisions (every distance mode, several
smoothing levels and thresholds, edge cases), and the FP32 path (certified
decisions + full FP64 recheck of the open pixels) equals the FP64 path on
whole 1080p frames."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0958_gb300 import build, vdf
    build.build()
    return vdf


@pytest.fixture(scope="module")
def O():
    import oracle
    oracle.build()
    return oracle


def run(V, img, win, dist, q, lam, T, prec):
    x = torch.from_numpy(img).cuda()
    M, N = img.shape[:2]
    ws = V.alloc_workspace(M, N, prec)
    out, idx = V.filter_acwddf(x, win, dist, q, lam, T, precision=prec, workspace=ws)
    torch.cuda.synchronize()
    stats = V.workspace_stats(ws) if ws is not None else (0, 0)
    return out.cpu().numpy(), idx.cpu().numpy(), stats


def images():
    from paper_1009_0958_gb300 import synth
    rng = np.random.default_rng(9)
    yield "rect20", synth.make_image(70, 101, 1, 0.20, rectangles=12)[1]
    yield "field10", synth.make_image(53, 77, 2, 0.10)[1]
    yield "small_range", rng.integers(0, 4, (41, 67, 3)).astype(np.uint8)
    yield "1x57", rng.integers(0, 256, (1, 57, 3)).astype(np.uint8)
    yield "45x1", rng.integers(0, 256, (45, 1, 3)).astype(np.uint8)
    yield "constant", np.full((20, 35, 3), 77, np.uint8)
    yield "black_specks", np.where(rng.random((21, 40, 1)) < 0.3, 0, rng.integers(0, 256, (21, 40, 3))).astype(np.uint8)


IMAGES = dict(images())


@pytest.mark.parametrize("name", list(IMAGES))
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("dist,q", [("exact", 4), ("minimax", 4), ("minimax", 3), ("rgb", 4)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_selection_matches_oracle(V, O, name, win, dist, q, prec):
    img = IMAGES[name]
    ref = O.filter_acwddf(img, win, dist, q, 2, 10.8)
    assert not (ref["flags"] & O.FLAG_GRAY).any()
    out, idx, (rc, ov) = run(V, img, win, dist, q, 2, 10.8, prec)
    assert np.array_equal(idx, ref["idx"]) and np.array_equal(out, ref["out"])
    assert ov == 0


@pytest.mark.parametrize("lam,T", [(1, 10.8), (3, 10.8), (2, 0.5), (2, 200.0), (2, -1.0), (2, 1e30)])
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_levels_and_thresholds(V, O, lam, T, win, prec):
    img = IMAGES["rect20"]
    ref = O.filter_acwddf(img, win, "exact", 4, lam, T)
    out, idx, _ = run(V, img, win, "exact", 4, lam, T, prec)
    assert np.array_equal(idx, ref["idx"]) and np.array_equal(out, ref["out"])
    if T == 1e30:
        assert np.array_equal(out, img)


@pytest.mark.parametrize("win,dist", [(3, "exact"), (5, "exact"), (3, "rgb")])
def test_full_size_1080p(V, O, win, dist):
    """1920 x 1080: the FP32 path equals the FP64 path on every pixel and the
    oracle on 3000 sampled pixels."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(1080, 1920, 12, 0.10, rectangles=12)
    out, idx, (rc, ov) = run(V, img, win, dist, 4, 2, 10.8, "fp32")
    out64, idx64, _ = run(V, img, win, dist, 4, 2, 10.8, "fp64")
    assert ov == 0 and np.array_equal(idx, idx64) and np.array_equal(out, out64)
    rng = np.random.default_rng(4)
    pix = np.concatenate([rng.integers(0, 1080 * 1920, 2996), [0, 1919, 1080 * 1920 - 1, 1079 * 1920]])
    ref = O.filter_acwddf(img, win, dist, 4, 2, 10.8, pixels=pix)
    assert np.array_equal(idx.reshape(-1)[pix], ref["idx"])
    assert np.array_equal(out.reshape(-1, 3)[pix], ref["out"])


def test_every_tile_shape(V):
    from paper_1009_0958_gb300 import synth
    x = torch.from_numpy(synth.make_image(203, 317, 9, 0.2, rectangles=8)[1]).cuda()
    ref = V.filter_acwddf(x, 5, precision="fp64")
    try:
        for s in range(len(V.tile_shapes())):
            V.set_tuned_shape(5, "ddf", "exact", s)
            o, i = V.filter_acwddf(x, 5, precision="fp32")
            assert torch.equal(o, ref[0]) and torch.equal(i, ref[1])
    finally:
        V.set_tuned_shape(5, "ddf", "exact", 0)


@pytest.mark.parametrize("win,dist", [(3, "exact"), (5, "exact"), (3, "minimax")])
def test_autotune_acwddf(V, O, win, dist):
    """The ACWDDF's own tile-shape autotuner: a shape in range, a valid time,
    and later calls (in the recorded shape) equal to the oracle."""
    from paper_1009_0958_gb300 import synth
    img = synth.make_image(130, 170, 31, 0.15, rectangles=8)[1]
    x = torch.from_numpy(img).cuda()
    try:
        shape, ms = V.autotune_acwddf(x, win, dist, 4, 2, 10.8, reps=2)
        assert 0 <= shape < len(V.tile_shapes()) and ms > 0
        o, i = V.filter_acwddf(x, win, dist, 4, 2, 10.8, precision="fp32")
        ref = O.filter_acwddf(img, win, dist, 4, 2, 10.8)
        assert np.array_equal(i.cpu().numpy(), ref["idx"]) and np.array_equal(o.cpu().numpy(), ref["out"])
    finally:
        V.set_tuned_shape(win, "ddf", dist, 0)


def test_bad_arguments(V):
    x = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    for lam in (0, 4):
        with pytest.raises(V.VdfError):
            V.filter_acwddf(x, 3, lam=lam)
    with pytest.raises(V.VdfError):
        V.filter_acwddf(x, 3, T=float("nan"))
    V.filter_acwddf(x, 5, lam=11)
