"""The vector median filter (Eq. (1)) and the Minkowski orders 1, 2 and
infinity (VMF, and the DDF's distance term), through vdf_filter_lp: the CUDA
selections equal the CPU oracle's bit for bit in both precisions, the FP64
aggregates agree within 1e-12, orders 1 and infinity need no recheck, and the
scalar median filter is reproduced on one-direction images."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KINDS = [("vmf", 0.5, 1), ("vmf", 0.5, 2), ("vmf", 0.5, "inf"),
         ("ddf", 0.25, 1), ("ddf", 0.3, 1), ("ddf", 0.25, "inf"), ("ddf", 0.5, "inf"), ("ddf", 0.0, 1),
         ("ddf", 1.0, "inf")]


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


def run(V, img, win, filter, p, order, prec, agg=False):
    x = torch.from_numpy(img).cuda()
    M, N = img.shape[:2]
    ag = torch.zeros((M, N, win * win, 2), dtype=torch.float64, device="cuda") if agg else None
    ws = V.alloc_workspace(M, N, prec)
    out, idx = V.filter(x, win, filter, p, "exact", 4, precision=prec, agg=ag, workspace=ws, order=order)
    torch.cuda.synchronize()
    stats = V.workspace_stats(ws) if ws is not None else (0, 0)
    return out.cpu().numpy(), idx.cpu().numpy(), (ag.cpu().numpy() if agg else None), stats


def images():
    from paper_1009_0958_gb300 import synth
    rng = np.random.default_rng(5)
    # several tiles of every shape plus ragged tails
    yield "rect20", synth.make_image(70, 101, 1, 0.20, rectangles=12)[1]
    yield "field10", synth.make_image(53, 77, 2, 0.10)[1]
    yield "small_range", rng.integers(0, 4, (41, 67, 3)).astype(np.uint8)   # many exact ties
    yield "1x1", rng.integers(0, 256, (1, 1, 3)).astype(np.uint8)
    yield "1x57", rng.integers(0, 256, (1, 57, 3)).astype(np.uint8)
    yield "45x1", rng.integers(0, 256, (45, 1, 3)).astype(np.uint8)
    yield "constant", np.full((20, 35, 3), 77, np.uint8)
    yield "black_specks", np.where(rng.random((21, 40, 1)) < 0.3, 0, rng.integers(0, 256, (21, 40, 3))).astype(np.uint8)


IMAGES = dict(images())


@pytest.mark.parametrize("name", list(IMAGES))
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p,order", KINDS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_selection_matches_oracle(V, O, name, win, filter, p, order, prec):
    img = IMAGES[name]
    ref = O.filter_u8(img, win, filter, p, "exact", 4, order=order)
    out, idx, _, (rc, ov) = run(V, img, win, filter, p, order, prec)
    assert np.array_equal(idx, ref["idx"]) and np.array_equal(out, ref["out"])
    assert ov == 0
    if filter == "vmf" and order != 2:
        assert rc == 0   # exact integer aggregates: nothing to recheck


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p,order", KINDS)
def test_fp64_aggregates_match_oracle(V, O, win, filter, p, order):
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(37, 41, 3, 0.15, rectangles=5)
    ref = O.filter_u8(img, win, filter, p, "exact", 4, order=order, want_agg=True)
    _, idx, agg, _ = run(V, img, win, filter, p, order, "fp64", agg=True)
    assert np.array_equal(idx, ref["idx"])
    assert np.allclose(agg, ref["agg"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("order", [1, 2, "inf"])
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("channel", [None, 1])
def test_vmf_is_the_median_filter_on_one_direction_images(V, order, win, channel):
    """Gray pixels, or one varying channel: the VMF output is numpy's median
    filter (edge replication), whatever the order."""
    from numpy.lib.stride_tricks import sliding_window_view
    rng = np.random.default_rng(7 + win)
    M, N = 67, 91
    s = rng.integers(0, 256, (M, N))
    s[rng.random((M, N)) < 0.3] = 200
    if channel is None:
        img = np.repeat(s[..., None], 3, axis=2).astype(np.uint8)
    else:
        img = np.tile(np.array([40, 0, 90]), (M, N, 1)).astype(np.uint8)
        img[..., channel] = s
    med = np.median(sliding_window_view(np.pad(s, win // 2, mode="edge"), (win, win)), axis=(-2, -1))
    for prec in ("fp32", "fp64"):
        out, _, _, _ = run(V, img, win, "vmf", 0.5, order, prec)
        assert np.array_equal(out[..., 0 if channel is None else channel], med.astype(np.uint8))


@pytest.mark.parametrize("filter,p,order,win", [("vmf", 0.5, 1, 5), ("vmf", 0.5, 2, 5), ("vmf", 0.5, "inf", 3),
                                                ("ddf", 0.25, 1, 5)])
def test_full_size_1080p(V, O, filter, p, order, win):
    """1920 x 1080: the FP32 path equals the FP64 path on every pixel and the
    oracle on 3000 sampled pixels."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(1080, 1920, 8, 0.10, rectangles=12)
    out, idx, _, (rc, ov) = run(V, img, win, filter, p, order, "fp32")
    out64, idx64, _, _ = run(V, img, win, filter, p, order, "fp64")
    assert ov == 0 and np.array_equal(idx, idx64) and np.array_equal(out, out64)
    rng = np.random.default_rng(3)
    pix = np.concatenate([rng.integers(0, 1080 * 1920, 2996), [0, 1919, 1080 * 1920 - 1, 1079 * 1920]])
    ref = O.filter_u8(img, win, filter, p, "exact", 4, pixels=pix, order=order)
    assert np.array_equal(idx.reshape(-1)[pix], ref["idx"])
    assert np.array_equal(out.reshape(-1, 3)[pix], ref["out"])


def test_vmf_every_tile_shape_and_order2_equals_ddf_p0(V):
    """Every FP32 tile shape gives the same VMF result; the order-2 VMF selects
    what the DDF with p = 0 selects (Eq. (3) at p = 0 is Eq. (1))."""
    from paper_1009_0958_gb300 import synth
    x = torch.from_numpy(synth.make_image(203, 317, 9, 0.2, rectangles=8)[1]).cuda()
    ref = V.filter(x, 5, "vmf", precision="fp64", order=1)
    try:
        for s in range(len(V.tile_shapes())):
            V.set_tuned_shape(5, "vmf", "exact", s)
            o, i = V.filter(x, 5, "vmf", precision="fp32", order=1)
            assert torch.equal(o, ref[0]) and torch.equal(i, ref[1])
    finally:
        V.set_tuned_shape(5, "vmf", "exact", 0)
    v2 = V.filter(x, 5, "vmf", precision="fp32", order=2)
    d0 = V.filter(x, 5, "ddf", 0.0, precision="fp32")
    assert torch.equal(v2[0], d0[0]) and torch.equal(v2[1], d0[1])


@pytest.mark.parametrize("order", [1, "inf"])
@pytest.mark.parametrize("p", [0.25, 0.3])
def test_ddf_orders_every_tile_shape(V, O, order, p):
    """The DDF with the Minkowski distance term of order 1 or infinity keeps
    raw slots (one plane buffer at 24x12 and 32x8): every FP32 tile shape
    equals the oracle on every pixel."""
    from paper_1009_0958_gb300 import synth
    img = synth.make_image(70, 101, 3, 0.2, rectangles=10)[1]
    ref = O.filter_u8(img, 5, "ddf", p, "exact", 4, order=order)
    try:
        for s in range(len(V.tile_shapes())):
            V.set_tuned_shape(5, "ddf", "exact", s)
            out, idx, _, (rc, ov) = run(V, img, 5, "ddf", p, order, "fp32")
            assert ov == 0
            assert np.array_equal(idx, ref["idx"]) and np.array_equal(out, ref["out"]), f"shape {s}"
    finally:
        V.set_tuned_shape(5, "ddf", "exact", 0)


def test_unsupported_combinations(V):
    x = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(V.VdfError):
        V.filter(x, 3, "ddf", 0.25, "rgb", order=1)
    with pytest.raises(V.VdfError):
        V.filter(x, 3, "vmf", order=3)
    with pytest.raises(V.VdfError):
        V.filter_f32(torch.zeros((1, 3, 8, 8), device="cuda"), 3, "vmf")
