"""Whole-image parity against the CPU oracle, every pixel.

* One benchmark frame (1920 x 1080, seed 100, 12 rectangles, 10% impulses),
  DDF 5x5, p = 1/4, exact arccos: the FP32 certified path in every tile shape
  and the plain FP64 path against the oracle on all 2,073,600 pixels; the
  oracle must flag no pixel gray (a real gap below its double-precision
  resolution) on that frame.
* The 512 x 512 sweep of the second configuration (BVDF and DDF p = 1/4, 3x3
  and 5x5, exact / Method 1 (q = 4) / Method 2, 20% impulses): both
  precisions against the oracle on every pixel.
* Every FP32 tile shape in Methods 1 and 2, since the autotuner may pick any
  of them for those modes, and every shape of the score-slot kernels (DDF
  5x5 at p = 1/4, 1/2, 3/4).

Selections are compared bit for bit: member index and RGB.
"""
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


def gpu(V, img, win, filter, p, dist, q, prec, shape=None):
    x = torch.from_numpy(img).cuda()
    M, N = img.shape[:2]
    if shape is not None:
        V.set_tuned_shape(win, filter, dist, shape)
    ws = V.alloc_workspace(M, N, prec)
    out, idx = V.filter(x, win, filter, p, dist, q, precision=prec, workspace=ws)
    torch.cuda.synchronize()
    stats = V.read_stats(ws) if ws is not None else None
    return out.cpu().numpy(), idx.cpu().numpy(), stats


def assert_same(out, idx, ref, what):
    bad = np.argwhere((idx != ref["idx"]) | (out != ref["out"]).any(axis=-1))
    assert bad.size == 0, f"{what}: {len(bad)} pixels differ from the oracle, first {bad[:5].tolist()}"


@pytest.fixture(scope="module")
def bench_frame(O):
    """The first frame the benchmark filters, and the oracle's result on it."""
    from paper_1009_0958_gb300 import synth
    img = synth.make_image(1080, 1920, 100, 0.10, rectangles=12)[1]
    return img, O.filter_u8(img, 5, "ddf", 0.25, "exact", 4)


def test_bench_frame_no_gray_pixels(O, bench_frame):
    _, ref = bench_frame
    assert not (ref["flags"] & O.FLAG_GRAY).any()


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_bench_frame_fp32_every_pixel(V, bench_frame, shape):
    img, ref = bench_frame
    out, idx, st = gpu(V, img, 5, "ddf", 0.25, "exact", 4, "fp32", shape=shape)
    V.set_tuned_shape(5, "ddf", "exact", 0)
    assert_same(out, idx, ref, f"FP32 shape {shape}")
    assert st["overflow"] == 0 and st["rechecked"] > 0 and st["structural_ties"] > 0


def test_bench_frame_fp64_every_pixel(V, bench_frame):
    img, ref = bench_frame
    out, idx, _ = gpu(V, img, 5, "ddf", 0.25, "exact", 4, "fp64")
    assert_same(out, idx, ref, "FP64")


@pytest.fixture(scope="module")
def sweep_image():
    from paper_1009_0958_gb300 import synth
    return synth.make_image(512, 512, 11, 0.20, rectangles=12)[1]


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", [("bvdf", 0.5), ("ddf", 0.25)])
@pytest.mark.parametrize("dist,q", [("exact", 4), ("minimax", 4), ("rgb", 4)])
def test_512_sweep_every_pixel(V, O, sweep_image, win, filter, p, dist, q):
    ref = O.filter_u8(sweep_image, win, filter, p, dist, q)
    assert not (ref["flags"] & O.FLAG_GRAY).any()
    for prec in ("fp64", "fp32"):
        out, idx, _ = gpu(V, sweep_image, win, filter, p, dist, q, prec)
        assert_same(out, idx, ref, prec)


@pytest.fixture(scope="module")
def small_image():
    from paper_1009_0958_gb300 import synth
    # 70 x 101: several tiles of every shape in each direction plus ragged tails
    return synth.make_image(70, 101, 1, 0.20, rectangles=12)[1]


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", [("bvdf", 0.5), ("ddf", 0.25), ("ddf", 0.3)])
@pytest.mark.parametrize("dist,q", [("minimax", 4), ("minimax", 3), ("rgb", 4)])
def test_tile_shapes_methods_1_and_2(V, O, small_image, shape, win, filter, p, dist, q):
    ref = O.filter_u8(small_image, win, filter, p, dist, q)
    out, idx, st = gpu(V, small_image, win, filter, p, dist, q, "fp32", shape=shape)
    V.set_tuned_shape(win, filter, dist, 0)
    assert_same(out, idx, ref, f"shape {shape}")
    assert st["overflow"] == 0


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("p", [0.25, 0.5, 0.75, 0.3])
@pytest.mark.parametrize("dist", ["exact", "rgb"])
def test_score_slot_kernels_every_shape(V, O, small_image, shape, p, dist):
    """The DDF 5x5 at p = 1/4, 1/2 and 3/4 runs with score slots (Omega^4 per
    slot), at p = 0.3 with raw slots (one plane buffer at 24x12 and 32x8), in
    every tile shape: every pixel equals the oracle."""
    ref = O.filter_u8(small_image, 5, "ddf", p, dist, 4)
    out, idx, st = gpu(V, small_image, 5, "ddf", p, dist, 4, "fp32", shape=shape)
    V.set_tuned_shape(5, "ddf", dist, 0)
    assert_same(out, idx, ref, f"shape {shape}")
    assert st["overflow"] == 0


def _edge_images():
    from tests.test_gpu_parity import EDGES
    return EDGES


@pytest.mark.parametrize("shape", [1, 2, 3])
@pytest.mark.parametrize("name", ["1x1", "1x57", "45x1", "2x2", "constant", "black", "checker", "collinear"])
@pytest.mark.parametrize("win,filter,p,dist", [(5, "ddf", 0.25, "exact"), (5, "bvdf", 0.5, "rgb"),
                                               (3, "ddf", 0.3, "minimax"), (5, "vmf", 0.5, "exact")])
def test_edge_images_every_shape(V, O, shape, name, win, filter, p, dist):
    """Edge images (single pixel, single row or column, constant, black,
    checkerboard, collinear) through every FP32 tile shape."""
    img = _edge_images()[name]
    ref = O.filter_u8(img, win, filter, p, dist, 4)
    d = "exact" if filter == "vmf" else dist
    out, idx, st = gpu(V, img, win, filter, p, d, 4, "fp32", shape=shape)
    V.set_tuned_shape(win, filter, d, 0)
    assert_same(out, idx, ref, f"shape {shape}")


@pytest.mark.parametrize("M,N", [(17, 29), (130, 61), (333, 250)])
def test_28x16_shape_ragged_sizes(V, O, M, N):
    """Odd widths (row pitches that are not multiples of 4 bytes) and ragged
    tails through the 28x16 tile shape."""
    from paper_1009_0958_gb300 import synth
    img = synth.make_image(M, N, 21, 0.2, rectangles=6)[1]
    ref = O.filter_u8(img, 5, "ddf", 0.25, "exact", 4)
    out, idx, st = gpu(V, img, 5, "ddf", 0.25, "exact", 4, "fp32", shape=3)
    V.set_tuned_shape(5, "ddf", "exact", 0)
    assert_same(out, idx, ref, "28x16 shape")
