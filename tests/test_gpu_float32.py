"""The FP32 certified path for float32 input (vdf_filter_f32 with the
fp32 precision): its terms within their bounds, and its selections equal to
the FP64 float path's (and the oracle's) on quantised, non-quantised and
adversarial float batches."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = 2.0 ** -24


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0958_gb300 import build, vdf
    build.build()
    return vdf


def exact_terms(pairs):
    """Reference in extended precision (at least 64-bit significands): the
    products of float32 values are exact, and so are the cross-product
    differences, since within a pair the components span at most 2^8."""
    x, y = pairs[:, :3].astype(np.longdouble), pairs[:, 3:].astype(np.longdouble)
    d = (x * y).sum(1)
    c = np.stack([x[:, 1] * y[:, 2] - x[:, 2] * y[:, 1], x[:, 2] * y[:, 0] - x[:, 0] * y[:, 2],
                  x[:, 0] * y[:, 1] - x[:, 1] * y[:, 0]], 1)
    th = np.arctan2(np.sqrt((c * c).sum(1)), d)
    zero = ((x * x).sum(1) == 0) | ((y * y).sum(1) == 0)
    th[zero] = np.pi / 2
    return th.astype(np.float64), np.sqrt(((x - y) ** 2).sum(1)).astype(np.float64)


def float_pairs(n, seed):
    rng = np.random.default_rng(seed)
    base = (2.0 ** -8 + (1 - 2.0 ** -8) * rng.random((n, 3))).astype(np.float32)
    scale = np.exp2(rng.integers(-40, 40, (n, 1))).astype(np.float32)
    x = base * scale
    kind = rng.integers(0, 4, n)
    y = ((2.0 ** -8 + (1 - 2.0 ** -8) * rng.random((n, 3))) * scale).astype(np.float32)
    # nearly collinear, nearly identical, scaled copies
    y[kind == 1] = (x[kind == 1] * np.float32(1.0 + 2 ** -20)).astype(np.float32)
    y[kind == 2] = np.nextafter(x[kind == 2], np.float32(np.inf))
    y[kind == 3] = (x[kind == 3] * np.float32(3.0)).astype(np.float32)
    p = np.concatenate([x, y], 1)
    p[rng.random(n) < 0.05, rng.integers(0, 6)] = 0.0
    return np.ascontiguousarray(p, dtype=np.float32)


def test_float_terms_within_bounds(V):
    pairs = float_pairs(300000, 1)
    ang, l2 = V.debug_fp32_terms_f32(torch.from_numpy(pairs).cuda())
    ang, l2 = ang.cpu().numpy().astype(np.float64), l2.cpu().numpy().astype(np.float64)
    assert not np.isnan(ang).any() and not np.isnan(l2).any()
    th, ref_l2 = exact_terms(pairs)
    assert np.all(np.abs(ang - th) <= 34 * U * th + 2.0 ** -58)   # kAngleFU
    assert np.all(np.abs(l2 - ref_l2) <= 8 * U * ref_l2 + 2.0 ** -62)
    assert np.all(ang[(pairs[:, :3] == pairs[:, 3:]).all(1) & (pairs[:, :3] != 0).any(1)] == 0.0)


def test_unsafe_pixels_are_flagged(V):
    bad = np.array([[-1, 0, 0, 1, 1, 1], [np.inf, 0, 0, 1, 1, 1], [1e-40, 0, 0, 1, 1, 1], [1e30, 1, 1, 1, 1, 1],
                    [1.0, 1e-25, 0, 1, 1, 1], [0, 0, 0, 1, 1, 1]], dtype=np.float32)
    ang, _ = V.debug_fp32_terms_f32(torch.from_numpy(bad).cuda())
    a = ang.cpu().numpy()
    assert np.isnan(a[:5]).all() and a[5] == np.float32(np.pi / 2)


def test_sqrt_approx_over_every_float(V):
    assert V.debug_sqrt_error() <= 2.0


def batch_quantised(B, M, N, seed, noise=0.10):
    from paper_1009_0958_gb300 import synth
    imgs = np.stack([synth.make_image(M, N, seed + b, noise, rectangles=4)[1] for b in range(B)])
    return synth.to_float_nchw(imgs)


def batch_continuous(B, M, N, seed):
    """Non-quantised floats: smooth fields of random scale, flat patches,
    exact duplicates, collinear scaled copies and impulses."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.linspace(0, 1, M), np.linspace(0, 1, N), indexing="ij")
    out = np.empty((B, 3, M, N), dtype=np.float32)
    for b in range(B):
        for c in range(3):
            f = 0.5 + 0.2 * np.sin(2 * np.pi * (rng.uniform(-2, 2) * xx + rng.uniform(-2, 2) * yy) + rng.uniform(0, 6))
            out[b, c] = (f * rng.uniform(0.5, 2.0)).astype(np.float32)
        r0, c0 = rng.integers(0, M // 2), rng.integers(0, N // 2)
        out[b, :, r0:r0 + M // 4, c0:c0 + N // 4] = rng.random((3, 1, 1)).astype(np.float32)
        out[b, :, r0 + 2:r0 + 6, c0 + 2:c0 + 6] *= np.float32(2.0)    # collinear copies
        imp = rng.random((M, N)) < 0.1
        out[b][:, imp] = rng.random((3, imp.sum())).astype(np.float32)
    return out


CASES = [(3, "ddf", 0.25), (5, "ddf", 0.25), (3, "bvdf", 0.5), (5, "bvdf", 0.5), (5, "ddf", 0.3), (3, "ddf", 1.0)]


@pytest.mark.parametrize("win,filter,p", CASES)
@pytest.mark.parametrize("kind", ["quantised", "continuous"])
def test_fp32_equals_fp64_float_path(V, win, filter, p, kind):
    x = batch_quantised(3, 97, 131, 5) if kind == "quantised" else batch_continuous(3, 97, 131, 5)
    xt = torch.from_numpy(x).cuda()
    y32, i32 = V.filter_f32(xt, win, filter, p, precision="fp32")
    y64, i64 = V.filter_f32(xt, win, filter, p, precision="fp64")
    assert torch.equal(i32, i64) and torch.equal(y32, y64)


def test_fp32_float_matches_oracle(V):
    import oracle
    oracle.build()
    x = batch_continuous(2, 41, 53, 9)
    ref = oracle.filter_f32(x, 5, "ddf", 0.25, "exact")
    assert not (ref["flags"] & oracle.FLAG_GRAY).any()
    y, idx = V.filter_f32(torch.from_numpy(x).cuda(), 5, "ddf", 0.25, precision="fp32")
    assert np.array_equal(idx.cpu().numpy(), ref["idx"])
    assert np.array_equal(y.cpu().numpy(), ref["out"])


def test_unsafe_tiles_equal_fp64(V):
    x = batch_continuous(2, 64, 80, 12)
    x[0, 0, 10, 10] = -0.5            # negative
    x[0, :, 40, 50] = 0.0             # black pixel (safe)
    x[1, 1, 5, 70] = 1e-41            # subnormal
    x[1, :, 60, 3] = np.float32(1e25)  # extreme magnitude
    xt = torch.from_numpy(x).cuda()
    for win, filt, p in [(3, "ddf", 0.25), (5, "bvdf", 0.5)]:
        y32, i32 = V.filter_f32(xt, win, filt, p, precision="fp32")
        y64, i64 = V.filter_f32(xt, win, filt, p, precision="fp64")
        assert torch.equal(i32, i64) and torch.equal(y32, y64)


def test_full_size_differentiable_batch(V):
    """32 x 3 x 512 x 512, DDF 3x3: the FP32 forward equals the FP64 one on
    every pixel, and the autograd function accepts it."""
    from paper_1009_0958_gb300.autograd import DirectionalFilterFn
    x = torch.from_numpy(batch_quantised(32, 512, 512, 40)).cuda()
    y32, i32 = V.filter_f32(x, 3, "ddf", 0.25, precision="fp32")
    y64, i64 = V.filter_f32(x, 3, "ddf", 0.25, precision="fp64")
    assert torch.equal(i32, i64) and torch.equal(y32, y64)
    xr = x[:2].clone().requires_grad_(True)
    y, idx = DirectionalFilterFn.apply(xr, 3, "ddf", 0.25, "exact", 4, "fp32")
    y.sum().backward()
    assert torch.equal(idx, i32[:2]) and xr.grad is not None
