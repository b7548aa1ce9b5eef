"""The differentiable float32 path: forward parity with the oracle, backward
against a reference gradient built from the oracle's indices, and finite
differences where the selection is locally constant."""
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


def batch(B, M, N, seed, noise=0.10):
    from paper_1009_0958_gb300 import synth
    imgs = np.stack([synth.make_image(M, N, seed + b, noise)[1] for b in range(B)])
    return synth.to_float_nchw(imgs)


def reference_grad(gy, idx, win):
    """Scatter-add of grad_y to the sources chosen by the oracle's indices."""
    B, C, M, N = gy.shape
    R = win // 2
    gx = np.zeros_like(gy, dtype=np.float64)
    yy, xx = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
    for b in range(B):
        i = idx[b].astype(np.int64)
        sy = np.clip(yy + i // win - R, 0, M - 1)
        sx = np.clip(xx + i % win - R, 0, N - 1)
        for c in range(C):
            np.add.at(gx[b, c], (sy, sx), gy[b, c].astype(np.float64))
    return gx


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", [("ddf", 0.25), ("bvdf", 0.5), ("ddf", 0.5)])
def test_forward_matches_oracle(V, O, win, filter, p):
    x = batch(2, 37, 45, 3)
    ref = O.filter_f32(x, win, filter, p, "exact")
    assert not (ref["flags"] & O.FLAG_GRAY).any()
    y, idx = V.filter_f32(torch.from_numpy(x).cuda(), win, filter, p, "exact", precision="fp64")
    assert np.array_equal(idx.cpu().numpy(), ref["idx"])
    assert np.array_equal(y.cpu().numpy(), ref["out"])


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("shape", [(2, 40, 57), (1, 3, 4), (3, 1, 9)])
def test_backward_matches_oracle_index_gradient(V, O, win, shape):
    from paper_1009_0958_gb300.autograd import DirectionalFilterFn
    B, M, N = shape
    x = batch(B, M, N, 7, noise=0.2)
    ref = O.filter_f32(x, win, "ddf", 0.25, "exact")
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    y, idx = DirectionalFilterFn.apply(xt, win, "ddf", 0.25, "exact", 4, "fp64")
    gy = torch.randn_like(y)
    y.backward(gy)
    want = reference_grad(gy.cpu().numpy(), ref["idx"], win)
    got = xt.grad.cpu().numpy().astype(np.float64)
    assert np.allclose(got, want, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("shape", [(2, 150, 260), (1, 37, 132), (1, 64, 128), (3, 9, 4), (1, 70, 57)])
def test_backward_random_index_maps(V, win, shape):
    """The gradient gather on random index maps, every pixel against a numpy
    scatter: strips and row segments with ragged tails (the streaming form for
    widths that are multiples of 4, the staged form otherwise), and bytes
    outside 0..n-1, which select nothing."""
    B, M, N = shape
    rng = np.random.default_rng(M * N + win)
    n = win * win
    idx = rng.integers(0, n, (B, M, N)).astype(np.int8)
    bad = rng.random((B, M, N)) < 0.02
    idx[bad] = rng.choice(np.array([-1, n, 127], dtype=np.int8), bad.sum())
    gy = rng.standard_normal((B, 3, M, N)).astype(np.float32)
    got = V.backward_f32(torch.from_numpy(gy).cuda(), torch.from_numpy(idx).cuda(), win).cpu().numpy()
    R = win // 2
    want = np.zeros((B, 3, M, N), np.float64)
    yy, xx = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
    for b in range(B):
        i = idx[b].astype(np.int64)
        ok = (i >= 0) & (i < n)
        sy = np.clip(yy + i // win - R, 0, M - 1)[ok]
        sx = np.clip(xx + i % win - R, 0, N - 1)[ok]
        for c in range(3):
            np.add.at(want[b, c], (sy, sx), gy[b, c][ok].astype(np.float64))
    assert np.allclose(got, want, rtol=1e-5, atol=1e-5)


def test_backward_deterministic(V):
    x = torch.from_numpy(batch(2, 64, 80, 11)).cuda()
    y, idx = V.filter_f32(x, 3, "ddf", 0.25)
    gy = torch.randn_like(y)
    a = V.backward_f32(gy, idx, 3)
    b = V.backward_f32(gy, idx, 3)
    assert torch.equal(a, b)


def test_finite_differences(V):
    """Central differences (eps = 1e-3) of L = sum(w * y) at random input
    entries whose perturbation leaves every selection unchanged (the pixel
    and all windows containing it are away from ties) equal the gradient."""
    from paper_1009_0958_gb300.autograd import DirectionalFilterFn
    torch.manual_seed(0)
    x = torch.from_numpy(batch(2, 48, 64, 21)).cuda().double().float()
    w = torch.randn((2, 3, 48, 64), device="cuda", dtype=torch.float64)
    xt = x.clone().requires_grad_(True)
    y, idx0 = DirectionalFilterFn.apply(xt, 3, "ddf", 0.25, "exact", 4, "fp64")
    (y.double() * w).sum().backward()
    g = xt.grad.double()
    rng = np.random.default_rng(5)
    eps = 1e-3
    checked = 0
    for _ in range(200):
        b, c, i, j = int(rng.integers(2)), int(rng.integers(3)), int(rng.integers(48)), int(rng.integers(64))
        vals = []
        ok = True
        for s in (+1, -1):
            xp = x.clone()
            xp[b, c, i, j] += s * eps
            yp, ip = V.filter_f32(xp, 3, "ddf", 0.25)
            ok = ok and torch.equal(ip, idx0)
            vals.append(float((yp.double() * w).sum()))
        if not ok:
            continue
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - float(g[b, c, i, j])) <= 1e-3 * max(1.0, abs(fd)), (b, c, i, j, fd, float(g[b, c, i, j]))
        checked += 1
    assert checked >= 100


def test_full_size_batch_32x512x512_sampled(V, O):
    """The differentiable workload at full size (32 x 3 x 512 x 512, DDF 3x3):
    forward selections at 3000 sampled pixels equal the oracle's, and the
    gradient at the sampled pixels' own positions equals the gather of
    grad_y over the oracle's sources (the sources of all pixels around it are
    taken from the GPU map, checked against the oracle on a strip)."""
    from paper_1009_0958_gb300 import synth
    from paper_1009_0958_gb300.autograd import DirectionalFilterFn
    B, M, N, win = 32, 512, 512, 3
    field = np.stack([synth.make_image(M, N, 40 + b, 0.10)[1] for b in range(B)])
    x = torch.from_numpy(synth.to_float_nchw(field)).cuda().requires_grad_(True)
    y, idx = DirectionalFilterFn.apply(x, win, "ddf", 0.25, "exact", 4, "fp64")
    rng = np.random.default_rng(3)
    pix = rng.integers(0, B * M * N, 3000)
    xn = x.detach().cpu().numpy()
    ref = O.filter_f32(xn, win, "ddf", 0.25, "exact", pixels=pix)
    got_idx = idx.cpu().numpy().reshape(-1)[pix]
    assert np.array_equal(got_idx, ref["idx"])
    yn = y.detach().cpu().numpy()
    got_out = yn.transpose(0, 2, 3, 1).reshape(-1, 3)[pix]
    assert np.array_equal(got_out, ref["out"])
    # one full image strip through the oracle, then the gradient there
    strip = np.arange(0, 6 * N) + 5 * M * N            # image 5, rows 0..5
    ref_s = O.filter_f32(xn, win, "ddf", 0.25, "exact", pixels=strip)
    assert np.array_equal(idx.cpu().numpy().reshape(-1)[strip], ref_s["idx"])
    gy = torch.randn_like(y)
    y.backward(gy)
    gx = x.grad.cpu().numpy()
    want = reference_grad(gy.cpu().numpy()[5:6, :, :8], idx.cpu().numpy()[5:6, :8], win)
    # rows 0..3 of image 5 only receive contributions from rows 0..4 (all in the strip)
    assert np.allclose(gx[5, :, :4], want[0, :, :4], rtol=1e-6, atol=1e-6)
