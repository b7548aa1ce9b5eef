"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Selections (uint8 output and member index) must equal the oracle bit for bit;
FP64 aggregates must agree within 1e-12 relative.  The FP32 path (certified
scores + FP64 recheck) must select exactly what the FP64 path selects.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DISTS = [("exact", 4), ("minimax", 4), ("minimax", 3), ("minimax", 2), ("rgb", 4)]
FILTERS = [("bvdf", 0.5), ("ddf", 0.25), ("ddf", 0.5), ("ddf", 0.3)]


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


def images():
    from paper_1009_0958_gb300 import synth
    # 70 x 101: several 32x16 / 16x12 tiles in each direction plus ragged tails
    yield "rect20", synth.make_image(70, 101, 1, 0.20, rectangles=12)[1]
    yield "field10", synth.make_image(53, 77, 2, 0.10)[1]


IMAGES = dict(images())


def run(V, img, win, filter, p, dist, q, prec, agg=False):
    x = torch.from_numpy(img).cuda()
    M, N = img.shape[:2]
    ag = torch.zeros((M, N, win * win, 2), dtype=torch.float64, device="cuda") if agg else None
    ws = V.alloc_workspace(M, N, prec)
    out, idx = V.filter(x, win, filter, p, dist, q, precision=prec, agg=ag, workspace=ws)
    torch.cuda.synchronize()
    stats = V.workspace_stats(ws) if ws is not None else (0, 0)
    return out.cpu().numpy(), idx.cpu().numpy(), (ag.cpu().numpy() if agg else None), stats


@pytest.mark.parametrize("name", list(IMAGES))
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", FILTERS)
@pytest.mark.parametrize("dist,q", DISTS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_selection_matches_oracle(V, O, name, win, filter, p, dist, q, prec):
    img = IMAGES[name]
    ref = O.filter_u8(img, win, filter, p, dist, q)
    assert not (ref["flags"] & O.FLAG_GRAY).any()
    out, idx, _, (rechecked, overflow) = run(V, img, win, filter, p, dist, q, prec)
    bad = np.argwhere(idx != ref["idx"])
    assert bad.size == 0, f"{len(bad)} index mismatches, first {bad[:5].tolist()}"
    assert np.array_equal(out, ref["out"])
    assert overflow == 0


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", [("bvdf", 0.5), ("ddf", 0.25)])
@pytest.mark.parametrize("dist,q", [("exact", 4), ("minimax", 4), ("rgb", 4)])
def test_fp64_aggregates_match_oracle(V, O, win, filter, p, dist, q):
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(37, 41, 3, 0.15, rectangles=5)
    ref = O.filter_u8(img, win, filter, p, dist, q, want_agg=True)
    _, idx, ag, _ = run(V, img, win, filter, p, dist, q, "fp64", agg=True)
    a, b = ag, ref["agg"]
    cols = [0, 1] if filter == "ddf" else [0]
    for c in cols:
        err = np.abs(a[..., c] - b[..., c]) / np.maximum(np.abs(b[..., c]), 1.0)
        assert err.max() <= 1e-12, err.max()


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", FILTERS + [("ddf", 0.0), ("ddf", 1.0), ("ddf", 0.75), ("ddf", 0.9)])
@pytest.mark.parametrize("dist,q", DISTS)
def test_fp32_equals_fp64_larger(V, win, filter, p, dist, q):
    """Both precisions select the same member everywhere (512 x 512, 20% noise)."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(512, 512, 11, 0.20, rectangles=12)
    o64, i64, _, _ = run(V, img, win, filter, p, dist, q, "fp64")
    o32, i32, _, (rc, ov) = run(V, img, win, filter, p, dist, q, "fp32")
    assert np.array_equal(i32, i64) and np.array_equal(o32, o64)
    assert ov == 0
    assert rc < 0.05 * img.shape[0] * img.shape[1]


def edge_images():
    rng = np.random.default_rng(0)
    yield "1x1", rng.integers(0, 256, (1, 1, 3)).astype(np.uint8)
    yield "1x57", rng.integers(0, 256, (1, 57, 3)).astype(np.uint8)
    yield "45x1", rng.integers(0, 256, (45, 1, 3)).astype(np.uint8)
    yield "2x2", rng.integers(0, 256, (2, 2, 3)).astype(np.uint8)
    yield "constant", np.full((20, 35, 3), 77, np.uint8)
    yield "black", np.zeros((18, 33, 3), np.uint8)
    g = rng.integers(0, 256, (19, 34, 1)).astype(np.uint8)
    yield "gray", np.repeat(g, 3, axis=2)
    b = rng.integers(0, 256, (21, 40, 3)).astype(np.uint8)
    b[rng.random((21, 40)) < 0.3] = 0
    yield "black_specks", b
    c = np.zeros((24, 36, 3), np.uint8)
    c[::2, ::2] = (255, 0, 0)
    c[1::2, 1::2] = (255, 0, 0)
    c[c.sum(2) == 0] = (0, 255, 0)
    yield "checker", c
    t = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 0]], np.uint8)[rng.integers(0, 3, (30, 30))] * 100
    yield "three_colours", t
    k = rng.integers(1, 5, (25, 31, 1)).astype(np.uint8)
    yield "collinear", (np.array([10, 20, 30], np.uint8)[None, None, :] * k).astype(np.uint8)


EDGES = dict(edge_images())


@pytest.mark.parametrize("name", list(EDGES))
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", [("bvdf", 0.5), ("ddf", 0.25)])
@pytest.mark.parametrize("dist,q", [("exact", 4), ("minimax", 3), ("rgb", 4)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_cases(V, O, name, win, filter, p, dist, q, prec):
    img = EDGES[name]
    ref = O.filter_u8(img, win, filter, p, dist, q)
    out, idx, _, _ = run(V, img, win, filter, p, dist, q, prec)
    assert np.array_equal(idx, ref["idx"]) and np.array_equal(out, ref["out"])


@pytest.mark.parametrize("filter,p,win", [("ddf", 0.25, 5), ("bvdf", 0.5, 3), ("ddf", 0.25, 3)])
def test_full_size_1080p_sampled(V, O, filter, p, win):
    """1920 x 1080 in the benchmark's launch configuration; the oracle checks
    a sample of 4000 pixels one by one."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(1080, 1920, 7, 0.10, rectangles=12)
    out, idx, _, (rc, ov) = run(V, img, win, filter, p, "exact", 4, "fp32")
    rng = np.random.default_rng(1)
    pix = np.concatenate([rng.integers(0, 1080 * 1920, 3990), [0, 1919, 1080 * 1920 - 1, 1079 * 1920]])
    ref = O.filter_u8(img, win, filter, p, "exact", 4, pixels=pix)
    assert np.array_equal(idx.reshape(-1)[pix], ref["idx"])
    assert np.array_equal(out.reshape(-1, 3)[pix], ref["out"])
    assert ov == 0


def test_full_size_4k_20pct_noise(V, O):
    """The precision stress case: DDF 5x5 (p = 0.25) on 3840 x 2160 with 20%
    impulsive noise.  The FP32 path with its FP64 recheck equals the plain
    FP64 path on every pixel, and the oracle on 4000 sampled pixels."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(2160, 3840, 11, 0.20, rectangles=12)
    out, idx, _, (rc, ov) = run(V, img, 5, "ddf", 0.25, "exact", 4, "fp32")
    out64, idx64, _, _ = run(V, img, 5, "ddf", 0.25, "exact", 4, "fp64")
    assert ov == 0 and rc > 0
    assert np.array_equal(idx, idx64) and np.array_equal(out, out64)
    rng = np.random.default_rng(2)
    pix = np.concatenate([rng.integers(0, 2160 * 3840, 3990), [0, 3839, 2160 * 3840 - 1, 2159 * 3840]])
    ref = O.filter_u8(img, 5, "ddf", 0.25, "exact", 4, pixels=pix)
    assert np.array_equal(idx.reshape(-1)[pix], ref["idx"])
    assert np.array_equal(out.reshape(-1, 3)[pix], ref["out"])


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", [("bvdf", 0.5), ("ddf", 0.25), ("ddf", 0.5), ("ddf", 0.3), ("ddf", 1.0)])
@pytest.mark.parametrize("dist,q", [("exact", 4), ("minimax", 4), ("minimax", 3), ("rgb", 4)])
def test_fp32_bounds_hold(V, win, filter, p, dist, q):
    """The FP32 scores lie within half their certified bound (the bound
    carries a factor-2 safety margin) of the FP64 scores."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(200, 300, 13, 0.20, rectangles=12)
    x = torch.from_numpy(img).cuda()
    fe = V.debug_fp32_scores(x, win, filter, p, dist, q).cpu().numpy().astype(np.float64)
    _, _, ag, _ = run(V, img, win, filter, p, dist, q, "fp64", agg=True)
    sa, sl = ag[..., 0], ag[..., 1]
    a = 4 * p
    if filter == "bvdf":
        f64, zero = sa, None
    elif a == round(a):                       # Omega^4 form
        f64 = np.maximum(sa, 0) ** int(a) * sl ** (4 - int(a))
        zero = 0.0
    else:
        with np.errstate(divide="ignore"):
            f64 = (p * np.log2(np.maximum(sa, 0)) if p > 0 else 0) + ((1 - p) * np.log2(sl) if p < 1 else 0)
        zero = -np.inf
    f32, E = fe[..., 0], fe[..., 1]
    certain = np.isfinite(E)                  # Method 1 flags sums too close to 0 with E = inf
    finite = np.isfinite(f64) & certain
    if zero is not None:
        assert np.all(((f32 == zero) == (f64 == zero))[certain])
    err = np.abs(f32[finite] - f64[finite])
    assert np.all(err <= 0.5 * E[finite] + 1e-30), (err / np.maximum(E[finite], 1e-30)).max()


def test_host_buffer_path_equals_device_path(V):
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(300, 500, 4, 0.1, rectangles=6)
    o_dev, i_dev, _, _ = run(V, img, 5, "ddf", 0.25, "exact", 4, "fp32")
    h = torch.from_numpy(img).pin_memory()
    oh = torch.empty_like(h).pin_memory()
    ih = torch.empty(img.shape[:2], dtype=torch.int8).pin_memory()
    V.filter_host(h, 5, "ddf", 0.25, "exact", 4, "fp32", oh, ih)
    assert np.array_equal(oh.numpy(), o_dev) and np.array_equal(ih.numpy(), i_dev)


def test_two_stream_pipeline_equals_sequential(V):
    """The two stages on two streams with alternating workspaces (the FP64
    recheck of frame i overlapping the FP32 pass of frame i+1) give exactly
    the single-call results."""
    from paper_1009_0958_gb300 import synth
    frames = [torch.from_numpy(synth.make_image(400, 640, 60 + k, 0.15, rectangles=8)[1]).cuda() for k in range(6)]
    ref = [V.filter(f, 5, "ddf", 0.25, precision="fp32") for f in frames]
    outs = [torch.empty_like(f) for f in frames]
    idxs = [torch.empty(f.shape[:2], dtype=torch.int8, device="cuda") for f in frames]
    ws = [V.alloc_workspace(400, 640, "fp32") for _ in range(2)]
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    done = [torch.cuda.Event() for _ in frames]
    for k, f in enumerate(frames):
        if k >= 2:
            main.wait_event(done[k - 2])
        V.fp32_pass(f, outs[k], idxs[k], ws[k % 2], 5, "ddf", 0.25, stream=main)
        passed = torch.cuda.Event()
        passed.record(main)
        side.wait_event(passed)
        V.fp64_recheck(f, outs[k], idxs[k], ws[k % 2], 5, "ddf", 0.25, stream=side)
        done[k].record(side)
    torch.cuda.synchronize()
    for k in range(len(frames)):
        assert torch.equal(outs[k], ref[k][0]) and torch.equal(idxs[k], ref[k][1])
