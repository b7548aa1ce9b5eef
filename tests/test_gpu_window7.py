"""The 7x7 window (Section II's sqrt(n) x sqrt(n) window at n = 49) through
the C ABI against the CPU oracle: selections bit for bit in both precisions,
every filter kind, distance mode and Minkowski order; FP64 aggregates within
1e-12; edge images; the FP32 path equal to the FP64 path on a larger image and
the oracle on sampled pixels of a full 1920 x 1080 frame."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [("bvdf", 0.5, "exact", 4, 2), ("bvdf", 0.5, "minimax", 4, 2), ("bvdf", 0.5, "minimax", 3, 2),
         ("bvdf", 0.5, "rgb", 4, 2), ("ddf", 0.25, "exact", 4, 2), ("ddf", 0.3, "exact", 4, 2),
         ("ddf", 0.5, "minimax", 4, 2), ("ddf", 0.25, "rgb", 4, 2), ("ddf", 0.25, "exact", 4, 1),
         ("ddf", 0.25, "exact", 4, "inf"), ("vmf", 0.5, "exact", 4, 2), ("vmf", 0.5, "exact", 4, 1),
         ("vmf", 0.5, "exact", 4, "inf")]


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
    # 70 x 101 and 53 x 77: ragged sizes, flat rectangles (ties) and impulses
    return {"rect20": synth.make_image(70, 101, 1, 0.20, rectangles=12)[1],
            "field10": synth.make_image(53, 77, 2, 0.10)[1]}


IMAGES = images()


def run(V, img, filter, p, dist, q, order, prec, agg=False):
    x = torch.from_numpy(img).cuda()
    M, N = img.shape[:2]
    ag = torch.zeros((M, N, 49, 2), dtype=torch.float64, device="cuda") if agg else None
    ws = V.alloc_workspace(M, N, prec)
    out, idx = V.filter(x, 7, filter, p, dist, q, precision=prec, agg=ag, workspace=ws, order=order)
    torch.cuda.synchronize()
    st = V.read_stats(ws) if ws is not None else None
    return out.cpu().numpy(), idx.cpu().numpy(), (ag.cpu().numpy() if agg else None), st


@pytest.mark.parametrize("name", list(IMAGES))
@pytest.mark.parametrize("filter,p,dist,q,order", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_window7_matches_oracle(V, O, name, filter, p, dist, q, order, prec):
    img = IMAGES[name]
    ref = O.filter_u8(img, 7, filter, p, dist, q, order=order)
    assert not (ref["flags"] & O.FLAG_GRAY).any()
    out, idx, _, st = run(V, img, filter, p, dist, q, order, prec)
    bad = np.argwhere(idx != ref["idx"])
    assert bad.size == 0, f"{len(bad)} index mismatches, first {bad[:5].tolist()}"
    assert np.array_equal(out, ref["out"])
    if st is not None:
        assert st["overflow"] == 0


@pytest.mark.parametrize("filter,p,dist,q,order", [c for c in CASES if c[4] == 2])
def test_window7_fp64_aggregates(V, O, filter, p, dist, q, order):
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(37, 41, 3, 0.15, rectangles=5)
    ref = O.filter_u8(img, 7, filter, p, dist, q, want_agg=True, order=order)
    _, _, ag, _ = run(V, img, filter, p, dist, q, order, "fp64", agg=True)
    cols = {"ddf": [0, 1], "bvdf": [0], "vmf": [1]}[filter]
    for c in cols:
        err = np.abs(ag[..., c] - ref["agg"][..., c]) / np.maximum(np.abs(ref["agg"][..., c]), 1.0)
        assert err.max() <= 1e-12, err.max()


def edge_images():
    rng = np.random.default_rng(0)
    yield "1x1", rng.integers(0, 256, (1, 1, 3)).astype(np.uint8)
    yield "1x57", rng.integers(0, 256, (1, 57, 3)).astype(np.uint8)
    yield "45x1", rng.integers(0, 256, (45, 1, 3)).astype(np.uint8)
    yield "3x3", rng.integers(0, 256, (3, 3, 3)).astype(np.uint8)
    yield "constant", np.full((20, 35, 3), 77, np.uint8)
    yield "black", np.zeros((18, 33, 3), np.uint8)
    g = rng.integers(0, 256, (19, 34, 1)).astype(np.uint8)
    yield "gray", np.repeat(g, 3, axis=2)
    b = rng.integers(0, 256, (21, 40, 3)).astype(np.uint8)
    b[rng.random((21, 40)) < 0.3] = 0
    yield "black_specks", b
    t = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 0]], np.uint8)[rng.integers(0, 3, (30, 30))] * 100
    yield "three_colours", t
    k = rng.integers(1, 5, (25, 31, 1)).astype(np.uint8)
    yield "collinear", (np.array([10, 20, 30], np.uint8)[None, None, :] * k).astype(np.uint8)


EDGES = dict(edge_images())


@pytest.mark.parametrize("name", list(EDGES))
@pytest.mark.parametrize("filter,p,dist,q,order", [("bvdf", 0.5, "exact", 4, 2), ("ddf", 0.25, "exact", 4, 2),
                                                   ("ddf", 0.25, "minimax", 3, 2), ("bvdf", 0.5, "rgb", 4, 2),
                                                   ("vmf", 0.5, "exact", 4, 1)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_window7_edge_cases(V, O, name, filter, p, dist, q, order, prec):
    img = EDGES[name]
    ref = O.filter_u8(img, 7, filter, p, dist, q, order=order)
    out, idx, _, _ = run(V, img, filter, p, dist, q, order, prec)
    assert np.array_equal(idx, ref["idx"]) and np.array_equal(out, ref["out"])


@pytest.mark.parametrize("filter,p,dist", [("ddf", 0.25, "exact"), ("bvdf", 0.5, "exact"), ("ddf", 0.25, "rgb")])
def test_window7_fp32_equals_fp64_512(V, filter, p, dist):
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(512, 512, 11, 0.20, rectangles=12)
    o64, i64, _, _ = run(V, img, filter, p, dist, 4, 2, "fp64")
    o32, i32, _, st = run(V, img, filter, p, dist, 4, 2, "fp32")
    assert np.array_equal(i32, i64) and np.array_equal(o32, o64)
    assert st["overflow"] == 0 and st["structural_ties"] > 0
    assert st["rechecked"] < 0.05 * 512 * 512


def test_window7_full_size_sampled(V, O):
    """1920 x 1080 DDF 7x7 (p = 1/4) in FP32; the oracle checks 3000 pixels."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(1080, 1920, 7, 0.10, rectangles=12)
    out, idx, _, st = run(V, img, "ddf", 0.25, "exact", 4, 2, "fp32")
    rng = np.random.default_rng(3)
    pix = np.concatenate([rng.integers(0, 1080 * 1920, 2996), [0, 1919, 1080 * 1920 - 1, 1079 * 1920]])
    ref = O.filter_u8(img, 7, "ddf", 0.25, "exact", 4, pixels=pix)
    assert np.array_equal(idx.reshape(-1)[pix], ref["idx"])
    assert np.array_equal(out.reshape(-1, 3)[pix], ref["out"])
    assert st["overflow"] == 0


def test_window7_noalloc_equals_workspace_path(V):
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(300, 400, 12, 0.20, rectangles=8)
    x = torch.from_numpy(img).cuda()
    o_ref, i_ref = V.filter(x, 7, "ddf", 0.25, precision="fp32")
    o, i = V.filter_noalloc(x, 7, "ddf", 0.25)
    torch.cuda.synchronize()
    assert torch.equal(o, o_ref) and torch.equal(i, i_ref)
