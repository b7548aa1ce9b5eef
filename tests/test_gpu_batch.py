"""Batches of uneven images (one launch per configuration, in the per-item
and the persistent work-queue forms), CUDA-graph replays and the tile-shape
autotuner: every result must equal the single-image path (and the oracle on
small images) bit for bit."""
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


@pytest.fixture(autouse=True)
def reset_shapes(V):
    yield
    for win in (3, 5):
        for f in ("bvdf", "ddf"):
            for d in ("exact", "minimax", "rgb"):
                V.set_tuned_shape(win, f, d, 0)


def batch_items(seed, count, hi=300, extra=True):
    from paper_1009_0958_gb300 import synth
    rng = np.random.default_rng(seed)
    shapes = synth.batch_shapes(count, seed, lo=8, hi=hi)
    if extra:
        shapes += [(1, 1), (1, 40), (40, 1), (2, 3), (17, 33)]
    items = []
    for k, (M, N) in enumerate(shapes):
        _, img = synth.make_image(M, N, seed * 1000 + k, 0.15, rectangles=3)
        items.append(dict(img=torch.from_numpy(img).cuda(), win=int(rng.choice([3, 5])),
                          filter=str(rng.choice(["bvdf", "ddf"])), p=float(rng.choice([0.0, 0.25, 0.5, 0.75, 1.0]))))
    return items


def check_against_single(V, plan, prec="fp32", dist="exact", q=4):
    for it in plan.items:
        o, i = V.filter(it["img"], it["win"], it["filter"], it["p"], dist, q, precision=prec)
        assert torch.equal(o, it["out"]) and torch.equal(i, it["index"])


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("shapes", [(0, 0, 0, 0), (1, 2, 2, 1), (2, 1, 0, 2), (3, 3, 3, 3)])
def test_batch_equals_single_image_calls(V, shapes, persistent):
    for (win, f), s in zip([(3, "bvdf"), (3, "ddf"), (5, "bvdf"), (5, "ddf")], shapes):
        V.set_tuned_shape(win, f, "exact", s)
    plan = V.Plan(batch_items(1, 24), persistent=persistent)
    plan.run()
    torch.cuda.synchronize()
    check_against_single(V, plan, "fp32")
    check_against_single(V, plan, "fp64")
    rechecked, overflow = plan.stats()
    assert overflow == 0 and rechecked > 0


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("dist,q", [("minimax", 4), ("minimax", 3), ("rgb", 4)])
@pytest.mark.parametrize("shapes", [(0, 0, 0, 0), (1, 2, 3, 1)])
def test_batch_methods_1_and_2(V, dist, q, shapes, persistent):
    """The paper's two speed-up methods (Section 2.1, Table 1; Section 2.2,
    Eq. (7)) through the batch: every image equals the single-image path in
    both precisions and the oracle."""
    import oracle
    oracle.build()
    for (win, f), s in zip([(3, "bvdf"), (3, "ddf"), (5, "bvdf"), (5, "ddf")], shapes):
        V.set_tuned_shape(win, f, dist, s)
    plan = V.Plan(batch_items(4, 16, hi=160), dist=dist, q=q, persistent=persistent)
    plan.run()
    torch.cuda.synchronize()
    check_against_single(V, plan, "fp32", dist, q)
    check_against_single(V, plan, "fp64", dist, q)
    for it in plan.items[:8]:
        ref = oracle.filter_u8(it["img"].cpu().numpy(), it["win"], it["filter"], it["p"], dist, q)
        assert np.array_equal(it["index"].cpu().numpy(), ref["idx"])
    assert plan.stats()[1] == 0


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_matches_oracle_on_small_images(V, persistent):
    import oracle
    oracle.build()
    plan = V.Plan(batch_items(2, 10, hi=48), persistent=persistent)
    plan.run()
    torch.cuda.synchronize()
    for it in plan.items:
        ref = oracle.filter_u8(it["img"].cpu().numpy(), it["win"], it["filter"], it["p"], "exact")
        assert np.array_equal(it["index"].cpu().numpy(), ref["idx"])
        assert np.array_equal(it["out"].cpu().numpy(), ref["out"])


def test_graph_replay_tracks_input_contents(V):
    from paper_1009_0958_gb300 import synth
    items = batch_items(3, 12)
    plan = V.Plan(items)
    plan.graph_launch()
    torch.cuda.synchronize()
    check_against_single(V, plan)
    # new contents in the same buffers: the captured graph sees them
    for k, it in enumerate(plan.items):
        M, N = it["img"].shape[:2]
        it["img"].copy_(torch.from_numpy(synth.make_image(M, N, 777 + k, 0.2, rectangles=2)[1]).cuda())
    plan.graph_launch()
    plan.graph_launch()
    torch.cuda.synchronize()
    check_against_single(V, plan)
    # switching the form drops the captured graph; the new one gives the same
    for it in plan.items:
        it["out"].zero_()
    plan.set_persistent(True)
    plan.graph_launch()
    torch.cuda.synchronize()
    check_against_single(V, plan)


@pytest.mark.parametrize("win,filter", [(5, "ddf"), (3, "bvdf")])
def test_every_tile_shape_gives_the_same_result(V, win, filter):
    from paper_1009_0958_gb300 import synth
    x = torch.from_numpy(synth.make_image(203, 317, 9, 0.2, rectangles=8)[1]).cuda()
    ref = V.filter(x, win, filter, 0.25, precision="fp64")
    for s in range(len(V.tile_shapes())):
        V.set_tuned_shape(win, filter, "exact", s)
        o, i = V.filter(x, win, filter, 0.25, precision="fp32")
        assert torch.equal(o, ref[0]) and torch.equal(i, ref[1])
    last = len(V.tile_shapes()) - 1
    shape, ms = V.autotune(x, win, filter, 0.25, reps=3)
    assert 0 <= shape < len(V.tile_shapes()) and ms > 0
    assert V.tuned_shape(win, filter, p=0.25) == shape
    # the DDF 5x5 at p = 1/4 (score slots) has its own entry: the other
    # exponents keep the shape set before
    assert V.tuned_shape(win, filter) == (last if (win, filter) == (5, "ddf") else shape)
    V.set_tuned_shape(win, filter, "exact", 0)


def test_plan_rejects_bad_descriptors(V):
    x = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(V.VdfError):
        V.Plan([dict(img=x, win=4)])
    with pytest.raises(V.VdfError):
        V.Plan([dict(img=x, win=3)], dist="minimax", q=5)
    with pytest.raises(V.VdfError):
        V.Plan([dict(img=x, win=3, filter="ddf", p=2.0)])


@pytest.mark.parametrize("persistent", [False, True])
def test_full_size_batch_workload(V, persistent):
    """The benchmark's batch (256 images, sides log-uniform in [64, 2048],
    150.8 Mpix, mixed 3x3/5x5 BVDF/DDF, tuned shapes) in the launch
    configuration the bench times (graph replay): every image equals the
    single-image FP32 path, and the oracle on 400 sampled pixels."""
    import oracle
    import bench
    oracle.build()
    imgs = bench.batch_images(256, 4242)
    rng = np.random.default_rng(7)
    cfgs = [(int(rng.choice([3, 5])), str(rng.choice(["bvdf", "ddf"]))) for _ in imgs]
    probe = torch.from_numpy(bench.frames(1)[0]).cuda()
    for win in (3, 5):
        for f in ("bvdf", "ddf"):
            V.autotune(probe, win, f, 0.25, reps=2)
    items = [dict(img=torch.from_numpy(x).cuda(), win=w, filter=f, p=0.25) for x, (w, f) in zip(imgs, cfgs)]
    plan = V.Plan(items, persistent=persistent)
    plan.graph_launch()
    plan.graph_launch()
    torch.cuda.synchronize()
    rechecked, overflow = plan.stats()
    assert overflow == 0 and rechecked > 0
    check_against_single(V, plan, "fp32")
    srng = np.random.default_rng(8)
    for k in srng.choice(len(imgs), 40, replace=False):
        it, img = plan.items[k], imgs[k]
        M, N = img.shape[:2]
        pix = srng.integers(0, M * N, 10)
        ref = oracle.filter_u8(img, it["win"], it["filter"], 0.25, "exact", 4, pixels=pix)
        assert np.array_equal(it["index"].cpu().numpy().reshape(-1)[pix], ref["idx"])
        assert np.array_equal(it["out"].cpu().numpy().reshape(-1, 3)[pix], ref["out"])
