"""vdf_filter_host_frames: a sequence of host frames, copies overlapped with
filtering through three device slots, must give every frame exactly what
vdf_filter gives it (and the oracle, on small frames)."""
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


def host_frames(M, N, count, seed):
    from paper_1009_0958_gb300 import synth
    return [torch.from_numpy(synth.make_image(M, N, seed + k, 0.15, rectangles=4)[1]).pin_memory()
            for k in range(count)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("win,filter,p", [(5, "ddf", 0.25), (3, "bvdf", 0.5), (5, "ddf", 0.3)])
def test_frames_equal_single_calls(V, precision, win, filter, p):
    frames = host_frames(97, 131, 5, 10)
    outs, idxs = V.filter_host_frames(frames, win, filter, p, precision=precision)
    for f, o, i in zip(frames, outs, idxs):
        ro, ri = V.filter(f.cuda(), win, filter, p, precision=precision)
        assert torch.equal(o, ro.cpu()) and torch.equal(i, ri.cpu())


def test_frames_match_oracle(V):
    import oracle
    oracle.build()
    frames = host_frames(40, 57, 3, 30)
    outs, idxs = V.filter_host_frames(frames, 5, "ddf", 0.25)
    for f, o, i in zip(frames, outs, idxs):
        ref = oracle.filter_u8(f.numpy(), 5, "ddf", 0.25, "exact")
        assert np.array_equal(o.numpy(), ref["out"]) and np.array_equal(i.numpy(), ref["idx"])


def test_frames_full_hd_and_reuse(V):
    """Three 1080p frames, one single frame, then the first frames again with
    the same buffer (slots reused across calls); some index maps omitted."""
    frames = host_frames(1080, 1920, 3, 50)
    buf = torch.empty(V.host_frames_buffer_bytes(1080, 1920) + 256, dtype=torch.uint8, device="cuda")
    outs, idxs = V.filter_host_frames(frames, dev_buffer=buf)
    refs = [V.filter(f.cuda(), 5, "ddf", 0.25) for f in frames]
    for o, i, (ro, ri) in zip(outs, idxs, refs):
        assert torch.equal(o, ro.cpu()) and torch.equal(i, ri.cpu())
    one, _ = V.filter_host_frames(frames[2:], dev_buffer=buf)
    assert torch.equal(one[0], refs[2][0].cpu())
    again, ix = V.filter_host_frames(frames[:2], dev_buffer=buf, indices=[None, torch.zeros((1080, 1920),
                                                                                           dtype=torch.int8)])
    assert torch.equal(again[0], refs[0][0].cpu()) and torch.equal(again[1], refs[1][0].cpu())
    assert torch.equal(ix[1], refs[1][1].cpu())


def test_frames_reject_bad_arguments(V):
    frames = host_frames(16, 16, 2, 1)
    with pytest.raises(V.VdfError):
        V.filter_host_frames(frames, 4)              # window size
    with pytest.raises(V.VdfError):
        V.filter_host_frames([frames[0], torch.zeros((16, 17, 3), dtype=torch.uint8)])
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(V.VdfError):
        V.filter_host_frames(frames, dev_buffer=small)
