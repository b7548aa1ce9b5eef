"""The FP32 pair terms that the certified path sums (vdf_debug_fp32_terms),
against exact values, within the error bounds its scores are built on
(u = 2^-24): |x - y| on every attainable input, the Eq. (2) angle on random
and structured pairs (float64 reference from exact integers), and the
Method 1 (Table 1) and Method 2 (Eq. (7)) terms against the oracle's
binary128 values."""
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


def gpu_terms(V, pairs, dist="exact", q=4):
    t = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    ang, l2 = V.debug_fp32_terms(t, dist, q)
    return ang.cpu().numpy().astype(np.float64), l2.cpu().numpy().astype(np.float64)


def structured_pairs():
    """Collinear, nearly collinear, orthogonal, zero and extreme vectors."""
    P = [
        (1, 2, 3, 2, 4, 6), (255, 255, 255, 1, 1, 1), (255, 255, 255, 255, 255, 254), (255, 255, 254, 254, 255, 255),
        (255, 0, 0, 0, 255, 0), (0, 0, 255, 255, 255, 0), (0, 0, 0, 10, 20, 30), (0, 0, 0, 0, 0, 0),
        (255, 255, 255, 255, 255, 255), (1, 0, 0, 255, 1, 0), (200, 100, 50, 201, 100, 50), (3, 5, 7, 6, 10, 14),
        (128, 128, 128, 127, 128, 129), (1, 1, 0, 0, 1, 1), (255, 254, 253, 253, 254, 255), (7, 0, 0, 0, 0, 9),
    ]
    rng = np.random.default_rng(11)
    # small perturbations of collinear pairs: the smallest angles
    base = rng.integers(1, 86, (400, 3))
    k = rng.integers(1, 4, (400, 1))
    y = np.clip(base * k + rng.integers(-1, 2, (400, 3)), 0, 255)
    P += [tuple(a) + tuple(b) for a, b in zip(base, y)]
    return np.array(P, dtype=np.int64)


def test_l2_every_attainable_square(V):
    """|x - y| for every value of |x - y|^2 that uint8 RGB pairs can produce
    (sums of three squares of 0..255), through pairs (a, b, c), (0, 0, 0)."""
    sq = np.arange(256, dtype=np.int64) ** 2
    e = (sq[:, None, None] + sq[None, :, None] + sq[None, None, :]).ravel()
    vals, first = np.unique(e, return_index=True)
    a, b, c = np.unravel_index(first, (256, 256, 256))
    pairs = np.stack([a, b, c, 0 * a, 0 * a, 0 * a], axis=1)
    _, l2 = gpu_terms(V, pairs)
    exact = np.sqrt(vals.astype(np.float64))
    assert l2[0] == 0.0 and vals[0] == 0
    rel = np.abs(l2[1:] - exact[1:]) / exact[1:]
    assert rel.max() <= 2 * U          # observed 1.7u; the FP32 bounds use 5u
    assert len(vals) > 100000


def test_l2_random_pairs_match_exact(V):
    rng = np.random.default_rng(2)
    pairs = rng.integers(0, 256, (100000, 6))
    _, l2 = gpu_terms(V, pairs)
    e = ((pairs[:, :3] - pairs[:, 3:]) ** 2).sum(1).astype(np.float64)
    exact = np.sqrt(e)
    nz = e > 0
    assert np.all(l2[~nz] == 0.0)
    assert (np.abs(l2[nz] - exact[nz]) / exact[nz]).max() <= 5 * U


def exact_angle(pairs):
    x, y = pairs[:, :3].astype(np.int64), pairs[:, 3:].astype(np.int64)
    d = (x * y).sum(1)
    c2 = (x * x).sum(1) * (y * y).sum(1) - d * d          # exact in int64
    th = np.arctan2(np.sqrt(c2.astype(np.float64)), d.astype(np.float64))
    zero = ((x * x).sum(1) == 0) | ((y * y).sum(1) == 0)
    th[zero] = np.pi / 2                                 # cosine of a zero vector taken as 0
    return th


def test_angle_relative_bound(V):
    rng = np.random.default_rng(3)
    pairs = np.concatenate([structured_pairs(), rng.integers(0, 256, (200000, 6))])
    ang, _ = gpu_terms(V, pairs, "exact")
    ref = exact_angle(pairs)
    assert np.all(ang[ref == 0.0] == 0.0)                # collinear: exactly 0
    nz = ref > 0
    rel = np.abs(ang[nz] - ref[nz]) / ref[nz]
    assert rel.max() <= 26 * U, rel.max() / U            # kAngleU


@pytest.mark.parametrize("q", [2, 3, 4])
def test_minimax_absolute_bound(V, q):
    import oracle
    oracle.build()
    rng = np.random.default_rng(40 + q)
    pairs = np.concatenate([structured_pairs()[:200], rng.integers(0, 256, (1500, 6))])
    ang, _ = gpu_terms(V, pairs, "minimax", q)
    ref = np.array([oracle.term(p[:3], p[3:], "angle", "minimax", q)[1] for p in pairs])
    assert np.abs(ang - ref).max() <= 24 * U


def test_chromaticity_relative_bound(V):
    import oracle
    oracle.build()
    rng = np.random.default_rng(5)
    pairs = np.concatenate([structured_pairs()[:200], rng.integers(0, 256, (1500, 6))])
    ang, _ = gpu_terms(V, pairs, "rgb")
    ref = np.array([oracle.term(p[:3], p[3:], "angle", "rgb")[1] for p in pairs])
    nz = ref > 0
    assert np.all(ang[~nz] == 0.0)
    assert (np.abs(ang[nz] - ref[nz]) / ref[nz]).max() <= 11 * U
