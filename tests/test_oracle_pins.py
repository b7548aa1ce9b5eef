"""Pins for the CPU oracle: what the paper and the mathematics fix.

None of these re-type the oracle's formulas.  They check it against printed
values (Table 1, Eq. (10)), closed forms, library routines (scipy distances,
numpy windowing, mpmath at high precision), invariants of the definitions
(Eqs. (1)-(3)) and brute force on small inputs.
"""
import math

import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view
from scipy.spatial.distance import cdist

from tests.conftest import read_table1

RNG = np.random.default_rng(12345)


# ----------------------------------------------------------- Table 1 / Method 1

@pytest.mark.parametrize("branch", ["ASIN", "ACOS"])
@pytest.mark.parametrize("q", [2, 3, 4])
def test_table1_oracle_coefficients_match_fixture(orc, table1, branch, q):
    """The oracle's polynomial equals the printed coefficients (numpy polyval)."""
    _, coef, _ = table1[(branch, q)]
    for t in np.linspace(0.0, 1.0, 17):
        hi, lo = orc.poly(branch.lower(), q, t)
        assert abs((hi + lo) - np.polynomial.polynomial.polyval(t, coef)) < 1e-14


@pytest.mark.parametrize("branch", ["ASIN", "ACOS"])
@pytest.mark.parametrize("q", [2, 3, 4])
def test_table1_max_error_reproduces_epsilon(orc, table1, branch, q):
    """Section 2.1: the max |error| of each printed polynomial over its range
    is the epsilon column (within 2%: the coefficients are printed to ~7
    digits).  Pins the coefficients, the branch ranges and Eq. (6)."""
    eps, coef, _ = table1[(branch, q)]
    if branch == "ASIN":
        t = np.linspace(0.0, 1.0 / math.sqrt(2.0), 200001)
        true = 2.0 * np.arcsin(t / math.sqrt(2.0))   # Eq. (6)
    else:
        t = np.linspace(0.0, 0.5, 200001)
        true = np.arccos(t)
    err = np.abs(np.polynomial.polynomial.polyval(t, coef) - true).max()
    assert abs(err - eps) <= 0.02 * eps, (err, eps)
    # the oracle evaluates the same polynomial
    for tt in t[::20000]:
        hi, lo = orc.poly(branch.lower(), q, tt)
        assert abs(hi - np.polynomial.polynomial.polyval(tt, coef)) < 1e-13


def test_eq5_eq6_identity_branch_value(orc):
    """Eqs. (5)-(6): for z >= 1/2 the ASIN polynomial in tau = sqrt(1 - z)
    approximates acos(z); for z < 1/2 the ACOS polynomial in z does.  So the
    minimax term must be within Table 1's epsilon of acos(z) on both sides."""
    tab = read_table1()
    for _ in range(400):
        x = RNG.integers(0, 256, 3).astype(float)
        y = RNG.integers(0, 256, 3).astype(float)
        if x.sum() == 0 or y.sum() == 0:
            continue
        z = x @ y / math.sqrt((x @ x) * (y @ y))
        for q in (2, 3, 4):
            d, hi, lo = orc.term(x, y, "angle", "minimax", q)
            eps = tab[("ASIN" if z >= 0.5 else "ACOS", q)][0]
            assert abs(hi - math.acos(min(z, 1.0))) <= eps * 1.03
            assert abs(d - hi) < 1e-9


# ------------------------------------------------------------- Eq. (2) angle

@pytest.mark.parametrize("x,y,expect", [
    ((255, 0, 0), (0, 255, 0), math.pi / 2),
    ((1, 1, 0), (1, 0, 0), math.pi / 4),
    ((1, 1, 0), (1, 0, 1), math.pi / 3),
    ((3, 4, 0), (3, 4, 0), 0.0),
    ((10, 20, 30), (20, 40, 60), 0.0),       # collinear
    ((0, 0, 0), (10, 20, 30), math.pi / 2),  # zero vector: cos := 0
    ((0, 0, 0), (0, 0, 0), math.pi / 2),
    ((1, 1, 1), (1, 0, 0), math.acos(1 / math.sqrt(3))),
])
def test_angle_closed_forms(orc, x, y, expect):
    d, hi, lo = orc.term(np.array(x, float), np.array(y, float), "angle", "exact")
    assert abs(d - expect) <= 4e-16 * max(1, expect)
    assert abs((hi + lo) - expect) <= 3.5e-16 * max(1, expect)   # expect is itself rounded


def test_angle_matches_scipy_cosine_distance(orc):
    """Eq. (2) against scipy's cosine distance (library routine)."""
    x = RNG.uniform(0.05, 1.0, (300, 3))
    y = RNG.uniform(0.05, 1.0, (300, 3))
    ref = np.arccos(np.clip(1.0 - np.array([cdist(x[i:i + 1], y[i:i + 1], "cosine")[0, 0] for i in range(300)]), -1, 1))
    for i in range(300):
        d, hi, lo = orc.term(x[i], y[i], "angle", "exact")
        if ref[i] > 1e-3:                 # arccos(1 - c) is ill-conditioned near 0
            assert abs(d - ref[i]) <= 1e-9 * ref[i]
        assert abs(d - hi) <= 4e-15 * hi + 1e-300


def test_terms_against_mpmath(orc, table1):
    """Binary128 terms agree with 50-digit mpmath evaluations of the paper's
    formulas (Eq. (2), Eq. (6)/Table 1, Eq. (7), Eq. (1))."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for _ in range(150):
        x = RNG.integers(0, 256, 3).astype(float)
        y = RNG.integers(0, 256, 3).astype(float)
        X = [mp.mpf(int(v)) for v in x]
        Y = [mp.mpf(int(v)) for v in y]
        dot = sum(a * b for a, b in zip(X, Y))
        P = sum(a * a for a in X) * sum(b * b for b in Y)
        # Eq. (2)
        want = mp.pi / 2 if P == 0 else mp.acos(dot / mp.sqrt(P))
        _, hi, lo = orc.term(x, y, "angle", "exact")
        assert abs(mp.mpf(hi) + mp.mpf(lo) - want) < mp.mpf("1e-26")
        # Method 1
        z = mp.mpf(0) if P == 0 else dot / mp.sqrt(P)
        for q in (2, 3, 4):
            branch = "ASIN" if (P != 0 and 4 * dot * dot >= P) else "ACOS"
            coef = [mp.mpf(s) for s in table1[(branch, q)][2]]
            t = mp.sqrt(1 - z) if branch == "ASIN" else z
            want = sum(c * t ** k for k, c in enumerate(coef))
            _, hi, lo = orc.term(x, y, "angle", "minimax", q)
            assert abs(mp.mpf(hi) + mp.mpf(lo) - want) < mp.mpf("1e-26")
        # Method 2, Eq. (7)
        sx, sy = sum(X), sum(Y)
        cx = [a / sx if sx else mp.mpf(0) for a in X]
        cy = [b / sy if sy else mp.mpf(0) for b in Y]
        want = mp.sqrt(sum((a - b) ** 2 for a, b in zip(cx, cy)))
        d, hi, lo = orc.term(x, y, "angle", "rgb")
        assert abs(mp.mpf(hi) + mp.mpf(lo) - want) < mp.mpf("1e-30")
        assert abs(d - float(want)) <= 1e-15 * float(want) + 1e-300
        # Eq. (1), p = 2
        want = mp.sqrt(sum((a - b) ** 2 for a, b in zip(X, Y)))
        d, hi, lo = orc.term(x, y, "l2")
        assert abs(mp.mpf(hi) + mp.mpf(lo) - want) < mp.mpf("1e-29") * max(1, want)


def test_chromaticity_distance_matches_scipy(orc):
    x = RNG.integers(1, 256, (200, 3)).astype(float)
    y = RNG.integers(1, 256, (200, 3)).astype(float)
    cx = x / x.sum(1, keepdims=True)
    cy = y / y.sum(1, keepdims=True)
    for i in range(200):
        ref = cdist(cx[i:i + 1], cy[i:i + 1])[0, 0]
        d, hi, lo = orc.term(x[i], y[i], "angle", "rgb")
        assert abs(d - ref) <= 1e-14 * max(ref, 1e-3)
    # identical chromaticity -> 0; one zero vector -> |x'| of the other
    assert orc.term([10, 20, 30], [20, 40, 60], "angle", "rgb")[0] == 0.0
    assert abs(orc.term([0, 0, 0], [0, 0, 7], "angle", "rgb")[0] - 1.0) < 1e-15


def test_eq10_refit_total_least_squares(orc):
    """Section 3.2: a line fitted between A and B over random RGB pairs gives
    Eq. (10).  Orthogonal (total) least squares on uniform RGB pairs lands
    within sampling noise of the printed slope and offset.  (The fit-error
    figure 0.005715 is not reproduced: its definition is not given.)"""
    with open("tests/golden/eq10_linear_map.txt") as fh:
        slope, offset, _ = [float(v) for v in [l for l in fh if not l.startswith("#")][0].split()]
    rng = np.random.default_rng(7)
    A, B = [], []
    for _ in range(40000):
        x = rng.integers(0, 256, 3).astype(float)
        y = rng.integers(0, 256, 3).astype(float)
        if x.sum() == 0 or y.sum() == 0:
            continue
        A.append(orc.term(x, y, "angle", "exact")[0])
        B.append(orc.term(x, y, "angle", "rgb")[0])
    A, B = np.array(A), np.array(B)
    Mx = np.c_[B - B.mean(), A - A.mean()]
    v = np.linalg.svd(Mx, full_matrices=False)[2][-1]
    s = -v[0] / v[1]
    o = A.mean() - s * B.mean()
    assert abs(s - slope) < 0.02 and abs(o - offset) < 0.006, (s, o)


# --------------------------------------------------------- window selection

def lib_scores(v, filter, p, dist, q=4, table=None):
    """Scores from library routines: scipy cosine/euclidean distances.  A
    vector's cosine distance to itself is exactly 0 (scipy returns ~1e-16,
    which arccos would amplify to ~1e-8)."""
    cos_d = cdist(v, v, "cosine")
    np.fill_diagonal(cos_d, 0.0)
    if dist == "exact":
        A = np.arccos(np.clip(1.0 - cos_d, -1.0, 1.0))
    elif dist == "rgb":
        c = v / v.sum(1, keepdims=True)
        A = cdist(c, c)
        if filter == "ddf":
            A = 1.436437 * A + 0.027664
    else:
        z = np.clip(1.0 - cos_d, -1.0, 1.0)
        ea, ca, _ = table[("ASIN", q)]
        ec, cc, _ = table[("ACOS", q)]
        A = np.where(z >= 0.5, np.polynomial.polynomial.polyval(np.sqrt(np.maximum(1 - z, 0)), ca),
                     np.polynomial.polynomial.polyval(z, cc))
    SA = A.sum(1)
    SL = cdist(v, v).sum(1)
    if filter == "bvdf":
        return SA, SA, SL
    return np.maximum(SA, 0) ** p * SL ** (1 - p), SA, SL


def tie_rule(scores, n, rel=1e-12):
    """Minimisers (equal up to library rounding); centre first, else lowest."""
    m = scores.min()
    mins = np.flatnonzero(scores <= m + rel * max(abs(m), 1e-3))
    c = (n - 1) // 2
    return c if c in mins else int(mins[0])


@pytest.mark.parametrize("n", [9, 25])
@pytest.mark.parametrize("filter,p", [("bvdf", 0.5), ("ddf", 0.25), ("ddf", 0.5), ("ddf", 0.0), ("ddf", 1.0)])
@pytest.mark.parametrize("dist", ["exact", "minimax", "rgb"])
def test_window_against_library(orc, table1, n, filter, p, dist):
    """Random windows without ties: the oracle's selection and aggregates
    equal those built from scipy distances (Eqs. (1)-(3), (7), Table 1)."""
    rng = np.random.default_rng(hash((n, filter, p, dist)) % 2**32)
    for _ in range(40):
        v = rng.uniform(1.0, 255.0, (n, 3))
        sel, sc, agg, fl = orc.window(v, filter, p, dist, 4)
        ref, SA, SL = lib_scores(v, filter, p, dist, 4, table1)
        assert sel == int(np.argmin(ref))
        assert np.allclose(agg[:, 0], SA, rtol=1e-10, atol=1e-12)
        if filter == "ddf":
            assert np.allclose(agg[:, 1], SL, rtol=1e-12)
        assert np.allclose(sc, ref, rtol=1e-9, atol=1e-12)


def test_ddf_p0_is_vmf_p1_is_bvdf(orc):
    """Eq. (3) limits: p = 0 gives the VMF of Eq. (1) (L2), p = 1 gives BVDF."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        v = rng.integers(0, 256, (25, 3)).astype(float)
        vmf = int(np.argmin(cdist(v, v).sum(1)))
        assert orc.window(v, "ddf", 0.0, "exact")[0] == vmf
        for dist in ("exact", "minimax", "rgb"):
            assert orc.window(v, "ddf", 1.0, dist)[0] == orc.window(v, "bvdf", 0.5, dist)[0]


def test_bvdf_scale_invariance(orc):
    """BVDF depends on directions only: positive per-vector scaling keeps the
    selected member (all three distance modes)."""
    rng = np.random.default_rng(4)
    for _ in range(60):
        v = rng.integers(1, 60, (9, 3)).astype(float)
        k = rng.integers(1, 5, (9, 1)).astype(float)
        for dist in ("exact", "minimax", "rgb"):
            a = orc.window(v, "bvdf", 0.5, dist)
            b = orc.window(v * k, "bvdf", 0.5, dist)
            if a[3] == 0 and b[3] == 0:
                assert a[0] == b[0]


def test_permutation_equivariance(orc):
    """The selected vector does not depend on member order (no ties)."""
    rng = np.random.default_rng(5)
    for _ in range(60):
        v = rng.uniform(0, 255, (25, 3))
        perm = rng.permutation(25)
        for filter in ("bvdf", "ddf"):
            a = orc.window(v, filter, 0.25, "exact")[0]
            b = orc.window(v[perm], filter, 0.25, "exact")[0]
            assert np.array_equal(v[a], v[perm][b])


@pytest.mark.parametrize("filter", ["bvdf", "ddf"])
@pytest.mark.parametrize("dist", ["exact", "minimax", "rgb"])
@pytest.mark.parametrize("q", [2, 3, 4])
def test_constant_window_returns_centre(orc, filter, dist, q):
    for n in (9, 25, 49):
        v = np.tile([[37.0, 99.0, 180.0]], (n, 1))
        sel, _, _, fl = orc.window(v, filter, 0.25, dist, q)
        assert sel == (n - 1) // 2 and fl & orc.FLAG_TIE


def test_tie_rule_lowest_index_without_centre(orc):
    """Eight identical neighbours around an outlier centre tie; the lowest
    raster index wins.  With the centre equal to them, the centre wins."""
    a = [100.0, 50.0, 20.0]
    v = np.tile([a], (9, 1))
    v[4] = [3.0, 200.0, 90.0]
    for filter in ("bvdf", "ddf"):
        for dist in ("exact", "minimax", "rgb"):
            assert orc.window(v, filter, 0.25, dist)[0] == 0
    # equal-multiset (non-collinear) tie: x=(1,0,0), y=(0,1,0) four times each,
    # centre (1,1,0) once; A sums of x and y are equal exactly.
    v = np.array([[1, 0, 0]] * 4 + [[1, 1, 0]] + [[0, 1, 0]] * 4, float)
    v = v[[0, 5, 1, 6, 4, 2, 7, 3, 8]]
    sel, sc, agg, fl = orc.window(v, "bvdf", 0.5, "exact")
    assert fl & orc.FLAG_TIE or sel == 4
    x_sum = 4 * math.pi / 2 + math.pi / 4
    assert abs(agg[0, 0] - x_sum) < 1e-15 and abs(agg[1, 0] - x_sum) < 1e-15


def test_zero_vector_conventions(orc):
    """A zero vector is at pi/2 from everything (cosine := 0)."""
    v = np.array([[0, 0, 0]] + [[10 * (i + 1), 5, 3] for i in range(8)], float)
    sel, sc, agg, fl = orc.window(v, "bvdf", 0.5, "exact")
    assert abs(agg[0, 0] - 9 * math.pi / 2) < 1e-14
    # minimax: a zero-vector pair uses P_ACOS(0) = a0 of the ACOS row
    tab = read_table1()
    sel, sc, agg, fl = orc.window(v, "bvdf", 0.5, "minimax", 4)
    assert abs(agg[0, 0] - 9 * tab[("ACOS", 4)][1][0]) < 1e-13


def test_minimax_q3_negative_sum_is_clamped(orc):
    """q = 3's a0 < 0: a collinear window has a negative angular sum; DDF uses
    max(sum, 0), so every member scores 0 and the centre wins."""
    v = np.array([[10 * (i + 1), 20 * (i + 1), 5 * (i + 1)] for i in range(9)], float)
    sel, sc, agg, fl = orc.window(v, "ddf", 0.25, "minimax", 3)
    assert (agg[:, 0] < 0).all() and np.all(sc == 0) and sel == 4


# ------------------------------------------------------------- whole images

@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("filter,p", [("bvdf", 0.5), ("ddf", 0.25)])
@pytest.mark.parametrize("dist", ["exact", "rgb", "minimax"])
def test_image_against_numpy_windowing(orc, table1, win, filter, p, dist):
    """Section II windowing: edge-replicated borders (np.pad 'edge'), raster
    member order (sliding_window_view), per-window argmin from scipy
    distances.  Random colours make ties improbable; the test skips none."""
    rng = np.random.default_rng(win * 100 + len(dist))
    M, N = 13, 17
    img = rng.integers(1, 256, (M, N, 3)).astype(np.uint8)
    r = orc.filter_u8(img, win, filter, p, dist, 4)
    R = win // 2
    pad = np.pad(img.astype(float), ((R, R), (R, R), (0, 0)), mode="edge")
    wins = sliding_window_view(pad, (win, win, 3))[:, :, 0]     # M x N x w x w x 3
    for i in range(M):
        for j in range(N):
            v = wins[i, j].reshape(-1, 3)
            sc = lib_scores(v, filter, p, dist, 4, table1)[0]
            ref = tie_rule(sc, len(v))
            assert r["idx"][i, j] == ref, (i, j)
            assert np.array_equal(r["out"][i, j], img[min(max(i + ref // win - R, 0), M - 1),
                                                      min(max(j + ref % win - R, 0), N - 1)])


def test_pixel_subset_equals_full_image(orc):
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(40, 33, 9, 0.2, rectangles=4)
    full = orc.filter_u8(img, 5, "ddf", 0.25, "exact")
    pix = np.array([0, 5, 100, 40 * 33 - 1, 17 * 33 + 3])
    sub = orc.filter_u8(img, 5, "ddf", 0.25, "exact", pixels=pix)
    assert np.array_equal(sub["idx"], full["idx"].ravel()[pix])
    assert np.array_equal(sub["out"], full["out"].reshape(-1, 3)[pix])


def test_float_path_matches_uint8_for_bvdf(orc):
    """Float inputs k/255 have the directions of the uint8 inputs up to
    float32 rounding; on a tie-free random image BVDF selects the same."""
    rng = np.random.default_rng(11)
    img = rng.integers(1, 256, (12, 14, 3)).astype(np.uint8)
    a = orc.filter_u8(img, 3, "bvdf", 0.5, "exact")
    f = (img.astype(np.float32) / np.float32(255)).transpose(2, 0, 1)[None]
    b = orc.filter_f32(f, 3, "bvdf", 0.5, "exact")
    assert np.array_equal(a["idx"], b["idx"][0])


def test_no_gray_pixels_on_standard_images(orc):
    """On the synthetic workloads no pixel falls where double precision
    cannot separate a tie from a non-tie."""
    from paper_1009_0958_gb300 import synth
    for seed, rect in ((0, 0), (1, 12)):
        _, img = synth.make_image(48, 64, seed, 0.1, rectangles=rect)
        for win in (3, 5):
            for filter in ("bvdf", "ddf"):
                for dist in ("exact", "minimax", "rgb"):
                    r = orc.filter_u8(img, win, filter, 0.25, dist, 4)
                    assert not (r["flags"] & orc.FLAG_GRAY).any()


def test_filter_removes_impulses():
    """Sanity of the whole procedure (Tables 2-3 show PSNR rising from ~18 dB
    to ~31 dB at 10% noise): the filtered image is much closer to the clean
    one than the noisy input is."""
    import oracle
    from paper_1009_0958_gb300 import synth
    clean, noisy = synth.make_image(64, 64, 21, 0.10)

    def psnr(a, b):
        mse = np.mean((a.astype(float) - b.astype(float)) ** 2)
        return 10 * np.log10(255.0 ** 2 / mse)
    for filter in ("bvdf", "ddf"):
        for dist in ("exact", "minimax", "rgb"):
            y = oracle.filter_u8(noisy, 3, filter, 0.25, dist, 4)["out"]
            assert psnr(y, clean) > psnr(noisy, clean) + 8.0


# ------------------------------------------ VMF and Minkowski orders (Eq. (1))

ORDER_METRIC = {1: "cityblock", 2: "euclidean", "inf": "chebyshev"}


@pytest.mark.parametrize("order", [1, 2, "inf"])
def test_minkowski_terms_match_scipy(orc, order):
    """Eq. (1) at orders 1, 2 and infinity against scipy's distances."""
    rng = np.random.default_rng(21)
    which = {1: "l1", 2: "l2", "inf": "linf"}[order]
    for _ in range(300):
        x, y = rng.integers(0, 256, 3).astype(float), rng.integers(0, 256, 3).astype(float)
        ref = cdist(x[None], y[None], ORDER_METRIC[order])[0, 0]
        d, hi, lo = orc.term(x, y, which)
        assert abs(d - ref) <= 1e-15 * ref and abs((hi + lo) - ref) <= 1e-15 * ref


def tie_rule_pick(minimisers, n):
    """Centre if it is a minimiser, else the lowest index."""
    centre = (n - 1) // 2
    return centre if centre in minimisers else min(minimisers)


@pytest.mark.parametrize("order", [1, 2, "inf"])
@pytest.mark.parametrize("n", [9, 25])
def test_vmf_window_brute_force(orc, order, n):
    """Eq. (1) VMF: argmin of the summed scipy distances, ties by the tie rule
    (integer vectors: the order-1 and infinity sums are exact integers)."""
    rng = np.random.default_rng(22 + n)
    for trial in range(150):
        hi = 256 if trial % 3 else 4   # small ranges make exact ties common
        v = rng.integers(0, hi, (n, 3)).astype(float)
        s = cdist(v, v, ORDER_METRIC[order]).sum(1)
        if order == 2:
            mins = np.flatnonzero(s <= s.min() * (1 + 1e-12))
            if len(mins) > 1 and not all(np.array_equal(np.sort(cdist(v[[i]], v)[0]), np.sort(cdist(v[[mins[0]]], v)[0]))
                                         for i in mins):
                continue   # near-equal L2 sums that are not equal multisets: left to the binary128 stage
        else:
            mins = np.flatnonzero(s == s.min())
        sel = orc.window(v, "vmf", order=order)[0]
        assert sel == tie_rule_pick(list(mins), n)


def gray_median_reference(img1, win):
    """Textbook median filter of a single-channel image (edge replication),
    returning, per pixel, the index the tie rule picks among the window
    members equal to the median."""
    R = win // 2
    pad = np.pad(img1, R, mode="edge")
    wins = sliding_window_view(pad, (win, win)).reshape(img1.shape + (win * win,))
    med = np.median(wins, axis=-1)
    eq = wins == med[..., None]
    centre = (win * win - 1) // 2
    first = np.argmax(eq, axis=-1)
    return np.where(eq[..., centre], centre, first)


@pytest.mark.parametrize("order", [1, 2, "inf"])
@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("channel", [None, 0, 1, 2])
def test_vmf_reduces_to_the_median_filter(orc, order, win, channel):
    """When the vectors differ along one direction only (gray pixels r = g = b,
    or a single varying channel), every Minkowski distance is a fixed multiple
    of the scalar difference, and the VMF of Eq. (1) is the scalar median
    filter (numpy's median of each window, odd n)."""
    rng = np.random.default_rng(23 + win)
    M, N = 23, 31
    s = rng.integers(0, 256, (M, N))
    s[rng.random((M, N)) < 0.3] = 77   # repeated values: ties on the median
    if channel is None:
        img = np.repeat(s[..., None], 3, axis=2).astype(np.uint8)
    else:
        img = np.tile(rng.integers(0, 256, 3), (M, N, 1)).astype(np.uint8)
        img[..., channel] = s
    res = orc.filter_u8(img, win, "vmf", order=order)
    assert np.array_equal(res["idx"], gray_median_reference(s, win))
    assert np.array_equal(res["out"][..., 0 if channel is None else channel],
                          np.median(sliding_window_view(np.pad(s, win // 2, mode="edge"), (win, win)),
                                    axis=(-2, -1)).astype(np.uint8))


@pytest.mark.parametrize("order", [1, "inf"])
def test_ddf_order_limits(orc, order):
    """Eq. (3) with the order-o distance: p = 0 gives the order-o VMF, p = 1
    gives BVDF (the distance drops out)."""
    rng = np.random.default_rng(24)
    for _ in range(80):
        v = rng.integers(0, 256, (25, 3)).astype(float)
        assert orc.window(v, "ddf", 0.0, order=order)[0] == orc.window(v, "vmf", order=order)[0]
        assert orc.window(v, "ddf", 1.0, order=order)[0] == orc.window(v, "bvdf", 0.5)[0]


@pytest.mark.parametrize("order", [1, 2, "inf"])
def test_vmf_constant_window_and_aggregates(orc, order):
    """A constant window returns its centre; the aggregates of a window are
    the scipy distance sums (first column 0 for VMF)."""
    for n in (9, 25):
        v = np.tile([[37.0, 99.0, 180.0]], (n, 1))
        sel, _, _, fl = orc.window(v, "vmf", order=order)
        assert sel == (n - 1) // 2 and fl & orc.FLAG_TIE
    rng = np.random.default_rng(25)
    v = rng.integers(0, 256, (25, 3)).astype(float)
    _, sc, agg, _ = orc.window(v, "vmf", order=order)
    ref = cdist(v, v, ORDER_METRIC[order]).sum(1)
    assert np.allclose(agg[:, 1], ref, rtol=1e-15) and np.all(agg[:, 0] == 0) and np.allclose(sc, ref, rtol=1e-15)


# ------------------------------------------------------------ ACWDDF (Eq. (9))

def test_acwddf_closed_forms(orc):
    """Eight equal neighbours a around a centre b, 3x3, lambda = 2 (centre
    weights 7, 5, 3): each CWVMF level picks a (weighted sum 7 L(a,b) for a
    against 8 L(a,b) for b), so the switching sum is 3 A(a,b) L2(a,b).
    Orthogonal a, b: 3 (pi/2) 10 sqrt(2) = 66.6 > 10.8, the DDF output (a,
    lowest index 0).  Nearly parallel: 3 atan(1/10) = 0.30 < 10.8, the
    centre."""
    v = np.tile([[10.0, 0.0, 0.0]], (9, 1))
    v[4] = [0.0, 10.0, 0.0]
    sel, cw, s, _ = orc.window_acwddf(v)
    assert cw == [0, 0, 0] and sel == 0
    assert abs(s - 3 * (math.pi / 2) * math.hypot(10, 10)) < 1e-12
    v[4] = [10.0, 1.0, 0.0]
    sel, cw, s, _ = orc.window_acwddf(v)
    assert cw == [0, 0, 0] and sel == 4
    assert abs(s - 3 * math.atan2(1, 10) * 1.0) < 1e-14


@pytest.mark.parametrize("n", [9, 25])
def test_cwvmf_is_the_centre_weighted_median_on_gray_windows(orc, n):
    """Gray vectors: the CWVMF of Eq. (9) is the centre-weighted median (the
    median of the values with the centre repeated w_d = n - 2k + 2 times;
    numpy), the tie rule choosing among the members with that value."""
    rng = np.random.default_rng(31 + n)
    d = (n - 1) // 2
    for _ in range(60):
        g = rng.integers(0, 40, n).astype(float)
        v = np.repeat(g[:, None], 3, axis=1)
        for k in range(1, d + 2):
            wd = n - 2 * k + 2
            med = np.median(np.concatenate([g, np.full(wd - 1, g[d])]))
            members = list(np.flatnonzero(g == med))
            sel, _ = orc.window_cwvmf(v, k)
            assert sel == tie_rule_pick(members, n)


@pytest.mark.parametrize("n", [9, 25])
def test_cwvmf_brute_force_scipy(orc, n):
    """Eq. (9)'s weighted sum of scipy Euclidean distances, every level k;
    at k = d the weights are all 1 and the CWVMF is the order-2 VMF."""
    rng = np.random.default_rng(33 + n)
    d = (n - 1) // 2
    for _ in range(40):
        v = rng.integers(0, 256, (n, 3)).astype(float)
        D = cdist(v, v)
        for k in range(1, d + 2):
            w = np.ones(n)
            w[d] = n - 2 * k + 2
            s = D @ w
            assert orc.window_cwvmf(v, k)[0] == int(np.argmin(s))
        assert orc.window_cwvmf(v, d + 1)[0] == orc.window(v, "vmf", order=2)[0]


def test_acwddf_switching_sum_matches_scipy(orc):
    """The switching sum is sum over the three levels of the angle (scipy
    cosine distance -> arccos) times the Euclidean distance between the CWVMF
    output and the centre; the output follows the test against T."""
    rng = np.random.default_rng(35)
    for n in (9, 25):
        d = (n - 1) // 2
        for _ in range(40):
            v = rng.integers(1, 256, (n, 3)).astype(float)
            v[d] = rng.integers(1, 256, 3)
            for T in (10.8, 0.5, 200.0):
                sel, cw, s, fl = orc.window_acwddf(v, T=T)
                ref = 0.0
                for y in cw:
                    cosd = cdist(v[[y]], v[[d]], "cosine")[0, 0]
                    ref += math.acos(min(1.0, max(-1.0, 1.0 - cosd))) * cdist(v[[y]], v[[d]])[0, 0]
                assert abs(s - ref) <= 1e-7 * max(1.0, ref)
                if not fl & orc.FLAG_GRAY:
                    ddf = orc.window(v, "ddf", 0.5, "exact")[0]
                    assert sel == (ddf if s > T else d)


@pytest.mark.parametrize("win", [3, 5])
@pytest.mark.parametrize("dist", ["exact", "minimax", "rgb"])
def test_acwddf_threshold_limits(orc, win, dist):
    """T above any attainable sum: the identity filter (the input image).  T
    below 0: the DDF (Eq. (3), p = 1/2) everywhere."""
    from paper_1009_0958_gb300 import synth
    _, img = synth.make_image(19, 23, 37, 0.2, rectangles=3)
    hi = orc.filter_acwddf(img, win, dist, T=1e30)
    assert np.array_equal(hi["out"], img) and np.all(hi["idx"] == (win * win - 1) // 2)
    lo = orc.filter_acwddf(img, win, dist, T=-1.0)
    ddf = orc.filter_u8(img, win, "ddf", 0.5, dist)
    assert np.array_equal(lo["idx"], ddf["idx"]) and np.array_equal(lo["out"], ddf["out"])


def test_acwddf_rejects_bad_levels(orc):
    v = np.zeros((9, 3))
    with pytest.raises(ValueError):
        orc.window_acwddf(v, lam=0)
    with pytest.raises(ValueError):
        orc.window_acwddf(v, lam=4)     # 3x3: k would exceed d = 5
    orc.window_acwddf(v, lam=3)
