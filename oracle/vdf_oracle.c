/*
 * vdf_oracle.c -- CPU oracle for the directional vector filters (BVDF, DDF)
 * and the vector median filter (VMF).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg may load it; the library never calls it.
 * It shares no code, header or constant with the CUDA sources.
 *
 * What it computes (M. E. Celebi, "Real-time implementation of
 * order-statistics based directional filters"):
 *   - Section II: every pixel x(r,c) of an M x N RGB image is replaced by the
 *     output of a filter over the sqrt(n) x sqrt(n) window W(r,c) centred on
 *     it.  Window members are taken in raster order, i = (dy+R)*w + (dx+R),
 *     so the centre is i = (n-1)/2 (the paper's d = (n+1)/2, 1-based).
 *     Pixels outside the image are replaced by the nearest edge pixel.
 *   - Eq. (2), BVDF: argmin_i sum_j A(x_i, x_j),
 *       A(x, y) = acos(<x, y> / (|x| |y|)).
 *   - Eq. (3), DDF: argmin_i (sum_j A)^p * (sum_j L2)^(1-p), with L2 the
 *     Minkowski distance of Eq. (1) at order 2 (Section III).  p = 1/2 orders
 *     candidates exactly like Eq. (3)'s plain product.
 *   - Eq. (1), VMF: argmin_i sum_j L(x_i, x_j), L the Minkowski distance
 *     (sum_k |x_k - y_k|^o)^(1/o).  Orders o = 1 and 2, and the limit
 *     o -> infinity, max_k |x_k - y_k|; the same orders may replace L2 inside
 *     the DDF.  Section III uses order 2 throughout.
 *   - Eq. (9), ACWDDF (Section 3.2): the DDF output if
 *     sum_{k=lambda}^{lambda+2} A(y_k, x_d) L2(y_k, x_d) > T, else the centre
 *     x_d, where y_k is the centre-weighted VMF output at smoothing level k,
 *     argmin_i sum_j w_j(k) L2(x_i, x_j) with w_d(k) = n - 2k + 2 and w_j = 1
 *     otherwise.  Readings: Eq. (9) names the outputs of the switching test
 *     CWDDF^k but defines CWVMF^k; the defined CWVMF^k are used.  The DDF
 *     inside is Eq. (3)'s plain product (p = 1/2 here) with A of the distance
 *     mode (Method 2 through Eq. (10), as the paper does for this filter);
 *     k stays within [1, d] (d = (n+1)/2, 1-based), so lambda is in
 *     [1, d - 2]; the test is strict (> T).
 *   - Method 1 (Section 2.1, Eqs. (4)-(6), Table 1): A replaced by the
 *     degree-q minimax polynomial of Table 1: P_ACOS(z) for z < 0.5 and
 *     P_ASIN(tau) with tau = sqrt(1 - z) for z >= 0.5.
 *   - Method 2 (Section 2.2, Eq. (7)): A replaced by B, the L2 distance of the
 *     chromaticity vectors x / (x1 + x2 + x3).  Inside DDF the value is first
 *     mapped through Eq. (10), A ~ 1.436437 B + 0.027664 (Section 3.2).
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes):
 *   - zero vectors: the cosine of a pair with a zero vector is taken as 0, so
 *     A = pi/2 and the minimax value is P_ACOS(0); a zero vector's
 *     chromaticity is the zero vector;
 *   - the power in DDF uses max(sum_j A, 0) (only the q = 3 polynomial can
 *     make the sum negative) and 0^0 = 1;
 *   - ties: if the centre attains the minimum it is selected, otherwise the
 *     lowest raster index among the minimisers.
 *
 * How the minimum is decided.  All scores are first evaluated in double
 * precision ("screening").  Candidates within 1e-8 (relative, with a 1e-3
 * floor) of the double minimum are re-evaluated in binary128 (_Float128) by
 * the literal formulas above.  Binary128 values within 1e-24 of each other
 * are a tie.  Pixels whose binary128 gap is non-zero but below 1e-9 are
 * flagged "gray": there a double-precision implementation cannot tell a tie
 * from a non-tie.
 *
 * Screening evaluates A through the identity
 *     acos(<x,y>/(|x||y|)) = atan2(|x cross y|, <x,y>)     (<x,y> >= 0),
 * which is well conditioned for nearly parallel vectors; the minimax branch
 * value 1 - z is evaluated as |x cross y|^2 / (s (s + <x,y>)) with s = |x||y|
 * (the same real number), and B as sqrt(sum_k (s_y x_k - s_x y_k)^2) /
 * (s_x s_y).  The binary128 stage uses the paper's formulas as written.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef _Float128 q128;

enum { O_BVDF = 0, O_DDF = 1, O_VMF = 2 };
/* Minkowski order of Eq. (1): 1, 2, or 0 for the limit of infinite order. */
enum { O_LINF = 0, O_L1 = 1, O_L2 = 2 };
enum { O_EXACT = 0, O_MINIMAX = 1, O_RGB = 2 };

/* Flags written per pixel. */
enum { O_FLAG_ESCALATED = 1, O_FLAG_TIE = 2, O_FLAG_GRAY = 4 };

/* Table 1 (minimax polynomials), as printed: rows q = 2, 3, 4, coefficients
 * a_0 .. a_q.  "ASIN" approximates acos(z) = 2 asin(tau / sqrt 2) as a
 * polynomial in tau = sqrt(1 - z) (Eq. (6)); "ACOS" is a polynomial in z. */
static const char *const TABLE1_ASIN[3][5] = {
    {"1.829125e-03", "1.371117", "1.480266e-01", NULL, NULL},
    {"-1.358425e-04", "1.419488", "-3.090315e-02", "1.666491e-01", NULL},
    {"2.097797e-05", "1.412840", "1.429881e-02", "6.704361e-02", "6.909677e-02"},
};
static const char *const TABLE1_ACOS[3][5] = {
    {"1.569882", "-9.695260e-01", "-1.480266e-01", NULL, NULL},
    {"1.570864", "-1.003730", "3.090318e-02", "-2.356775e-01", NULL},
    {"1.570786", "-9.990285e-01", "-1.429899e-02", "-9.481335e-02", "-1.381942e-01"},
};

/* Eq. (10). */
static const char *const EQ10_SLOPE = "1.436437";
static const char *const EQ10_OFFSET = "0.027664";

typedef struct {
    double asin_d[3][5], acos_d[3][5];
    q128 asin_q[3][5], acos_q[3][5];
    double slope_d, offset_d;
    q128 slope_q, offset_q;
    q128 half_pi_q;
    double half_pi_d;
} consts_t;

static consts_t K;
static int K_ready = 0;

static void init_consts(void)
{
    if (K_ready) return;
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 5; ++k) {
            const char *a = TABLE1_ASIN[r][k], *b = TABLE1_ACOS[r][k];
            K.asin_d[r][k] = a ? strtod(a, NULL) : 0.0;
            K.acos_d[r][k] = b ? strtod(b, NULL) : 0.0;
            K.asin_q[r][k] = a ? strtof128(a, NULL) : (q128)0;
            K.acos_q[r][k] = b ? strtof128(b, NULL) : (q128)0;
        }
    K.slope_d = strtod(EQ10_SLOPE, NULL);
    K.offset_d = strtod(EQ10_OFFSET, NULL);
    K.slope_q = strtof128(EQ10_SLOPE, NULL);
    K.offset_q = strtof128(EQ10_OFFSET, NULL);
    K.half_pi_q = acosf128((q128)0);
    K.half_pi_d = acos(0.0);
    K_ready = 1;
}

/* ---------------------------------------------------------------- terms -- */

/* Inner products and derived quantities of one pair, in double.  For uint8
 * inputs every one of these is an exact integer below 2^53; for float32
 * inputs the products are exact and each sum is rounded once. */
static double dot3_d(const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; }

static double cross2_d(const double *x, const double *y)
{
    double c0 = x[1] * y[2] - x[2] * y[1];
    double c1 = x[2] * y[0] - x[0] * y[2];
    double c2 = x[0] * y[1] - x[1] * y[0];
    return c0 * c0 + c1 * c1 + c2 * c2;
}

static q128 dot3_q(const double *x, const double *y)
{
    return (q128)x[0] * y[0] + (q128)x[1] * y[1] + (q128)x[2] * y[2];
}

/* Eq. (4)-(6) branch test z >= 1/2, i.e. 4 <x,y>^2 >= |x|^2 |y|^2, decided
 * in binary128 (exact for uint8 and float32 inputs). */
static int minimax_upper_branch(const double *x, const double *y)
{
    q128 d = dot3_q(x, y);
    q128 P = dot3_q(x, x) * dot3_q(y, y);
    if (P == 0) return 0;                        /* zero vector: z := 0 */
    return 4 * d * d >= P;
}

/* Eq. (2) angle, double screening value. */
static double angle_d(const double *x, const double *y)
{
    double P = dot3_d(x, x) * dot3_d(y, y);
    if (P == 0.0) return K.half_pi_d;
    return atan2(sqrt(cross2_d(x, y)), dot3_d(x, y));
}

/* Eq. (2) angle, binary128, as written. */
static q128 angle_q(const double *x, const double *y)
{
    q128 P = dot3_q(x, x) * dot3_q(y, y);
    if (P == 0) return K.half_pi_q;
    q128 z = dot3_q(x, y) / sqrtf128(P);
    if (z > 1) z = 1;                            /* never taken for exact inputs */
    return acosf128(z);
}

static double horner_d(const double *a, int q, double t)
{
    double v = a[q];
    for (int k = q - 1; k >= 0; --k) v = v * t + a[k];
    return v;
}

static q128 horner_q(const q128 *a, int q, q128 t)
{
    q128 v = a[q];
    for (int k = q - 1; k >= 0; --k) v = v * t + a[k];
    return v;
}

/* Method 1: minimax replacement of A, double screening value. */
static double minimax_d(const double *x, const double *y, int q)
{
    double nx = dot3_d(x, x), ny = dot3_d(y, y);
    if (nx * ny == 0.0) return horner_d(K.acos_d[q - 2], q, 0.0);
    double s = sqrt(nx * ny), d = dot3_d(x, y);
    if (minimax_upper_branch(x, y)) {
        double one_minus_z = cross2_d(x, y) / (s * (s + d));
        return horner_d(K.asin_d[q - 2], q, sqrt(one_minus_z));
    }
    return horner_d(K.acos_d[q - 2], q, d / s);
}

/* Method 1, binary128, as written: z, then tau = sqrt(1 - z). */
static q128 minimax_q(const double *x, const double *y, int q)
{
    q128 P = dot3_q(x, x) * dot3_q(y, y);
    if (P == 0) return horner_q(K.acos_q[q - 2], q, 0);
    q128 z = dot3_q(x, y) / sqrtf128(P);
    if (minimax_upper_branch(x, y)) {
        q128 om = 1 - z;
        if (om < 0) om = 0;
        return horner_q(K.asin_q[q - 2], q, sqrtf128(om));
    }
    return horner_q(K.acos_q[q - 2], q, z);
}

/* Method 2: chromaticity distance B of Eq. (7), double screening value. */
static double chroma_d(const double *x, const double *y)
{
    double sx = x[0] + x[1] + x[2], sy = y[0] + y[1] + y[2];
    if (sx == 0.0 && sy == 0.0) return 0.0;
    if (sx == 0.0) return sqrt(dot3_d(y, y)) / sy;
    if (sy == 0.0) return sqrt(dot3_d(x, x)) / sx;
    double n = 0.0;
    for (int k = 0; k < 3; ++k) {
        double t = sy * x[k] - sx * y[k];
        n += t * t;
    }
    return sqrt(n) / (sx * sy);
}

/* Method 2, binary128, as written: L2 between x / sum(x) and y / sum(y). */
static q128 chroma_q(const double *x, const double *y)
{
    q128 sx = (q128)x[0] + x[1] + x[2], sy = (q128)y[0] + y[1] + y[2];
    q128 n = 0;
    for (int k = 0; k < 3; ++k) {
        q128 a = sx == 0 ? (q128)0 : (q128)x[k] / sx;
        q128 b = sy == 0 ? (q128)0 : (q128)y[k] / sy;
        n += (a - b) * (a - b);
    }
    return sqrtf128(n);
}

/* Eq. (1) at order 2. */
static double l2_d(const double *x, const double *y)
{
    double e = 0.0;
    for (int k = 0; k < 3; ++k) e += (x[k] - y[k]) * (x[k] - y[k]);
    return sqrt(e);
}

static q128 l2_q(const double *x, const double *y)
{
    q128 e = 0;
    for (int k = 0; k < 3; ++k) {
        q128 t = (q128)x[k] - y[k];
        e += t * t;
    }
    return sqrtf128(e);
}

/* Eq. (1) at order 1, 2 or infinity (the maximum of the component
 * differences, the limit of the order-o distance as o grows). */
static double lterm_d(const double *x, const double *y, int lp)
{
    if (lp == O_L2) return l2_d(x, y);
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double a = fabs(x[k] - y[k]);
        if (lp == O_L1) s += a;
        else if (a > s) s = a;
    }
    return s;
}

static q128 lterm_q(const double *x, const double *y, int lp)
{
    if (lp == O_L2) return l2_q(x, y);
    q128 s = 0;
    for (int k = 0; k < 3; ++k) {
        q128 a = (q128)x[k] - y[k];
        if (a < 0) a = -a;
        if (lp == O_L1) s += a;
        else if (a > s) s = a;
    }
    return s;
}

/* Angular term of the chosen distance mode (the value summed into the first
 * aggregate).  For DDF with Method 2 the chromaticity distance goes through
 * Eq. (10) first. */
static double aterm_d(const double *x, const double *y, int filter, int dist, int q)
{
    switch (dist) {
    case O_EXACT: return angle_d(x, y);
    case O_MINIMAX: return minimax_d(x, y, q);
    default: {
        double b = chroma_d(x, y);
        return filter == O_DDF ? K.slope_d * b + K.offset_d : b;
    }
    }
}

static q128 aterm_q(const double *x, const double *y, int filter, int dist, int q)
{
    switch (dist) {
    case O_EXACT: return angle_q(x, y);
    case O_MINIMAX: return minimax_q(x, y, q);
    default: {
        q128 b = chroma_q(x, y);
        return filter == O_DDF ? K.slope_q * b + K.offset_q : b;
    }
    }
}

/* ------------------------------------------------------------- windows -- */

typedef struct {
    int filter, dist, q;
    double p;
    int lp;   /* Minkowski order of the distance term (DDF, VMF) */
} cfg_t;

/* Minimum of n scores with the tie rule: screening in double, binary128
 * re-evaluation (score_q(i, ctx)) of the candidates within 1e-8 of the double
 * minimum, ties within 1e-24; *flags receives the O_FLAG_* bits. */
typedef q128 (*score_q_fn)(int i, const void *ctx);

static int decide_min(const double *score, int n, score_q_fn fq, const void *ctx, int *flags);

/* Scores of all n members in double.  sa/sl receive the aggregates. */
static void scores_d(const double *v, int n, const cfg_t *c, double *score, double *sa, double *sl)
{
    for (int i = 0; i < n; ++i) {
        double a = 0.0, l = 0.0;
        for (int j = 0; j < n; ++j) {
            if (c->filter != O_VMF) a += aterm_d(v + 3 * i, v + 3 * j, c->filter, c->dist, c->q);
            if (c->filter != O_BVDF) l += lterm_d(v + 3 * i, v + 3 * j, c->lp);
        }
        sa[i] = a;
        sl[i] = l;
        if (c->filter == O_BVDF) score[i] = a;
        else if (c->filter == O_VMF) score[i] = l;
        else score[i] = pow(a > 0.0 ? a : 0.0, c->p) * pow(l, 1.0 - c->p);
    }
}

/* One member's aggregates and score in binary128. */
static q128 score_q(const double *v, int n, int i, const cfg_t *c, q128 *sa, q128 *sl)
{
    q128 a = 0, l = 0;
    for (int j = 0; j < n; ++j) {
        if (c->filter != O_VMF) a += aterm_q(v + 3 * i, v + 3 * j, c->filter, c->dist, c->q);
        if (c->filter != O_BVDF) l += lterm_q(v + 3 * i, v + 3 * j, c->lp);
    }
    if (sa) *sa = a;
    if (sl) *sl = l;
    if (c->filter == O_BVDF) return a;
    if (c->filter == O_VMF) return l;
    q128 pq = (q128)c->p;
    return powf128(a > 0 ? a : (q128)0, pq) * powf128(l, 1 - pq);
}

#define O_MAXN 49

/* Select the output member of one window (vectors v, n of them, raster
 * order).  Returns the member index; *flags receives the O_FLAG_* bits.  If
 * agg is non-NULL it receives the binary128 aggregates rounded to double,
 * laid out as agg[2*i] = sum_j A (0 for VMF), agg[2*i+1] = sum_j L (0 for
 * BVDF). */
static int select_window(const double *v, int n, const cfg_t *c, int *flags, double *agg)
{
    double score[O_MAXN], sa[O_MAXN], sl[O_MAXN];
    scores_d(v, n, c, score, sa, sl);
    const int centre = (n - 1) / 2;
    *flags = 0;

    if (agg) {
        for (int i = 0; i < n; ++i) {
            q128 a, l;
            score_q(v, n, i, c, &a, &l);
            agg[2 * i] = (double)a;
            agg[2 * i + 1] = (double)l;
        }
    }

    double m = score[0];
    for (int i = 1; i < n; ++i)
        if (score[i] < m) m = score[i];
    const double screen = 1e-8 * (fabs(m) + 1e-3);
    int cand[O_MAXN], nc = 0;
    for (int i = 0; i < n; ++i)
        if (score[i] - m <= screen) cand[nc++] = i;
    if (nc == 1) return cand[0];

    *flags |= O_FLAG_ESCALATED;
    q128 s[O_MAXN];
    q128 mq = 0;
    for (int k = 0; k < nc; ++k) {
        s[k] = score_q(v, n, cand[k], c, NULL, NULL);
        if (k == 0 || s[k] < mq) mq = s[k];
    }
    q128 scale = (mq < 0 ? -mq : mq) + (q128)1e-3;
    q128 tie_tol = (q128)1e-24 * scale;
    q128 gray_tol = (q128)1e-9 * scale;
    int best = -1, nt = 0;
    for (int k = 0; k < nc; ++k) {
        q128 gap = s[k] - mq;
        if (gap <= tie_tol) {
            ++nt;
            if (cand[k] == centre) best = centre;
            else if (best < 0) best = cand[k];
        } else if (gap <= gray_tol) {
            *flags |= O_FLAG_GRAY;
        }
    }
    if (nt > 1) *flags |= O_FLAG_TIE;
    return best;
}

static int decide_min(const double *score, int n, score_q_fn fq, const void *ctx, int *flags)
{
    const int centre = (n - 1) / 2;
    double m = score[0];
    for (int i = 1; i < n; ++i)
        if (score[i] < m) m = score[i];
    const double screen = 1e-8 * (fabs(m) + 1e-3);
    int cand[O_MAXN], nc = 0;
    for (int i = 0; i < n; ++i)
        if (score[i] - m <= screen) cand[nc++] = i;
    if (nc == 1) return cand[0];
    *flags |= O_FLAG_ESCALATED;
    q128 s[O_MAXN], mq = 0;
    for (int k = 0; k < nc; ++k) {
        s[k] = fq(cand[k], ctx);
        if (k == 0 || s[k] < mq) mq = s[k];
    }
    q128 scale = (mq < 0 ? -mq : mq) + (q128)1e-3;
    int best = -1, nt = 0;
    for (int k = 0; k < nc; ++k) {
        q128 gap = s[k] - mq;
        if (gap <= (q128)1e-24 * scale) {
            ++nt;
            if (cand[k] == centre) best = centre;
            else if (best < 0) best = cand[k];
        } else if (gap <= (q128)1e-9 * scale) {
            *flags |= O_FLAG_GRAY;
        }
    }
    if (nt > 1) *flags |= O_FLAG_TIE;
    return best;
}

/* ------------------------------------------------------- ACWDDF, Eq. (9) -- */

typedef struct {
    const double *v;
    int n;
    double wd;   /* weight of the centre member */
} cw_ctx;

static q128 cwvmf_q(int i, const void *p)
{
    const cw_ctx *c = (const cw_ctx *)p;
    const int d = (c->n - 1) / 2;
    q128 s = 0;
    for (int j = 0; j < c->n; ++j) s += (j == d ? (q128)c->wd : (q128)1) * l2_q(c->v + 3 * i, c->v + 3 * j);
    return s;
}

/* Centre-weighted VMF of Eq. (9) at smoothing level k (1-based, k <= d). */
static int select_cwvmf(const double *v, int n, int k, int *flags)
{
    const int d = (n - 1) / 2;
    const cw_ctx c = {v, n, (double)(n - 2 * k + 2)};
    double score[O_MAXN];
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += (j == d ? c.wd : 1.0) * l2_d(v + 3 * i, v + 3 * j);
        score[i] = s;
    }
    return decide_min(score, n, cwvmf_q, &c, flags);
}

/* ACWDDF of one window: returns the member index; cw[3] (optional) receives
 * the three CWVMF outputs, *sum (optional) the switching sum. */
static int select_acwddf(const double *v, int n, int dist, int q, int lambda, double T, int *flags, int *cw,
                         double *sum)
{
    const cfg_t ddf = {O_DDF, dist, q, 0.5, O_L2};
    const int d = (n - 1) / 2;
    int fl = 0;
    const int sel = select_window(v, n, &ddf, &fl, NULL);
    q128 sq = 0;
    for (int k = lambda; k <= lambda + 2; ++k) {
        const int y = select_cwvmf(v, n, k, &fl);
        if (cw) cw[k - lambda] = y;
        sq += aterm_q(v + 3 * y, v + 3 * d, O_DDF, dist, q) * l2_q(v + 3 * y, v + 3 * d);
    }
    const q128 gap = sq - (q128)T;
    if ((gap < 0 ? -gap : gap) <= (q128)1e-9 * ((q128)fabs(T) + 1)) fl |= O_FLAG_GRAY;
    if (sum) *sum = (double)sq;
    *flags = fl;
    return sq > (q128)T ? sel : d;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int check_cfg(int win, int filter, double p, int dist, int q, int lp)
{
    if (win < 1 || win > 7 || (win & 1) == 0) return -1;
    if (filter != O_BVDF && filter != O_DDF && filter != O_VMF) return -1;
    if (lp != O_L1 && lp != O_L2 && lp != O_LINF) return -1;
    if (dist < O_EXACT || dist > O_RGB) return -1;
    if (dist == O_MINIMAX && (q < 2 || q > 4)) return -1;
    if (filter == O_DDF && !(p >= 0.0 && p <= 1.0)) return -1;
    return 0;
}

/* ------------------------------------------------------------- exports -- */

/* Filter an M x N uint8 HWC image.  Pixels: all of them when pix == NULL
 * (outputs then have M*N entries), else the `count` linear pixel ids in pix
 * (outputs have `count` entries).  out: 3 bytes per output pixel; idx: the
 * selected member's raster index; flags (optional): O_FLAG_* bits; agg
 * (optional): 2*n doubles per output pixel.  Returns 0 or -1 on bad input. */
int vdf_oracle_filter_u8_lp(const uint8_t *img, int M, int N, int win, int filter, double p, int lp, int dist,
                            int q, const int64_t *pix, int64_t count, uint8_t *out, int8_t *idx, int32_t *flags,
                            double *agg, int nthreads)
{
    if (!img || !out || M < 1 || N < 1 || check_cfg(win, filter, p, dist, q, lp)) return -1;
    init_consts();
    const int R = win / 2, n = win * win;
    const cfg_t c = {filter, dist, q, p, lp};
    const int64_t total = pix ? count : (int64_t)M * N;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t t = 0; t < total; ++t) {
        const int64_t lin = pix ? pix[t] : t;
        const int r = (int)(lin / N), col = (int)(lin % N);
        double v[3 * O_MAXN];
        int i = 0;
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx, ++i) {
                const uint8_t *px = img + 3 * ((int64_t)clampi(r + dy, 0, M - 1) * N + clampi(col + dx, 0, N - 1));
                v[3 * i] = px[0];
                v[3 * i + 1] = px[1];
                v[3 * i + 2] = px[2];
            }
        int fl;
        int sel = select_window(v, n, &c, &fl, agg ? agg + (int64_t)2 * n * t : NULL);
        out[3 * t] = (uint8_t)v[3 * sel];
        out[3 * t + 1] = (uint8_t)v[3 * sel + 1];
        out[3 * t + 2] = (uint8_t)v[3 * sel + 2];
        if (idx) idx[t] = (int8_t)sel;
        if (flags) flags[t] = fl;
    }
    return 0;
}

/* The same at Minkowski order 2. */
int vdf_oracle_filter_u8(const uint8_t *img, int M, int N, int win, int filter, double p, int dist, int q,
                         const int64_t *pix, int64_t count, uint8_t *out, int8_t *idx, int32_t *flags,
                         double *agg, int nthreads)
{
    return vdf_oracle_filter_u8_lp(img, M, N, win, filter, p, O_L2, dist, q, pix, count, out, idx, flags, agg,
                                   nthreads);
}

/* Filter a B x 3 x M x N float32 (NCHW) batch; same conventions, pixel ids
 * run over B*M*N; Minkowski order 2. */
int vdf_oracle_filter_f32(const float *img, int B, int M, int N, int win, int filter, double p, int dist, int q,
                          const int64_t *pix, int64_t count, float *out, int8_t *idx, int32_t *flags,
                          double *agg, int nthreads)
{
    if (!img || !out || B < 1 || M < 1 || N < 1 || check_cfg(win, filter, p, dist, q, O_L2)) return -1;
    init_consts();
    const int R = win / 2, n = win * win;
    const cfg_t c = {filter, dist, q, p, O_L2};
    const int64_t plane = (int64_t)M * N;
    const int64_t total = pix ? count : (int64_t)B * plane;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t t = 0; t < total; ++t) {
        const int64_t lin = pix ? pix[t] : t;
        const int64_t b = lin / plane, rc = lin % plane;
        const int r = (int)(rc / N), col = (int)(rc % N);
        const float *base = img + b * 3 * plane;
        double v[3 * O_MAXN];
        int i = 0;
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx, ++i) {
                const int64_t o = (int64_t)clampi(r + dy, 0, M - 1) * N + clampi(col + dx, 0, N - 1);
                for (int k = 0; k < 3; ++k) v[3 * i + k] = base[k * plane + o];
            }
        int fl;
        int sel = select_window(v, n, &c, &fl, agg ? agg + (int64_t)2 * n * t : NULL);
        if (pix) {
            for (int k = 0; k < 3; ++k) out[3 * t + k] = (float)v[3 * sel + k];
        } else {
            float *ob = out + b * 3 * plane;
            for (int k = 0; k < 3; ++k) ob[k * plane + rc] = (float)v[3 * sel + k];
        }
        if (idx) idx[t] = (int8_t)sel;
        if (flags) flags[t] = fl;
    }
    return 0;
}

/* One window given directly as n vectors (n an odd square, raster order).
 * Writes the double screening scores and binary128 aggregates (rounded) and
 * returns the selected index, or -1 on bad input. */
int vdf_oracle_window_lp(const double *v, int n, int filter, double p, int lp, int dist, int q,
                         double *score, double *agg, int32_t *flags)
{
    int w = 1;
    while (w * w < n) ++w;
    if (!v || w * w != n || check_cfg(w, filter, p, dist, q, lp)) return -1;
    init_consts();
    const cfg_t c = {filter, dist, q, p, lp};
    double sa[O_MAXN], sl[O_MAXN], sc[O_MAXN];
    scores_d(v, n, &c, sc, sa, sl);
    if (score) memcpy(score, sc, sizeof(double) * n);
    int fl;
    int sel = select_window(v, n, &c, &fl, agg);
    if (flags) *flags = fl;
    return sel;
}

int vdf_oracle_window(const double *v, int n, int filter, double p, int dist, int q,
                      double *score, double *agg, int32_t *flags)
{
    return vdf_oracle_window_lp(v, n, filter, p, O_L2, dist, q, score, agg, flags);
}

/* One pair term for the pins.  which: 0 = angular term of `dist` (BVDF
 * form), 1 = L2, 2 = L1, 3 = L-infinity.  The double screening value goes to
 * *d; the binary128 value is returned split as *hi + *lo. */
int vdf_oracle_term(const double *x, const double *y, int which, int dist, int q,
                    double *d, double *hi, double *lo)
{
    if (!x || !y || dist < O_EXACT || dist > O_RGB || (dist == O_MINIMAX && (q < 2 || q > 4))) return -1;
    init_consts();
    q128 t;
    if (which >= 1 && which <= 3) {
        const int lp = which == 1 ? O_L2 : (which == 2 ? O_L1 : O_LINF);
        if (d) *d = lterm_d(x, y, lp);
        t = lterm_q(x, y, lp);
    } else {
        if (d) *d = aterm_d(x, y, O_BVDF, dist, q);
        t = aterm_q(x, y, O_BVDF, dist, q);
    }
    double h = (double)t;
    if (hi) *hi = h;
    if (lo) *lo = (double)(t - (q128)h);
    return 0;
}

/* Table 1 polynomial of one branch (0 = ACOS in z, 1 = ASIN in tau) at t,
 * evaluated in binary128 and returned as hi + lo. */
int vdf_oracle_poly(int branch, int q, double t, double *hi, double *lo)
{
    if (q < 2 || q > 4 || branch < 0 || branch > 1) return -1;
    init_consts();
    q128 v = horner_q(branch ? K.asin_q[q - 2] : K.acos_q[q - 2], q, (q128)t);
    double h = (double)v;
    *hi = h;
    *lo = (double)(v - (q128)h);
    return 0;
}

/* ACWDDF (Eq. (9)) of an M x N uint8 image, pixel subset as
 * vdf_oracle_filter_u8.  lambda in [1, d - 2] with d = (win*win + 1)/2. */
int vdf_oracle_filter_acwddf(const uint8_t *img, int M, int N, int win, int dist, int q, int lambda, double T,
                             const int64_t *pix, int64_t count, uint8_t *out, int8_t *idx, int32_t *flags,
                             int nthreads)
{
    const int n = win * win, d1 = (n + 1) / 2;
    if (!img || !out || M < 1 || N < 1 || check_cfg(win, O_DDF, 0.5, dist, q, O_L2)) return -1;
    if (lambda < 1 || lambda > d1 - 2 || !isfinite(T)) return -1;
    init_consts();
    const int R = win / 2;
    const int64_t total = pix ? count : (int64_t)M * N;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t t = 0; t < total; ++t) {
        const int64_t lin = pix ? pix[t] : t;
        const int r = (int)(lin / N), col = (int)(lin % N);
        double v[3 * O_MAXN];
        int i = 0;
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx, ++i) {
                const uint8_t *px = img + 3 * ((int64_t)clampi(r + dy, 0, M - 1) * N + clampi(col + dx, 0, N - 1));
                v[3 * i] = px[0];
                v[3 * i + 1] = px[1];
                v[3 * i + 2] = px[2];
            }
        int fl;
        const int sel = select_acwddf(v, n, dist, q, lambda, T, &fl, NULL, NULL);
        out[3 * t] = (uint8_t)v[3 * sel];
        out[3 * t + 1] = (uint8_t)v[3 * sel + 1];
        out[3 * t + 2] = (uint8_t)v[3 * sel + 2];
        if (idx) idx[t] = (int8_t)sel;
        if (flags) flags[t] = fl;
    }
    return 0;
}

/* ACWDDF of one window (n vectors, raster order), with its intermediate
 * results: cw[3] the CWVMF outputs at k = lambda .. lambda + 2, *sum the
 * switching sum, *flags the O_FLAG_* bits.  Returns the index or -1. */
int vdf_oracle_window_acwddf(const double *v, int n, int dist, int q, int lambda, double T, int32_t *cw,
                             double *sum, int32_t *flags)
{
    int w = 1;
    while (w * w < n) ++w;
    if (!v || w * w != n || check_cfg(w, O_DDF, 0.5, dist, q, O_L2)) return -1;
    if (lambda < 1 || lambda > (n + 1) / 2 - 2 || !isfinite(T)) return -1;
    init_consts();
    int c3[3], fl;
    double s;
    const int sel = select_acwddf(v, n, dist, q, lambda, T, &fl, c3, &s);
    if (cw)
        for (int k = 0; k < 3; ++k) cw[k] = c3[k];
    if (sum) *sum = s;
    if (flags) *flags = fl;
    return sel;
}

/* Centre-weighted VMF of one window at smoothing level k (1..d). */
int vdf_oracle_window_cwvmf(const double *v, int n, int k, int32_t *flags)
{
    int w = 1;
    while (w * w < n) ++w;
    if (!v || w * w != n || (w & 1) == 0 || k < 1 || k > (n + 1) / 2) return -1;
    init_consts();
    int fl = 0;
    const int sel = select_cwvmf(v, n, k, &fl);
    if (flags) *flags = fl;
    return sel;
}

int vdf_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
