// vdf_tile.cuh -- the tile kernel of the directional vector filters.
//
// One CTA filters a TW x TH tile of output pixels.  The candidate region C is
// the tile plus an R-pixel halo (R = win/2): every member of every window of
// the tile lies in C, and so does every pair partner that such a window
// needs.  One thread owns one candidate pixel p of C and accumulates, for
// each of the n windows W(q) that contain p (q = p - e, e in [-R,R]^2), the
// aggregate sum_{j in W(q)} term(x_p, x_j) of Eqs. (2)/(3).
//
// Pair terms are computed once per unordered pair: the (2w-1)^2 - 1 offsets
// between members of a common window are processed in 2R+1 slices of equal
// vertical offset dy' = 0..2R.  In a slice, each p computes its terms with
// the partners p + (dy', dx) and stores them in shared-memory planes; after a
// barrier, p reads its own row (offset +dy') and the mirrored row (offset
// -dy', written by the pixels above it), forms the horizontal window sums and
// adds them into the n accumulators of the windows whose rows they belong to.
// Two plane buffers pipeline the slices: the terms of slice k+1 are computed
// in the same phase as the accumulation of slice k (2R+2 barriers, not 4R+2).
//
// After the slices every thread turns its n aggregates into scores and
// scatters them to the windows (shared memory), and one thread per output
// pixel selects the minimum (Section II: reduced ordering, argmin).
//
// Summation order (relied on by the FP64 recheck kernel, which reproduces it
// bit for bit): a window row sum adds dx = -R-ex .. R-ex left to right; the
// aggregate adds the row sums in the order dy = 0, +1, -1, +2, -2, ...
#pragma once

#include <atomic>
#include <type_traits>
#include <utility>

#include "vdf_internal.cuh"

namespace vdf {

struct TileParams {
    const void *img;       // uint8 HWC, or float32 NCHW (batch)
    void *out;             // same layout and type as img
    int8_t *idx;           // M*N (per image), may be null
    double *agg;           // FP64: M*N*n*2 aggregates, may be null
    float *dbg_fe;         // FP32: M*N*n*2 (score, bound), may be null (diagnostic)
    int2 *recheck_list;    // FP32: {pixel id, member mask} needing the FP64 path
    unsigned *recheck_ctr; // [0] = count, [1] = overflow flag
    unsigned recheck_cap;
    int pix_base;          // added to pixel ids in the recheck list (batches)
    int M, N, B;
    double p;
    int q;
    int lam;               // ACWDDF: first smoothing level lambda and threshold T (Eq. (9))
    double T;
};

template <int R_, int FILTER_, int DIST_, bool FP64_, bool F32IN_, int TW_, int TH_, int NORM_ = NL2, bool ACW_ = false,
          int SQ_ = -1>
struct TileCfg {
    static constexpr int R = R_, FILTER = FILTER_, DIST = DIST_, TW = TW_, TH = TH_, NORM = NORM_;
    static constexpr bool FP64 = FP64_, F32IN = F32IN_;
    // ACWDDF (Eq. (9)): the DDF's aggregates, then the centre-weighted VMF
    // levels and the switch in the selection
    static constexpr bool ACW = ACW_;
    static_assert(!ACW || (FILTER == DDF && NORM == NL2 && !F32IN), "ACWDDF: uint8 DDF at order 2");
    // Score slots (FP32 DDF with p = SQ / 4, exact or chromaticity terms):
    // each (window, member) slot holds the score Omega^4 = SA^SQ SL^(4-SQ),
    // formed where the aggregates are emitted, instead of the two aggregates
    // (half the slot bytes, so that two blocks share an SM).  -1: raw slots.
    static constexpr int SQ = SQ_;
    static_assert(SQ < 0 || (FILTER == DDF && !FP64 && !F32IN && !ACW && NORM == NL2 && DIST != MINIMAX && SQ <= 4),
                  "score slots: FP32 uint8 DDF with p = SQ / 4, exact or chromaticity terms");
    static_assert(FILTER != VMF || DIST == EXACT, "VMF has no angular term");
    static_assert(!F32IN || (FILTER != VMF && NORM == NL2), "float input: BVDF / DDF at order 2");
    // VMF at order 1 or infinity: the aggregates are exact integers in both
    // precisions, so equal scores are exact ties
    static constexpr bool EXACT_SCORES = FILTER == VMF && NORM != NL2;
    static constexpr int W = 2 * R + 1, NW = W * W, CENTRE = (NW - 1) / 2;
    static constexpr int CW = TW + 2 * R, CH = TH + 2 * R, NC = CW * CH;
    static constexpr int NT = (NC + 31) / 32 * 32;
    static constexpr int PXW = CW + 4 * R;            // pixel columns -2R .. CW+2R-1 of C
    static constexpr int PLW = CW + 4 * R;            // plane columns -2R .. CW+2R-1
    static constexpr int PLH = CH + 2 * R;            // plane rows -2R .. CH-1
    static constexpr int NPL = 4 * R + 1;             // planes per slice (dx = -2R..2R)
    static constexpr bool AUX = !FP64 && (DIST != EXACT);
    using Real = typename std::conditional<FP64, double, float>::type;
    using Pix = typename std::conditional<FP64 && !F32IN, int4, float4>::type;
    // DDF terms and aggregates are (angular, L2) pairs: .x and .y
    using Pair = typename std::conditional<FP64, double2, float2>::type;
    using PlaneT = typename std::conditional<FILTER == DDF, Pair, Real>::type;
    // per (window, member) slot: the raw aggregates (FP64: later the score in
    // place); one value for the single-aggregate filters (BVDF, VMF) and for
    // score slots
    using HwT = typename std::conditional<FILTER == DDF && SQ < 0,
                                          typename std::conditional<FP64, double2, float2>::type, Real>::type;
    static constexpr size_t PIX_BYTES = sizeof(Pix) * CH * PXW;
    static constexpr size_t AUX_BYTES = AUX ? (sizeof(Aux) * CH * PXW + 15) / 16 * 16 : 0;
    // FP32: packed RGB key per pixel for the identical-vector test
    static constexpr size_t KEY_BYTES = !FP64 ? (sizeof(unsigned) * CH * PXW + 15) / 16 * 16 : 0;
    // FP64: padded planes (PLH x PLW each).  FP32: planes packed with stride
    // NC (entry = thread index); reads for pixels outside C land in the
    // neighbouring plane, the preceding arrays or a 4R-entry tail and only
    // feed windows outside the tile
    static constexpr int PSTRIDE = FP64 ? PLH * PLW : NC;
    static constexpr int PBUF = FP64 ? NPL * PLH * PLW : NPL * NC + 4 * R;
    static constexpr size_t PLANE_BYTES = sizeof(PlaneT) * PBUF;
    static constexpr size_t HW_BYTES = sizeof(HwT) * TW * TH * NW;
    // two plane buffers (slice pipeline); FP64 reuses them for the per-window
    // slots afterwards, FP32 writes each slot as soon as its aggregate is final.
    // FP32 DDF 5x5 with raw slots takes one plane buffer (the slices then take
    // two barriers each, mirrored row first) where that, and only that, lets
    // two blocks share an SM (24x12 and 32x8)
    static constexpr bool TWO_CTA_REGS = 2 * NT * (R == 1 ? 48 : 64) <= 65536;
    static constexpr size_t FIXED_BYTES = PIX_BYTES + AUX_BYTES + KEY_BYTES + HW_BYTES;
    static constexpr size_t PLANE1_BYTES = (PLANE_BYTES + 15) / 16 * 16;
    static constexpr size_t PLANE2_BYTES = (2 * PLANE_BYTES + 15) / 16 * 16;
    static constexpr bool PB1 = !FP64 && SQ < 0 && FILTER == DDF && R == 2 && TWO_CTA_REGS &&
                                2 * (FIXED_BYTES + PLANE2_BYTES + 1024) > 228 * 1024 &&
                                2 * (FIXED_BYTES + PLANE1_BYTES + 1024) <= 228 * 1024;
    static constexpr size_t PLANES2_BYTES = PB1 ? PLANE1_BYTES : PLANE2_BYTES;
    static constexpr size_t HW_OFFSET = FP64 ? 0 : PLANES2_BYTES;
    static constexpr size_t UNION_BYTES =
        FP64 ? (2 * PLANE_BYTES > HW_BYTES ? 2 * PLANE_BYTES : HW_BYTES) : PLANES2_BYTES + HW_BYTES;
    static constexpr size_t SMEM = PIX_BYTES + AUX_BYTES + KEY_BYTES + UNION_BYTES;
    static_assert(FP64 || PIX_BYTES >= sizeof(PlaneT) * (2 * R * CW + 2 * R), "FP32 plane reads stay in the block");
    // CTAs per SM the register budget is sized for: two when two fit in the
    // SM's 228 KB of shared memory (1 KB reserved per CTA) with at least 48
    // registers per thread (64 for 5x5, whose slice pipeline spills below
    // that), so one CTA's barrier waits overlap the other's work
    static constexpr int MINB = (2 * (SMEM + 1024) <= 228 * 1024 && TWO_CTA_REGS) ? 2 : 1;
};

// ------------------------------------------------------------ scores ------

// FP64 score of one member from its aggregates (Eq. (2) / Eq. (3)).  DDF is
// compared in the log domain: p ln(max(SA,0)) + (1-p) ln(SL), 0 ln 0 := 0.
template <int FILTER>
__device__ __forceinline__ double score64(double sa, double sl, double p)
{
    if (FILTER != DDF) return sa;   // BVDF: sum of angles; VMF: sum of distances
    double f = 0.0;
    if (p > 0.0) f = __dmul_rn(p, log(sa > 0.0 ? sa : 0.0));
    if (p < 1.0) f = __dadd_rn(f, __dmul_rn(1.0 - p, log(sl)));
    return f;
}

// Member selection of the FP64 path: scores within 1e-11 of the minimum
// (relative with floor 1e-3 for BVDF; absolute in the log domain for DDF)
// are tied; the centre wins a tie, else the lowest index.
template <int FILTER, int NW, class F>
__device__ __forceinline__ int select64(F f)
{
    double m = f(0);
#pragma unroll 1
    for (int k = 1; k < NW; ++k) m = fmin(m, f(k));
    const double tol = (FILTER != DDF) ? 1e-11 * fmax(fabs(m), 1e-3) : 1e-11;
    constexpr int c = (NW - 1) / 2;
    if (f(c) == m || f(c) - m <= tol) return c;
#pragma unroll 1
    for (int k = 0; k < NW; ++k)
        if (f(k) == m || f(k) - m <= tol) return k;
    return c;   // not reached
}

// FP32 score and certified bound.  Relative error bounds (in units of
// u = 2^-24) of the aggregates: angle kAngleU + 4R (terms + two summation
// stages), chromaticity 11 + 4R (+2 for Eq. (10)), L2 6 + 4R; Method 1 has
// an absolute bound 24u per term plus 4R u |SA|.  Bounds are doubled.
// Omega^4 = SA^a SL^(4-a) for p = a/4, with at most three rounded products.
template <int A>
__device__ __forceinline__ float pow4_product(float sa0, float sl)
{
    const float sa2 = sa0 * sa0, sl2 = sl * sl;
    if constexpr (A == 0) return sl2 * sl2;
    else if constexpr (A == 1) return sa0 * (sl * sl2);
    else if constexpr (A == 2) return sa2 * sl2;
    else if constexpr (A == 3) return (sa0 * sa2) * sl;
    else return sa2 * sa2;
}

constexpr float kSafety = 2.0f;   // factor applied to every analytic FP32 bound

// Relative bound of Omega^4 for the exact and chromaticity modes (the
// angular and L2 aggregate bounds of score32 below, a of them and 4 - a).
template <int R, int DIST, bool F32IN = false>
__device__ __forceinline__ float pow4_erel(int a)
{
    constexpr float S = 4.0f * R;
    constexpr float relA = (DIST == RGB ? 13.0f + S : (F32IN ? kAngleFU : kAngleU) + S) * kU;
    constexpr float relL = ((F32IN ? 8.0f : 6.0f) + S) * kU;
    return kSafety * (a * relA + (4 - a) * relL + 3.0f * kU);
}

template <int R, int FILTER, int DIST, bool F32IN = false, int NORM = NL2>
__device__ __forceinline__ float2 score32(float sa, float sl, float p, int quarter)
{
    constexpr int NW = (2 * R + 1) * (2 * R + 1);
    constexpr float S = 4.0f * R;
    constexpr float kA = F32IN ? kAngleFU : kAngleU, kL = F32IN ? 8.0f : 6.0f;   // term bounds, float / integer input
    if (FILTER == VMF)   // sum of distances: order 2 as the L2 aggregate, orders 1 and infinity exact
        return make_float2(sa, NORM == NL2 ? kSafety * (kL + S) * kU * sa : 0.0f);
    if (FILTER == BVDF) {
        float E;
        if (DIST == EXACT) E = (kA + S) * kU * sa;
        else if (DIST == RGB) E = (11.0f + S) * kU * sa;
        else E = 24.0f * NW * kU + S * kU * (fabsf(sa) + NW * 2e-4f);
        return make_float2(sa, kSafety * E);
    }
    // DDF, log2 domain
    float relA;
    bool unsure = false;
    if (DIST == EXACT) relA = (kA + S) * kU;
    else if (DIST == RGB) relA = (13.0f + S) * kU;
    else {
        const float absA = 24.0f * NW * kU + S * kU * (fabsf(sa) + NW * 2e-4f);
        unsure = (p > 0.0f) && (sa <= 2.0f * absA);
        relA = absA / fmaxf(sa, 1e-30f);
    }
    if (unsure) return make_float2(-1e30f, INFINITY);   // Method 1 sum too close to 0 to take its log
    const float relL = (kL + S) * kU;
    if (quarter >= 0) {
        // p = a/4: Omega^4 = SA^a SL^(4-a) orders like Omega, with a relative
        // bound (a relA + (4-a) relL + 3 roundings) and no logarithm
        const float sa0 = fmaxf(sa, 0.0f);
        float g;
        switch (quarter) {
        case 0: g = pow4_product<0>(sa0, sl); break;
        case 1: g = pow4_product<1>(sa0, sl); break;
        case 2: g = pow4_product<2>(sa0, sl); break;
        case 3: g = pow4_product<3>(sa0, sl); break;
        default: g = pow4_product<4>(sa0, sl); break;
        }
        if (g == 0.0f) return make_float2(0.0f, 0.0f);   // an aggregate is exactly 0
        if constexpr (DIST != MINIMAX) return make_float2(g, g * pow4_erel<R, DIST, F32IN>(quarter));
        return make_float2(g, kSafety * g * (quarter * relA + (4 - quarter) * relL + 3.0f * kU));
    }
    constexpr float kLg2Abs = 1.6e-7f;   // __log2f on [1,2): 2^-22.6
    constexpr float kInvLn2 = 1.4426950f;
    float f = 0.0f, E = 0.0f, lsum = 0.0f;
    if (p > 0.0f) {
        const float l1 = log2_rr(fmaxf(sa, 0.0f));
        f = p * l1;
        E += p * relA * kInvLn2 + kLg2Abs + kU * fabsf(l1);
        lsum += fabsf(l1);
    }
    if (p < 1.0f) {
        const float l2 = log2_rr(sl);
        f = fmaf(1.0f - p, l2, f);
        E += (1.0f - p) * relL * kInvLn2 + kLg2Abs + kU * fabsf(l2);
        lsum += fabsf(l2);
    }
    if (f == -INFINITY) return make_float2(f, 0.0f);   // an aggregate is exactly 0
    E += 2.0f * kU * (fabsf(f) + lsum);                 // combine rounding, float p
    return make_float2(f, kSafety * E);
}

// Aggregates of an FP32 slot: (sum A, sum L2) for the DDF, one aggregate
// otherwise (sum A for BVDF, sum L for the VMF).
__device__ __forceinline__ float slot_a(const float2 &v) { return v.x; }
__device__ __forceinline__ float slot_l(const float2 &v) { return v.y; }
__device__ __forceinline__ float slot_a(float v) { return v; }
__device__ __forceinline__ float slot_l(float) { return 0.0f; }

// ---------------------------------------------------------- the kernel ----

template <class C>
__device__ __forceinline__ typename C::Pix load_pixel(const TileParams &prm, int b, int gy, int gx)
{
    gy = min(max(gy, 0), prm.M - 1);
    gx = min(max(gx, 0), prm.N - 1);
    if constexpr (C::F32IN) {
        const size_t plane = (size_t)prm.M * prm.N;
        const float *base = (const float *)prm.img + (size_t)b * 3 * plane + (size_t)gy * prm.N + gx;
        return make_float4(base[0], base[plane], base[2 * plane], 0.0f);
    } else {
        const uint8_t *px = (const uint8_t *)prm.img + 3 * ((size_t)gy * prm.N + gx);
        const int x = px[0], y = px[1], z = px[2];
        if constexpr (C::FP64) return make_int4(x, y, z, x * x + y * y + z * z);
        else return make_float4((float)x, (float)y, (float)z, (float)(x * x + y * y + z * z));
    }
}

template <class C>
__device__ __forceinline__ typename C::PlaneT pair_term(const typename C::Pix &a, const typename C::Pix &b,
                                                        const Aux &xa, const Aux &xb, int q)
{
    typename C::PlaneT t;
    if constexpr (C::FP64 && C::FILTER == VMF) {
        t = lterm64<C::NORM>(a, b);   // Eq. (1)
    } else if constexpr (C::FP64) {
        double ang, l2 = 0.0;
        if constexpr (C::F32IN) {
            ang = aterm64f(a, b);
            if constexpr (C::FILTER == DDF) l2 = l2term64f(a, b);
        } else {
            ang = aterm64<C::DIST>(a, b, q);
            if constexpr (C::FILTER == DDF) l2 = lterm64<C::NORM>(a, b);
        }
        if constexpr (C::FILTER == DDF) t = make_double2(ang, l2);
        else t = ang;
    } else if constexpr (C::FILTER == VMF) {
        float d = 0.0f;   // <x,y>, exact; order 2 only
        if constexpr (C::NORM == NL2) d = fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x));
        t = lterm32<C::NORM>(a, b, d);
    } else if constexpr (C::F32IN) {
        // float input, exact mode: normalised pixels (see normalize_f32)
        if constexpr (C::FILTER == DDF) t = make_float2(angle32f(a, b), l2term32f(a, b));
        else t = angle32f(a, b);
    } else {
        const PairInts r = pair_ints(a, b);
        float ang;
        if constexpr (C::DIST == EXACT) ang = angle32(r);
        else if constexpr (C::DIST == MINIMAX) ang = minimax32(r, xa, xb, q);
        else ang = chroma32(a, b, xa, xb);
        if constexpr (C::FILTER == DDF) t = make_float2(ang, lterm32<C::NORM>(a, b, r.d));
        else t = ang;
    }
    return t;
}

template <class C>
__device__ __forceinline__ void add_term(typename C::PlaneT &x, const typename C::PlaneT &y)
{
    if constexpr (C::FILTER == DDF && !C::FP64) {
        // FP32 (angular, L2) pair: one packed add, each lane rounded as a
        // scalar add.rn.ftz (the FP32 units are built flush-to-zero), so the
        // sums are bit-identical to two scalar adds in one issue slot
        asm("{\n\t.reg .b64 ra, rb;\n\tmov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %3};\n\t"
            "add.rn.ftz.f32x2 ra, ra, rb;\n\tmov.b64 {%0, %1}, ra;\n\t}"
            : "+f"(x.x), "+f"(x.y)
            : "f"(y.x), "f"(y.y));
    } else if constexpr (C::FILTER == DDF) {
        x.x += y.x;
        x.y += y.y;
    } else {
        x += y;
    }
}

// Add the horizontal window sums of row offset dy (values g[dx + 2R]) into
// the aggregates of every window whose rows contain that offset.
template <class C, int DY>
__device__ __forceinline__ void accumulate_row(const typename C::PlaneT *g, typename C::PlaneT (*acc)[C::W])
{
    constexpr int R = C::R;
    using PT = typename C::PlaneT;
    if constexpr (!C::FP64 && R == 2) {
        // FP32, 5x5: the five window sums share pair sums (18 adds, depth 3)
        PT pr[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            pr[j] = g[j];
            add_term<C>(pr[j], g[j + 1]);
        }
#pragma unroll
        for (int ex = -R; ex <= R; ++ex) {
            const int j = R - ex;   // the window covers g[j .. j + 4]
            PT rs = pr[j];
            add_term<C>(rs, pr[j + 2]);
            add_term<C>(rs, g[j + 4]);
#pragma unroll
            for (int ey = -R; ey <= R; ++ey)
                if (DY >= -R - ey && DY <= R - ey) add_term<C>(acc[ey + R][ex + R], rs);
        }
    } else {
        // left to right (the FP64 recheck reproduces this order)
#pragma unroll
        for (int ex = -R; ex <= R; ++ex) {
            PT rs = g[2 * R + (-R - ex)];
#pragma unroll
            for (int dx = -R - ex + 1; dx <= R - ex; ++dx) add_term<C>(rs, g[2 * R + dx]);
#pragma unroll
            for (int ey = -R; ey <= R; ++ey)
                if (DY >= -R - ey && DY <= R - ey) add_term<C>(acc[ey + R][ex + R], rs);
        }
    }
}

// Terms of slice DYP: this thread's pixel p with partners p + (DYP, dx),
// stored in the planes of the slice's buffer.
template <class C, int DYP>
__device__ __forceinline__ void slice_terms(const typename C::Pix *pix, const Aux *aux, typename C::PlaneT *planes,
                                            int tid, int cy, int cx, const typename C::Pix &self_px,
                                            const Aux &self_aux, int q)
{
    constexpr int R = C::R, PXW = C::PXW, PLW = C::PLW, PLANE = C::PLH * C::PLW;
    const int pc = (cy + 2 * R) * PLW + (cx + 2 * R);
    if (tid < C::NC && cy + DYP < C::CH) {
        constexpr int K0 = (DYP == 0) ? 1 : -2 * R;
        constexpr int NK = (DYP == 0) ? 2 * R : 4 * R + 1;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int dx = K0 + k;
            const int bi = (cy + DYP) * PXW + (cx + 2 * R + dx);
            Aux xb{};
            if constexpr (C::AUX) xb = aux[bi];
            planes[k * PLANE + pc] = pair_term<C>(self_px, pix[bi], self_aux, xb, q);
        }
    }
}

// Accumulation of slice DYP: p's own row (offset +DYP) and the mirrored row
// (offset -DYP, terms written by the pixels above p).
template <class C, int DYP>
__device__ __forceinline__ void slice_acc(const typename C::PlaneT *planes, int tid, int cy, int cx,
                                          const typename C::PlaneT &self_term, typename C::PlaneT (*acc)[C::W])
{
    constexpr int R = C::R, PLW = C::PLW, PLANE = C::PLH * C::PLW;
    using PT = typename C::PlaneT;
    const int pc = (cy + 2 * R) * PLW + (cx + 2 * R);
    if (tid < C::NC) {
        PT g[4 * R + 1];
        if constexpr (DYP == 0) {
            g[2 * R] = self_term;
#pragma unroll
            for (int dx = 1; dx <= 2 * R; ++dx) {
                g[2 * R + dx] = planes[(dx - 1) * PLANE + pc];
                g[2 * R - dx] = planes[(dx - 1) * PLANE + pc - dx];
            }
            accumulate_row<C, 0>(g, acc);
        } else {
#pragma unroll
            for (int k = 0; k <= 4 * R; ++k) g[k] = planes[k * PLANE + pc];
            accumulate_row<C, DYP>(g, acc);
#pragma unroll
            for (int k = 0; k <= 4 * R; ++k) {
                const int dx = k - 2 * R;
                g[k] = planes[(2 * R - dx) * PLANE + pc - DYP * PLW + dx];
            }
            accumulate_row<C, -DYP>(g, acc);
        }
    }
}

// One phase of the double-buffered slice pipeline: the terms of slice D+1
// (other buffer) and the accumulation of slice D, then a barrier.
template <class C, int D>
__device__ __forceinline__ void slice_step(const typename C::Pix *pix, const Aux *aux, typename C::PlaneT *buf0,
                                           typename C::PlaneT *buf1, int tid, int cy, int cx,
                                           const typename C::Pix &self_px, const Aux &self_aux,
                                           const typename C::PlaneT &self_term, typename C::PlaneT (*acc)[C::W], int q)
{
    if constexpr (D < 2 * C::R)
        slice_terms<C, D + 1>(pix, aux, ((D + 1) & 1) ? buf1 : buf0, tid, cy, cx, self_px, self_aux, q);
    slice_acc<C, D>((D & 1) ? buf1 : buf0, tid, cy, cx, self_term, acc);
    __syncthreads();
}

template <class C, int... D>
__device__ __forceinline__ void all_slices(std::integer_sequence<int, D...>, const typename C::Pix *pix,
                                           const Aux *aux, typename C::PlaneT *buf0, typename C::PlaneT *buf1, int tid,
                                           int cy, int cx, const typename C::Pix &self_px, const Aux &self_aux,
                                           const typename C::PlaneT &self_term, typename C::PlaneT (*acc)[C::W],
                                           int q)
{
    slice_terms<C, 0>(pix, aux, buf0, tid, cy, cx, self_px, self_aux, q);
    __syncthreads();
    (slice_step<C, D>(pix, aux, buf0, buf1, tid, cy, cx, self_px, self_aux, self_term, acc, q), ...);
}

// ------------------------------------------------ FP32 slice pipeline ----
// The FP32 path keeps the same slices but not the FP64 summation order (its
// bounds need only the depth of each sum).  A thread keeps the terms of its
// own row offset +D in registers and forms their window sums at once; only
// the mirrored row -D passes through shared memory.  The row window sums H(DY)
// reach the 2R+1 vertical window sums through shared partial sums (vstep32),
// in the arrival order +1, 0, +2, -1, ..., +2R, -(2R-1), -2R.  Depth of an
// aggregate: R = 2: 4 (row) + 4 (vertical); R = 1: 2 + 2; 4R either way.

template <class C>
__device__ __forceinline__ typename C::PlaneT psum(typename C::PlaneT a, const typename C::PlaneT &b)
{
    add_term<C>(a, b);
    return a;
}

// Window sums of one row offset: h[ex + R] = sum of g[2R + dx], dx = -R-ex .. R-ex.
// Every window contains the middle value g[2R]; each sum is a suffix sum of
// the values left of it plus a prefix sum of the middle value and the values
// right of it (R = 2: 11 adds instead of 18, depth 4; R = 1: 5 adds, depth 2).
template <class C>
__device__ __forceinline__ void hsum32(const typename C::PlaneT *g, typename C::PlaneT *h)
{
    using PT = typename C::PlaneT;
    if constexpr (C::R == 2) {
        const PT l2 = psum<C>(g[2], g[3]), l1 = psum<C>(g[1], l2), l0 = psum<C>(g[0], l1);
        const PT g5 = psum<C>(g[4], g[5]), g6 = psum<C>(g5, g[6]), g7 = psum<C>(g6, g[7]);
        h[0] = psum<C>(g7, g[8]);   // g4 .. g8
        h[1] = psum<C>(g[3], g7);   // g3 .. g7
        h[2] = psum<C>(l2, g6);     // g2 .. g6
        h[3] = psum<C>(l1, g5);     // g1 .. g5
        h[4] = psum<C>(l0, g[4]);   // g0 .. g4
    } else {
        const PT g3 = psum<C>(g[2], g[3]);
        h[0] = psum<C>(g3, g[4]);                  // g2 .. g4
        h[1] = psum<C>(g[1], g3);                  // g1 .. g3
        h[2] = psum<C>(psum<C>(g[0], g[1]), g[2]); // g0 .. g2
    }
}

// Row offset DY arrives with its window sums h[ex]: update the partial sums
// st; emit(ey, ex, A) receives each aggregate A = sum of H(ey + j), |j| <= R,
// as soon as it is complete.
template <class C, int DY, class Emit>
__device__ __forceinline__ void vstep32(typename C::PlaneT (*st)[C::W], const typename C::PlaneT *h, Emit &emit)
{
#pragma unroll
    for (int x = 0; x < C::W; ++x) {
        const int ex = x - C::R;
        if constexpr (C::R == 1) {
            // st0 = H0+H1, st1 = H0 (+H-1)
            if constexpr (DY == 1) st[0][x] = h[x];
            else if constexpr (DY == 0) {
                st[1][x] = h[x];
                st[0][x] = psum<C>(st[0][x], h[x]);
            } else if constexpr (DY == 2) emit(-1, ex, psum<C>(st[0][x], h[x]));
            else if constexpr (DY == -1) {
                emit(0, ex, psum<C>(st[0][x], h[x]));
                st[1][x] = psum<C>(st[1][x], h[x]);
            } else emit(1, ex, psum<C>(st[1][x], h[x]));
        } else {
            // st0 = H0+H1 (+H-1 +H-2), st1 = H0 (+H-1 +H-2 +H-3),
            // st2 = H0+H1+H2 (+H3), st3 = H-1+H0+H1+H2
            if constexpr (DY == 1) st[0][x] = h[x];
            else if constexpr (DY == 0) {
                st[1][x] = h[x];
                st[0][x] = psum<C>(st[0][x], h[x]);
            } else if constexpr (DY == 2) st[2][x] = psum<C>(st[0][x], h[x]);
            else if constexpr (DY == -1) {
                st[3][x] = psum<C>(st[2][x], h[x]);
                st[0][x] = psum<C>(st[0][x], h[x]);
                st[1][x] = psum<C>(st[1][x], h[x]);
            } else if constexpr (DY == 3) {
                emit(-1, ex, psum<C>(st[3][x], h[x]));
                st[2][x] = psum<C>(st[2][x], h[x]);
            } else if constexpr (DY == -2) {
                emit(0, ex, psum<C>(st[3][x], h[x]));
                st[0][x] = psum<C>(st[0][x], h[x]);
                st[1][x] = psum<C>(st[1][x], h[x]);
            } else if constexpr (DY == 4) emit(-2, ex, psum<C>(st[2][x], h[x]));
            else if constexpr (DY == -3) {
                emit(1, ex, psum<C>(st[0][x], h[x]));
                st[1][x] = psum<C>(st[1][x], h[x]);
            } else emit(2, ex, psum<C>(st[1][x], h[x]));
        }
    }
}

// The same for the arrival order of one plane buffer, mirrored row first:
// 0, +1, -1, +2, -2, ..., +2R, -2R.  R = 2: st0 = H0 (+H-1 +H-2 +H-3),
// st1 = H0+H1 (+H2 +H3), st2 = H-1+H0+H1 (+H-2), st3 = H-1+H0+H1+H2; 14 adds
// per column, every aggregate a chain of 2R+1 values (depth 2R).
template <class C, int DY, class Emit>
__device__ __forceinline__ void vstep32_mf(typename C::PlaneT (*st)[C::W], const typename C::PlaneT *h, Emit &emit)
{
    static_assert(C::R == 2, "one plane buffer: 5x5 only");
#pragma unroll
    for (int x = 0; x < C::W; ++x) {
        const int ex = x - C::R;
        if constexpr (DY == 0) st[0][x] = h[x];
        else if constexpr (DY == 1) st[1][x] = psum<C>(st[0][x], h[x]);
        else if constexpr (DY == -1) {
            st[2][x] = psum<C>(st[1][x], h[x]);
            st[0][x] = psum<C>(st[0][x], h[x]);
        } else if constexpr (DY == 2) {
            st[3][x] = psum<C>(st[2][x], h[x]);
            st[1][x] = psum<C>(st[1][x], h[x]);
        } else if constexpr (DY == -2) {
            emit(0, ex, psum<C>(st[3][x], h[x]));
            st[2][x] = psum<C>(st[2][x], h[x]);
            st[0][x] = psum<C>(st[0][x], h[x]);
        } else if constexpr (DY == 3) {
            emit(-1, ex, psum<C>(st[3][x], h[x]));
            st[1][x] = psum<C>(st[1][x], h[x]);
        } else if constexpr (DY == -3) {
            emit(1, ex, psum<C>(st[2][x], h[x]));
            st[0][x] = psum<C>(st[0][x], h[x]);
        } else if constexpr (DY == 4) emit(-2, ex, psum<C>(st[1][x], h[x]));
        else emit(2, ex, psum<C>(st[0][x], h[x]));
    }
}

// One phase of the FP32 pipeline: the terms of slice D+1 (stored, and summed
// for this thread's own row at once), the mirrored row -D of slice D (row 0
// for D = 0), then a barrier.
template <class C, int D, class Emit>
__device__ __forceinline__ void phase32(const typename C::Pix *pix, const Aux *aux, typename C::PlaneT *buf0,
                                        typename C::PlaneT *buf1, int tid, int cy, int cx,
                                        const typename C::Pix &self_px, const Aux &self_aux,
                                        const typename C::PlaneT &self_term, const typename C::PlaneT *g0,
                                        typename C::PlaneT (*st)[C::W], Emit &emit, int q)
{
    constexpr int R = C::R, W = C::W, NC = C::NC, PXW = C::PXW, CW = C::CW;
    using PT = typename C::PlaneT;
    if constexpr (C::PB1) {
        // one plane buffer: the mirrored row -D of slice D first, a barrier,
        // then the terms of slice D+1 into the same buffer
        if (tid < NC) {
            PT g[4 * R + 1], h[W];
            if constexpr (D == 0) {
                g[2 * R] = self_term;
#pragma unroll
                for (int dx = 1; dx <= 2 * R; ++dx) {
                    g[2 * R + dx] = g0[dx - 1];
                    g[2 * R - dx] = buf0[(dx - 1) * NC + tid - dx];
                }
            } else {
#pragma unroll
                for (int k = 0; k <= 4 * R; ++k) {
                    const int dx = k - 2 * R;
                    g[k] = buf0[(2 * R - dx) * NC + tid - D * CW + dx];
                }
            }
            hsum32<C>(g, h);
            vstep32_mf<C, -D>(st, h, emit);
        }
        if constexpr (D < 2 * R) {
            constexpr int DYP = D + 1;
            __syncthreads();   // slice D is read: the buffer takes slice D+1
            if (tid < NC) {
                PT g[4 * R + 1], h[W];
                if (cy + DYP < C::CH) {
#pragma unroll
                    for (int k = 0; k <= 4 * R; ++k) {
                        const int bi = (cy + DYP) * PXW + (cx + k);   // partner p + (DYP, k - 2R)
                        Aux xb{};
                        if constexpr (C::AUX) xb = aux[bi];
                        g[k] = pair_term<C>(self_px, pix[bi], self_aux, xb, q);
                        buf0[k * NC + tid] = g[k];
                    }
                    hsum32<C>(g, h);
                } else {
#pragma unroll
                    for (int x = 0; x < W; ++x) h[x] = PT{};
                }
                vstep32_mf<C, DYP>(st, h, emit);
            }
        }
        __syncthreads();
        return;
    }
    if (tid < NC) {
        if constexpr (D < 2 * R) {
            constexpr int DYP = D + 1;
            PT *pl = (DYP & 1) ? buf1 : buf0;
            PT g[4 * R + 1], h[W];
            if (cy + DYP < C::CH) {
#pragma unroll
                for (int k = 0; k <= 4 * R; ++k) {
                    const int bi = (cy + DYP) * PXW + (cx + k);   // partner p + (DYP, k - 2R)
                    Aux xb{};
                    if constexpr (C::AUX) xb = aux[bi];
                    g[k] = pair_term<C>(self_px, pix[bi], self_aux, xb, q);
                    pl[k * NC + tid] = g[k];
                }
                hsum32<C>(g, h);
            } else {
                // partners below C: only windows outside the tile use this row
#pragma unroll
                for (int x = 0; x < W; ++x) h[x] = PT{};
            }
            vstep32<C, DYP>(st, h, emit);
        }
        const PT *pl = (D & 1) ? buf1 : buf0;
        PT g[4 * R + 1], h[W];
        if constexpr (D == 0) {
            g[2 * R] = self_term;
#pragma unroll
            for (int dx = 1; dx <= 2 * R; ++dx) {
                g[2 * R + dx] = g0[dx - 1];
                g[2 * R - dx] = pl[(dx - 1) * NC + tid - dx];
            }
        } else {
#pragma unroll
            for (int k = 0; k <= 4 * R; ++k) {
                const int dx = k - 2 * R;
                g[k] = pl[(2 * R - dx) * NC + tid - D * CW + dx];
            }
        }
        hsum32<C>(g, h);
        vstep32<C, -D>(st, h, emit);
    }
    __syncthreads();
}

// What an FP32 slot holds: the aggregates, or for score slots the score
// Omega^4 formed from them (the chromaticity terms through Eq. (10) first),
// with the same operations the selection applies to raw aggregates.
template <class C>
__device__ __forceinline__ typename C::HwT slot_value(const typename C::PlaneT &a)
{
    if constexpr (C::SQ >= 0) {
        float sa = a.x;
        if constexpr (C::DIST == RGB) sa = fmaf(kSlope32, sa, (float)C::NW * kOffset32);
        return pow4_product<C::SQ>(sa, a.y);
    } else {
        return a;
    }
}

// The FP32 aggregates of this thread's pixel p, each written to its
// (window, member) slot of hw when final (windows inside the tile and image).
template <class C, int... D>
__device__ __forceinline__ void all_slices32(std::integer_sequence<int, D...>, const TileParams &prm, int x0, int y0,
                                             const typename C::Pix *pix, const Aux *aux, typename C::PlaneT *buf0,
                                             typename C::PlaneT *buf1, typename C::HwT *hw, int tid, int cy, int cx,
                                             const typename C::Pix &self_px, const Aux &self_aux,
                                             const typename C::PlaneT &self_term, int q)
{
    constexpr int R = C::R, NC = C::NC, PXW = C::PXW;
    using PT = typename C::PlaneT;
    // slice 0: partners p + (0, dx), dx = 1 .. 2R
    PT g0[2 * R];
    if (tid < NC) {
#pragma unroll
        for (int dx = 1; dx <= 2 * R; ++dx) {
            const int bi = cy * PXW + (cx + 2 * R + dx);
            Aux xb{};
            if constexpr (C::AUX) xb = aux[bi];
            g0[dx - 1] = pair_term<C>(self_px, pix[bi], self_aux, xb, q);
            buf0[(dx - 1) * NC + tid] = g0[dx - 1];
        }
    }
    __syncthreads();
    // windows q = p - e inside the tile and the image: bit (ey+R) W + (ex+R)
    // of `valid` (rows of W bits where the window row is inside, and the
    // inside columns repeated in every row)
    constexpr int W = C::W;
    constexpr unsigned ROW = (1u << W) - 1u;
    unsigned rows = 0, cols = 0;
#pragma unroll
    for (int e = -R; e <= R; ++e) {
        const int ty = cy - e - R, tx = cx - e - R;
        if (ty >= 0 && ty < C::TH && y0 + ty < prm.M) rows |= ROW << ((e + R) * W);
        if (tx >= 0 && tx < C::TW && x0 + tx < prm.N) cols |= 1u << (e + R);
    }
    unsigned rep = 0;   // the column bits repeated in each row
#pragma unroll
    for (int i = 0; i < W; ++i) rep |= cols << (i * W);
    const unsigned valid = rows & rep;
    auto emit = [&](int ey, int ex, const PT &a) {
        if (valid & (1u << ((ey + R) * W + (ex + R)))) {
            const int slot = ((cy - ey - R) * C::TW + (cx - ex - R)) * C::NW + (ey + R) * C::W + (ex + R);
            hw[slot] = slot_value<C>(a);
        }
    };
    PT st[2 * R][C::W];
    (phase32<C, D>(pix, aux, buf0, buf1, tid, cy, cx, self_px, self_aux, self_term, g0, st, emit, q), ...);
}

// Step 4a of the tile: the score of every (window, member) slot of the tile
// from its raw aggregates, in place, spread over all threads of the block.
template <class C, int NTL>
__device__ __forceinline__ void score_slots(const TileParams &prm, int b, int x0, int y0, int tid,
                                            typename C::HwT *hw)
{
    constexpr int R = C::R, NW = C::NW;
    int quarter = -1;   // FP32 DDF with p = quarter / 4: the score is Omega^4, else log2 Omega
    if constexpr (!C::FP64 && C::FILTER == DDF) {
        const float p4 = 4.0f * (float)prm.p;
        if (p4 == rintf(p4)) quarter = (int)p4;
    }
#pragma unroll 1
    for (int s = tid; s < C::TW * C::TH * NW; s += NTL) {
        const int w = s / NW, k = s - w * NW;
        const int gy = y0 + w / C::TW, gx = x0 + w % C::TW;
        if (gy >= prm.M || gx >= prm.N) continue;
        const size_t lin = (size_t)gy * prm.N + gx;
        if constexpr (C::FP64) {
            double sa, sl = 0.0;
            if constexpr (C::FILTER == DDF) {
                sa = hw[s].x;
                sl = hw[s].y;
            } else {
                sa = hw[s];
            }
            if constexpr (C::FILTER == DDF && C::DIST == RGB)
                sa = __fma_rn(kSlope64, sa, (double)NW * kOffset64);   // Eq. (10) summed over j
            if (prm.agg) {
                // sum_j A, sum_j L (VMF: 0, sum_j L)
                double *ag = prm.agg + (((size_t)b * prm.M * prm.N + lin) * NW + k) * 2;
                ag[0] = C::FILTER == VMF ? 0.0 : sa;
                ag[1] = C::FILTER == VMF ? sa : sl;
            }
            const double sc = score64<C::FILTER>(sa, sl, prm.p);
            if constexpr (C::FILTER == DDF) hw[s].x = sc;
            else hw[s] = sc;
        } else {
            // (diagnostic only: the scores go to dbg_fe, no selection follows)
            float sa = slot_a(hw[s]);
            if constexpr (C::FILTER == DDF && C::DIST == RGB) sa = fmaf(kSlope32, sa, (float)NW * kOffset32);
            const float2 v = score32<R, C::FILTER, C::DIST, false, C::NORM>(sa, slot_l(hw[s]), (float)prm.p, quarter);
            if (prm.dbg_fe) reinterpret_cast<float2 *>(prm.dbg_fe)[lin * NW + k] = v;
        }
    }
}

// Minimum of n values by a pairwise tree (depth log2 n instead of n - 1).
template <int N>
__device__ __forceinline__ float tree_min(const float *g)
{
    float m[N];
#pragma unroll
    for (int k = 0; k < N; ++k) m[k] = g[k];
#pragma unroll
    for (int w = 1; w < N; w *= 2)
#pragma unroll
        for (int k = 0; k + w < N; k += 2 * w) m[k] = fminf(m[k], m[k + w]);
    return m[0];
}

// Bit k set where pred(k), combined by a pairwise tree of ORs.
template <int N, class P>
__device__ __forceinline__ unsigned bit_mask(P pred)
{
    unsigned m[N];
#pragma unroll
    for (int k = 0; k < N; ++k) m[k] = pred(k) ? (1u << k) : 0u;
#pragma unroll
    for (int w = 1; w < N; w *= 2)
#pragma unroll
        for (int k = 0; k + w < N; k += 2 * w) m[k] |= m[k + w];
    return m[0];
}

// The member selected from the near set (the members that can still be
// minimal), FP32 path.  A single near member is the minimum.  Several near
// members that are provably equal (identical vectors; collinear non-zero
// vectors for BVDF, whose scores depend on directions only; or all exact
// zeros) are exact ties: the tie rule picks the centre, else the lowest
// index.  Otherwise the pixel goes to the FP64 recheck list with the member
// mask wide(), and the provisional choice is argmin().
template <class C, class ZeroF, class WideF, class ArgF>
__device__ __forceinline__ int resolve_near(unsigned near, const TileParams &prm, const typename C::Pix *pix,
                                            const unsigned *keys, int b, int ty, int tx, int gy, int gx, ZeroF zero,
                                            WideF wide, ArgF argmin, bool &tied)
{
    constexpr int R = C::R, W = C::W, NW = C::NW, PXW = C::PXW;
    if (near == 0) near = 1u << C::CENTRE;   // not reached: the member attaining the minimum is near
    const int first = __ffs(near) - 1;
    if ((near & (near - 1)) == 0) return first;
    const int base = ty * PXW + tx + 2 * R;   // member 0 of the window
    const unsigned rkey = keys[base + (first / W) * PXW + first % W];
    unsigned same = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) same |= (keys[base + (k / W) * PXW + k % W] == rkey ? 1u : 0u) << k;
    if constexpr (C::F32IN) {
        // float keys are hashes: equal keys are confirmed on the pixel values
        const float4 ref = pix[base + (first / W) * PXW + first % W];
#pragma unroll 1
        for (unsigned m = near & same; m; m &= m - 1) {
            const int k = __ffs(m) - 1;
            const float4 xk = pix[base + (k / W) * PXW + k % W];
            if (!(xk.x == ref.x && xk.y == ref.y && xk.z == ref.z && xk.w == ref.w)) same &= ~(1u << k);
        }
    }
    bool equal = (near & ~same) == 0;
    if constexpr (C::FILTER == BVDF && !C::F32IN) {
        if (!equal) {
            // same direction: integer cross product is 0, both non-zero
            const float4 ref = pix[base + (first / W) * PXW + first % W];
            equal = true;
#pragma unroll 1
            for (unsigned m = near & ~same; m; m &= m - 1) {
                const int k = __ffs(m) - 1;
                const float4 xk = pix[base + (k / W) * PXW + k % W];
                const float c0 = fmaf(xk.y, ref.z, -(xk.z * ref.y));
                const float c1 = fmaf(xk.z, ref.x, -(xk.x * ref.z));
                const float c2 = fmaf(xk.x, ref.y, -(xk.y * ref.x));
                equal = equal && c0 == 0.0f && c1 == 0.0f && c2 == 0.0f && xk.w > 0.0f && ref.w > 0.0f;
            }
        }
    }
    if constexpr (C::EXACT_SCORES) equal = true;   // equal exact scores are ties
    if (!equal) {
        bool all_zero = true;
#pragma unroll
        for (int k = 0; k < NW; ++k)
            if ((near >> k) & 1u) all_zero = all_zero && zero(k);
        equal = all_zero;
    }
    if (equal) {
        tied = true;   // several near members, provably equal: a structural tie
        return ((near >> C::CENTRE) & 1u) ? C::CENTRE : first;
    }
    const unsigned mask = wide();
    const unsigned slot = atomicAdd(prm.recheck_ctr, 1u);
    if (slot < prm.recheck_cap)
        prm.recheck_list[slot] = make_int2(prm.pix_base + ((C::F32IN ? b : 0) * prm.M + gy) * prm.N + gx, (int)mask);
    else atomicOr(prm.recheck_ctr + 1, 1u);
    return argmin();
}

// ------------------------------------------------ ACWDDF (Eq. (9)) -------
// After the DDF's choice sel_ddf (Eq. (3), p = 1/2), the centre-weighted VMF
// at the smoothing levels k = lam .. lam+2: argmin_i sum_j w_j(k) L2(x_i, x_j)
// with w_d = n - 2k + 2, i.e. S_i + (n - 2k + 1) Lc_i from the member's L2
// aggregate S_i and its distance Lc_i to the centre; then the switch: the DDF
// output if sum_k A(y_k, x_d) L2(y_k, x_d) > T, else the centre.
//
// FP64 (the FP64 tile kernel and the recheck, bit for bit): S(k) and Lc(k)
// are the FP64 path's aggregates and terms; every operation is rounded
// explicitly, so both call sites give the same decision.
template <int R, int DIST, class SF, class LF, class PF>
__device__ __forceinline__ int acw_decide64(int sel_ddf, SF S, LF lc, PF px, int lam, double T, int q)
{
    constexpr int W = 2 * R + 1, NW = W * W, CENTRE = (NW - 1) / 2;
    const int4 xd = px(CENTRE);
    double sum = 0.0;
#pragma unroll 1
    for (int lev = 0; lev < 3; ++lev) {
        const double c = (double)(NW - 2 * (lam + lev) + 1);   // w_d - 1
        const int y = select64<VMF, NW>([&](int k) { return __dadd_rn(S(k), __dmul_rn(c, lc(k))); });
        const int4 xy = px(y);
        double a = aterm64<DIST>(xy, xd, q);
        if constexpr (DIST == RGB) a = __dadd_rn(__dmul_rn(kSlope64, a), kOffset64);   // Eq. (10)
        sum = __dadd_rn(sum, __dmul_rn(a, l2term64(xy, xd)));
    }
    return sum > T ? sel_ddf : CENTRE;
}

// FP32: every decision with its certified bound.  Returns the member, or
// sets *unsure (the caller lists the pixel for the FP64 recheck, which then
// decides everything) and returns a provisional member.  f: the window's raw
// slots (sum A, sum L2); P(k): shared-memory index of member k.
template <class C, class PF>
__device__ __forceinline__ int acw_select32(const TileParams &prm, const float4 *pix, const Aux *aux,
                                            const unsigned *keys, const float2 *f, PF P, bool &unsure, bool &tied)
{
    constexpr int R = C::R, W = C::W, NW = C::NW, CENTRE = C::CENTRE, DIST = C::DIST;
    (void)W;
    // members with provably equal scores: identical vectors (equal keys)
    auto resolve = [&](unsigned near, auto argmin) -> int {
        const int first = __ffs(near) - 1;
        if ((near & (near - 1)) == 0) return first;
        const unsigned rkey = keys[P(first)];
        bool same = true;
#pragma unroll
        for (int k = 0; k < NW; ++k)
            if ((near >> k) & 1u) same = same && keys[P(k)] == rkey;
        if (same) {
            tied = true;
            return ((near >> CENTRE) & 1u) ? CENTRE : first;
        }
        unsure = true;
        return argmin();
    };
    // near set of n non-negative scores g with relative bounds E_k = erel g_k:
    // {g - E <= min (g + E)} = {g <= gmin (1 + erel) / (1 - erel)}, the
    // threshold evaluated with five roundings and padded by 1 + 6u (as in
    // select_and_store), so the computed set contains the near set
    auto near_rel = [&](const float *g, float erel) -> unsigned {
        const float thr = tree_min<NW>(g) * ((1.0f + erel) / (1.0f - erel)) * (1.0f + 6.0f * kU);
        return bit_mask<NW>([&](int k) { return g[k] <= thr; });
    };
    auto argmin_of = [&](const float *g) {
        int arg = 0;
        float best = g[0];
#pragma unroll
        for (int k = 1; k < NW; ++k)
            if (g[k] < best) {
                best = g[k];
                arg = k;
            }
        return arg;
    };
    // 1. the DDF, Eq. (3) (p = 1/2: Omega^4 = SA^2 SL^2 with its bound)
    int sel_ddf;
    if constexpr (DIST != MINIMAX) {
        // exact and chromaticity terms: relative bounds (pow4_erel)
        float g[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            float sa = f[k].x;
            if constexpr (DIST == RGB) sa = fmaf(kSlope32, sa, (float)NW * kOffset32);
            g[k] = pow4_product<2>(sa, f[k].y);
        }
        const unsigned near = near_rel(g, pow4_erel<R, DIST>(2));
        bool zeros = true;   // all near scores exactly 0: exact ties
#pragma unroll
        for (int k = 0; k < NW; ++k)
            if ((near >> k) & 1u) zeros = zeros && g[k] == 0.0f;
        if (zeros && near) {
            tied = tied || (near & (near - 1)) != 0;
            sel_ddf = ((near >> CENTRE) & 1u) ? CENTRE : __ffs(near) - 1;
        } else {
            sel_ddf = resolve(near, [&]() { return argmin_of(g); });
        }
    } else {
        float2 v[NW];
        float hi[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            float sa = f[k].x;
            if constexpr (DIST == RGB) sa = fmaf(kSlope32, sa, (float)NW * kOffset32);
            v[k] = score32<R, DDF, DIST>(sa, f[k].y, 0.5f, 2);
            hi[k] = v[k].x + v[k].y;
        }
        const float U = tree_min<NW>(hi);
        const unsigned near = bit_mask<NW>([&](int k) { return v[k].x - v[k].y <= U; });
        bool zeros = true;   // all near scores exactly 0 with a zero bound: exact ties
#pragma unroll
        for (int k = 0; k < NW; ++k)
            if ((near >> k) & 1u) zeros = zeros && v[k].x == 0.0f && v[k].y == 0.0f;
        if (zeros && near) {
            tied = tied || (near & (near - 1)) != 0;
            sel_ddf = ((near >> CENTRE) & 1u) ? CENTRE : __ffs(near) - 1;
        } else {
            sel_ddf = resolve(near, [&]() {
                int arg = 0;
                float best = v[0].x;
#pragma unroll
                for (int k = 1; k < NW; ++k)
                    if (v[k].x < best) {
                        best = v[k].x;
                        arg = k;
                    }
                return arg;
            });
        }
    }
    // 2. the centre-weighted VMF levels and the switching sum
    const float4 xd = pix[P(CENTRE)];
    float lc[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const float4 xk = pix[P(k)];
        lc[k] = l2term32(xk, xd, fmaf(xk.z, xd.z, fmaf(xk.y, xd.y, xk.x * xd.x)));
    }
    // Level k scores sc = S + c Lc, all parts >= 0: S (the L2 aggregate) has
    // relative error <= kS u, c Lc <= 6u (the centre distance; c is exact),
    // the FMA one rounding, so |error| <= (kS S + 6 c Lc + sc) u <=
    // (kS + 2) u sc (kS >= 6, S + c Lc <= sc (1 + u)): a relative bound,
    // doubled like every FP32 bound.
    constexpr float kS = 6.0f + 4.0f * R;   // relative bound of an L2 aggregate (units of u)
    constexpr float kLevelRel = kSafety * (kS + 2.0f) * kU;
    float sum = 0.0f, Es = 0.0f;
#pragma unroll 1
    for (int lev = 0; lev < 3; ++lev) {
        const float c = (float)(NW - 2 * (prm.lam + lev) + 1);
        float sc[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) sc[k] = fmaf(c, lc[k], f[k].y);
        const unsigned near = near_rel(sc, kLevelRel);
        const int y = resolve(near, [&]() { return argmin_of(sc); });
        // A(y, x_d) L2(y, x_d): relative (exact, Eq. (10)) or absolute (Method 1) bounds
        const float4 xy = pix[P(y)];
        const PairInts r = pair_ints(xy, xd);
        float a, relA = 0.0f, absA = 0.0f;
        if constexpr (DIST == EXACT) {
            a = angle32(r);
            relA = kAngleU;
        } else if constexpr (DIST == MINIMAX) {
            a = minimax32(r, aux[P(y)], aux[P(CENTRE)], prm.q);
            absA = 24.0f;
        } else {
            a = fmaf(kSlope32, chroma32(xy, xd, aux[P(y)], aux[P(CENTRE)]), kOffset32);
            relA = 13.0f;
        }
        const float l = l2term32(xy, xd, r.d);
        const float t = a * l;
        sum += t;
        Es += (fabsf(a) * (relA + 7.0f) + absA) * l + 2.0f * fabsf(t);
    }
    const float T = (float)prm.T;
    Es = kSafety * kU * (Es + fabsf(T)) + 2.0f * (float)fabs((double)T - prm.T);
    if (fabsf(sum - T) <= Es) unsure = true;
    return sum > T ? sel_ddf : CENTRE;
}

// Step 4b of the tile, one thread per output pixel: the member selection
// from the window's scores (FP32: computed here, in registers, from the raw
// aggregates) and the stores.
template <class C>
__device__ __forceinline__ void select_and_store(const TileParams &prm, int b, int x0, int y0, int tid,
                                                 const typename C::Pix *pix, const unsigned *keys,
                                                 const typename C::HwT *hw, bool unsafe_tile = false,
                                                 const Aux *aux = nullptr)
{
    constexpr int R = C::R, W = C::W, NW = C::NW, PXW = C::PXW;
    using Pix = typename C::Pix;
    const int ty = tid / C::TW, tx = tid % C::TW;
    const int gy = y0 + ty, gx = x0 + tx;
    if (gy >= prm.M || gx >= prm.N) return;
    const size_t lin = (size_t)gy * prm.N + gx;
    const auto *f = hw + tid * NW;
    int sel;
    bool tied = false;   // FP32: settled by provable equality of the near members
    if constexpr (C::FP64 && C::ACW) {
        // ACWDDF: the DDF's choice, then the centre-weighted VMF levels and the switch
        const int sel_ddf = select64<DDF, NW>([&](int k) { return f[k].x; });
        auto px = [&](int k) { return pix[(ty + k / W) * PXW + (tx + k % W) + 2 * R]; };
        const Pix xd = px(C::CENTRE);
        double lc[NW];
#pragma unroll 1
        for (int k = 0; k < NW; ++k) lc[k] = l2term64(px(k), xd);
        sel = acw_decide64<R, C::DIST>(sel_ddf, [&](int k) { return f[k].y; }, [&](int k) { return lc[k]; }, px,
                                       prm.lam, prm.T, prm.q);
    } else if constexpr (C::FP64) {
        if constexpr (C::FILTER == DDF) sel = select64<C::FILTER, NW>([&](int k) { return f[k].x; });
        else sel = select64<C::FILTER, NW>([&](int k) { return f[k]; });
    } else if constexpr (C::ACW) {
        bool unsure = false;
        sel = acw_select32<C>(prm, pix, aux, keys, f,
                              [&](int k) { return (ty + k / W) * PXW + (tx + k % W) + 2 * R; }, unsure, tied);
        tied = tied && !unsure;
        if (unsure) {
            // the FP64 recheck decides the whole of Eq. (9) (every member)
            constexpr unsigned ALL = (1u << NW) - 1u;
            const unsigned slot = atomicAdd(prm.recheck_ctr, 1u);
            if (slot < prm.recheck_cap) prm.recheck_list[slot] = make_int2(prm.pix_base + gy * prm.N + gx, (int)ALL);
            else atomicOr(prm.recheck_ctr + 1, 1u);
        }
    } else {
        int quarter = -1;
        if constexpr (C::SQ >= 0) {
            quarter = C::SQ;   // score slots: p = SQ / 4 (the launcher's choice)
        } else if constexpr (C::FILTER == DDF) {
            const float p4 = 4.0f * (float)prm.p;
            if (p4 == rintf(p4)) quarter = (int)p4;
        }
        // Float input: the bounds also carry absolute parts (underflow of
        // tiny products, at most 2^-53 in an aggregate), negligible against
        // aggregates >= 2^-23.  A window with a smaller aggregate, or in a
        // tile with an unsafe pixel, is decided by the FP64 recheck over all
        // its members (unless they are all identical).
        constexpr unsigned ALL = (NW == 32) ? 0xffffffffu : ((1u << NW) - 1u);
        bool unsure = false;
        if constexpr (C::F32IN) {
            float am[NW];
#pragma unroll
            for (int k = 0; k < NW; ++k) am[k] = C::FILTER == DDF ? fminf(slot_a(f[k]), slot_l(f[k])) : slot_a(f[k]);
            unsure = unsafe_tile || tree_min<NW>(am) < 0x1p-23f;
        }
        // Relative bounds (BVDF with the exact or chromaticity terms, and DDF
        // with p = quarter / 4 scored by Omega^4): E = g * erel, g >= 0
        bool relative = (C::FILTER == BVDF && C::DIST != MINIMAX) || C::FILTER == VMF;
        if constexpr (C::FILTER == DDF && C::DIST != MINIMAX) relative = quarter >= 0;
        if (relative) {
            float g[NW];
            float erel;
            if constexpr (C::FILTER == VMF) {
#pragma unroll
                for (int k = 0; k < NW; ++k) g[k] = slot_a(f[k]);
                // order 2: the L2 aggregate's bound; orders 1, infinity: exact
                erel = C::NORM == NL2 ? kSafety * (6.0f + 4.0f * R) * kU : 0.0f;
            } else if constexpr (C::FILTER == BVDF) {
#pragma unroll
                for (int k = 0; k < NW; ++k) g[k] = slot_a(f[k]);
                erel = kSafety * ((C::DIST == RGB ? 11.0f : (C::F32IN ? kAngleFU : kAngleU)) + 4.0f * R) * kU;
            } else {
                // the uniform switch keeps each unrolled loop branch-free
                erel = pow4_erel<R, C::DIST, C::F32IN>(quarter);
                auto fill = [&](auto a) {
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        float sa = slot_a(f[k]);   // >= 0 in these modes (sums of non-negative terms)
                        if constexpr (C::DIST == RGB) sa = fmaf(kSlope32, sa, (float)NW * kOffset32);
                        g[k] = pow4_product<decltype(a)::value>(sa, slot_l(f[k]));
                    }
                };
                if constexpr (C::SQ >= 0) {
#pragma unroll
                    for (int k = 0; k < NW; ++k) g[k] = f[k];   // Omega^4, formed at emission
                } else {
                    switch (quarter) {
                    case 0: fill(std::integral_constant<int, 0>{}); break;
                    case 1: fill(std::integral_constant<int, 1>{}); break;
                    case 2: fill(std::integral_constant<int, 2>{}); break;
                    case 3: fill(std::integral_constant<int, 3>{}); break;
                    default: fill(std::integral_constant<int, 4>{}); break;
                    }
                }
            }
            // The near set {g - E <= min (g + E)} is {g <= gmin (1 + erel) / (1 - erel)}.
            // The threshold is evaluated with five roundings (each <= u
            // relative) and padded by 1 + 6u, so the set computed here
            // contains the near set.
            const float gmin = tree_min<NW>(g);
            const float up = 1.0f + 6.0f * kU;
            const float thr = gmin * ((1.0f + erel) / (1.0f - erel)) * up;
            const unsigned near = unsure ? ALL : bit_mask<NW>([&](int k) { return g[k] <= thr; });
            sel = resolve_near<C>(
                near, prm, pix, keys, b, ty, tx, gy, gx, [&](int k) { return !C::F32IN && g[k] == 0.0f; },
                [&]() {
                    // widened by 100x the FP64 tie tolerance (1e-11: relative
                    // with floor 1e-3 for BVDF; in the log domain for DDF, a
                    // relative 4e-11 on Omega^4)
                    const float U = gmin * (1.0f + erel);
                    const float delta = (C::FILTER != DDF) ? 1e-9f * fmaxf(U, 1e-3f) + 1e-12f : 4e-9f * U;
                    const float thw = (U + delta) / (1.0f - erel) * up;
                    return unsure ? ALL : bit_mask<NW>([&](int k) { return g[k] <= thw; });
                },
                [&]() {
                    // provisional choice (the recheck replaces it); the running
                    // minimum keeps the scores in registers (no dynamic index)
                    int arg = 0;
                    float best = g[0];
#pragma unroll
                    for (int k = 1; k < NW; ++k)
                        if (g[k] < best) {
                            best = g[k];
                            arg = k;
                        }
                    return arg;
                },
                tied);
        } else {
            // general bounds (Method 1, and DDF with p not a multiple of 1/4):
            // the n scores (f, E) of the window, in registers
            float2 v[NW];
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                float sa = slot_a(f[k]);
                if constexpr (C::FILTER == DDF && C::DIST == RGB) sa = fmaf(kSlope32, sa, (float)NW * kOffset32);
                v[k] = score32<R, C::FILTER, C::DIST, C::F32IN, C::NORM>(sa, slot_l(f[k]), (float)prm.p, quarter);
            }
            // U = min (f + E); the near set {f - E <= U} holds every true minimiser
            float hi[NW];
#pragma unroll
            for (int k = 0; k < NW; ++k) hi[k] = v[k].x + v[k].y;
            const float U = tree_min<NW>(hi);
            const unsigned near = unsure ? ALL : bit_mask<NW>([&](int k) { return v[k].x - v[k].y <= U; });
            sel = resolve_near<C>(
                near, prm, pix, keys, b, ty, tx, gy, gx,
                [&](int k) {
                    // exact zeros: f == 0 (or -inf) with a zero bound (integer input only)
                    return !C::F32IN && (v[k].y == 0.0f) &&
                           ((C::FILTER == DDF && (v[k].x == -INFINITY || v[k].x == 0.0f)) ||
                            (C::FILTER == BVDF && C::DIST != MINIMAX && v[k].x == 0.0f));
                },
                [&]() {
                    // widened by 100x the FP64 tie tolerance (1e-11: relative for
                    // BVDF, natural-log units for DDF, whose score here is Omega^4
                    // or log2 Omega)
                    const float delta = (C::FILTER != DDF) ? 1e-9f * fmaxf(fabsf(U), 1e-3f) + 1e-12f
                                        : quarter >= 0   ? 4e-9f * fabsf(U)
                                                         : 1e-9f;
                    return unsure ? ALL : bit_mask<NW>([&](int k) { return v[k].x - v[k].y <= U + delta; });
                },
                [&]() {
                    // provisional choice (the recheck replaces it); the running
                    // minimum keeps the scores in registers (no dynamic index)
                    int arg = 0;
                    float best = v[0].x;
#pragma unroll
                    for (int k = 1; k < NW; ++k)
                        if (v[k].x < best) {
                            best = v[k].x;
                            arg = k;
                        }
                    return arg;
                },
                tied);
        }
    }
    if constexpr (!C::FP64) {
        // structural ties of this warp's pixels, one atomic per warp
        const unsigned act = __activemask();
        const unsigned m = __ballot_sync(act, tied);
        if (m && (threadIdx.x & 31) == __ffs(act) - 1) atomicAdd(prm.recheck_ctr + kTieCounter, (unsigned)__popc(m));
    }
    const Pix v = pix[(ty + sel / W) * PXW + (tx + sel % W) + 2 * R];
    if constexpr (C::F32IN) {
        const size_t plane = (size_t)prm.M * prm.N;
        float *o = (float *)prm.out + (size_t)b * 3 * plane + lin;
        // FP32: the pixel is held normalised ({x 2^-k, 2^k}); the product is exact
        const float sc = C::FP64 ? 1.0f : v.w;
        o[0] = v.x * sc;
        o[plane] = v.y * sc;
        o[2 * plane] = v.z * sc;
        if (prm.idx) prm.idx[(size_t)b * plane + lin] = (int8_t)sel;
    } else {
        uint8_t *o = (uint8_t *)prm.out + 3 * lin;
        o[0] = (uint8_t)v.x;
        o[1] = (uint8_t)v.y;
        o[2] = (uint8_t)v.z;
        if (prm.idx) prm.idx[lin] = (int8_t)sel;
    }
}

// Step 1 of the tile with top-left output pixel (x0, y0) of image b: the
// pixels of C plus a 2R column margin on each side, edge-replicated, in
// shared memory (then a barrier).  Every load of a thread is issued before
// the first is used (one memory round trip per tile).  Returns, for float
// input in FP32, whether the tile holds a pixel the FP32 bounds do not cover.
template <class C, int NTL>
__device__ __forceinline__ bool tile_load(const TileParams &prm, int b, int x0, int y0, unsigned char *smem)
{
    constexpr int R = C::R, PXW = C::PXW;
    using Pix = typename C::Pix;
    Pix *pix = reinterpret_cast<Pix *>(smem);
    Aux *aux = reinterpret_cast<Aux *>(smem + C::PIX_BYTES);
    unsigned *keys = reinterpret_cast<unsigned *>(smem + C::PIX_BYTES + C::AUX_BYTES);
    const int tid = threadIdx.x;
    bool unsafe = false;
    {
        constexpr int NP = C::CH * PXW, PER = (NP + NTL - 1) / NTL;
        Pix v[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * NTL;
            if (i < NP) v[k] = load_pixel<C>(prm, b, y0 - R + i / PXW, x0 - 3 * R + i % PXW);
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * NTL;
            if (i >= NP) continue;
            if constexpr (!C::FP64 && C::F32IN) {
                // float input: normalised pixel, a hash of its bits as the key
                // (equal keys are confirmed on the values), the unsafe flag
                bool safe;
                pix[i] = normalize_f32(v[k].x, v[k].y, v[k].z, safe);
                keys[i] = (unsigned)__float_as_int(v[k].x) * 0x9E3779B1u ^
                          (unsigned)__float_as_int(v[k].y) * 0x85EBCA77u ^ (unsigned)__float_as_int(v[k].z) * 0xC2B2AE3Du;
                unsafe = unsafe || !safe;
            } else {
                pix[i] = v[k];
                if constexpr (!C::FP64)
                    keys[i] = (unsigned)v[k].x | ((unsigned)v[k].y << 8) | ((unsigned)v[k].z << 16);
                if constexpr (C::AUX) aux[i] = make_aux<C::DIST>(v[k]);
            }
        }
    }
    if constexpr (!C::FP64 && C::F32IN) unsafe = __syncthreads_or(unsafe) != 0;
    else __syncthreads();
    return unsafe;
}

// Steps 2-4 of the tile (its pixels staged by tile_load or convert_tile):
// aggregates, scores, selection and stores.  Called by all NTL >= C::NT
// threads of the block (every barrier is reached by all).
// Step 4b of the tile: the selection, one thread per output pixel.
template <class C>
__device__ __forceinline__ void tile_select(const TileParams &prm, int b, int x0, int y0, unsigned char *smem,
                                            bool unsafe, int tid)
{
    using Pix = typename C::Pix;
    Pix *pix = reinterpret_cast<Pix *>(smem);
    Aux *aux = reinterpret_cast<Aux *>(smem + C::PIX_BYTES);
    unsigned *keys = reinterpret_cast<unsigned *>(smem + C::PIX_BYTES + C::AUX_BYTES);
    typename C::HwT *hw =
        reinterpret_cast<typename C::HwT *>(smem + C::PIX_BYTES + C::AUX_BYTES + C::KEY_BYTES + C::HW_OFFSET);
    bool selects = tid < C::TW * C::TH;
    if constexpr (!C::FP64) selects = selects && !prm.dbg_fe;
    if (selects) select_and_store<C>(prm, b, x0, y0, tid, pix, keys, hw, unsafe, aux);
}

template <class C, int NTL>
__device__ __forceinline__ void tile_rest(const TileParams &prm, int b, int x0, int y0, unsigned char *smem,
                                          bool unsafe)
{
    constexpr int R = C::R, W = C::W, NW = C::NW, CW = C::CW, PXW = C::PXW;
    using PT = typename C::PlaneT;
    using Pix = typename C::Pix;
    Pix *pix = reinterpret_cast<Pix *>(smem);
    Aux *aux = reinterpret_cast<Aux *>(smem + C::PIX_BYTES);
    unsigned *keys = reinterpret_cast<unsigned *>(smem + C::PIX_BYTES + C::AUX_BYTES);
    PT *planes = reinterpret_cast<PT *>(smem + C::PIX_BYTES + C::AUX_BYTES + C::KEY_BYTES);
    typename C::HwT *hw =
        reinterpret_cast<typename C::HwT *>(smem + C::PIX_BYTES + C::AUX_BYTES + C::KEY_BYTES + C::HW_OFFSET);
    const int tid = threadIdx.x;

    // 2. aggregates of the n windows containing this thread's pixel
    const int cy = tid / CW, cx = tid % CW;
    const int own = cy * PXW + cx + 2 * R;
    Pix self_px{};
    Aux self_aux{};
    PT self_term{};
    if (tid < C::NC) {
        self_px = pix[own];
        if constexpr (C::AUX) self_aux = aux[own];
        self_term = pair_term<C>(self_px, self_px, self_aux, self_aux, prm.q);
    }
    if constexpr (!C::FP64) {
        // FP32: each slot is written inside the pipeline once its aggregate is final
        all_slices32<C>(std::make_integer_sequence<int, 2 * R + 1>{}, prm, x0, y0, pix, aux, planes,
                        C::PB1 ? planes : planes + C::PBUF, hw, tid, cy, cx, self_px, self_aux, self_term, prm.q);
    } else {
        PT acc[W][W];
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int j = 0; j < W; ++j) acc[i][j] = PT{};
        all_slices<C>(std::make_integer_sequence<int, 2 * R + 1>{}, pix, aux, planes, planes + C::PBUF, tid, cy, cx,
                      self_px, self_aux, self_term, acc, prm.q);

        // 3. raw aggregates, scattered to the windows of the tile
        if (tid < C::NC) {
            // windows q = p - e inside the tile and the image, as bit masks over ey and ex
            unsigned vy = 0, vx = 0;
#pragma unroll
            for (int e = -R; e <= R; ++e) {
                const int ty = cy - e - R, tx = cx - e - R;
                if (ty >= 0 && ty < C::TH && y0 + ty < prm.M) vy |= 1u << (e + R);
                if (tx >= 0 && tx < C::TW && x0 + tx < prm.N) vx |= 1u << (e + R);
            }
#pragma unroll
            for (int ey = -R; ey <= R; ++ey)
#pragma unroll
                for (int ex = -R; ex <= R; ++ex) {
                    if (!((vy >> (ey + R)) & (vx >> (ex + R)) & 1u)) continue;
                    const int slot = ((cy - ey - R) * C::TW + (cx - ex - R)) * NW + (ey + R) * W + (ex + R);
                    hw[slot] = acc[ey + R][ex + R];
                }
        }
        __syncthreads();
    }

    // 4. FP64 (and the FP32 diagnostic): scores of all slots (all threads);
    //    then the selection, one thread per output pixel (the FP32 selection
    //    scores its own window in registers)
    bool score_all = C::FP64;
    if constexpr (!C::FP64 && C::SQ < 0) score_all = prm.dbg_fe != nullptr;   // (never launched with score slots)
    if (score_all) {
        score_slots<C, NTL>(prm, b, x0, y0, tid, hw);
        __syncthreads();
    }
    tile_select<C>(prm, b, x0, y0, smem, unsafe, tid);
}

// Filters the tile with top-left output pixel (x0, y0) of image b.  Called
// by all NTL >= C::NT threads of the block (every barrier is reached by all).
template <class C, int NTL>
__device__ __forceinline__ void tile_body(const TileParams &prm, int b, int x0, int y0, unsigned char *smem)
{
    const bool unsafe = tile_load<C, NTL>(prm, b, x0, y0, smem);
    tile_rest<C, NTL>(prm, b, x0, y0, smem, unsafe);
}

template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB) tile_kernel(const TileParams prm)
{
    extern __shared__ __align__(16) unsigned char smem[];
    tile_body<C, C::NT>(prm, blockIdx.z, blockIdx.x * C::TW, blockIdx.y * C::TH, smem);
}

template <class C>
cudaError_t launch_tile(const TileParams &prm, cudaStream_t st)
{
    // set once per instantiation and device
    static std::atomic<bool> configured[kMaxDevices];
    cudaError_t e = once_per_device(configured, [] {
        return cudaFuncSetAttribute(tile_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (e != cudaSuccess) return e;
    dim3 grid((prm.N + C::TW - 1) / C::TW, (prm.M + C::TH - 1) / C::TH, prm.B);
    tile_kernel<C><<<grid, C::NT, C::SMEM, st>>>(prm);
    return cudaGetLastError();
}

// ------------------------------------------------- FP64 recheck (one warp
// per listed pixel): recomputes, for the members in the pixel's mask, the
// window scores with the FP64 tile kernel's term function and summation
// order, so the result equals the FP64 path bit for bit.  Members outside the
// mask are certified (by the FP32 bounds) to exceed the minimum by more than
// the FP64 tie tolerance; they cannot be selected or tie, and are given +inf.

struct RecheckParams {
    const void *img;   // uint8 HWC, or float32 B x 3 x M x N
    void *out;
    int8_t *idx;
    const int2 *list;
    const unsigned *ctr;
    unsigned cap;
    int M, N;
    double p;
    int q;
    int lam;           // ACWDDF only
    double T;
};

// Warps per recheck block (one listed pixel per warp at a time).
constexpr int kRecheckWarps = 1;

template <int R, int FILTER, int DIST>
struct RecheckCfg {
    // (the per-warp region also holds n doubles of L2 aggregates for ACWDDF)
    // one warp per block: consecutive list entries go to different SMs, whose
    // FP64 pipes (1/64 of the FP32 rate) bound the recheck
    static constexpr int W = 2 * R + 1, NW = W * W, WARPS = kRecheckWarps;
    static constexpr int MATS = (FILTER == DDF) ? 2 : 1;
    // per warp: int4 members first (16-byte aligned), then doubles; the size
    // is a multiple of 16 so every warp's region stays 16-byte aligned
    static constexpr size_t PER_WARP = (sizeof(int4) * NW + sizeof(double) * (MATS * NW * NW + 2 * NW) + 15) / 16 * 16;
    static constexpr size_t SMEM = PER_WARP * WARPS;
};

// Member mask of a window: 32 bits up to 5x5, 64 bits for 7x7.
template <int NW>
using MemberMask = typename std::conditional<(NW > 32), unsigned long long, unsigned>::type;

template <int NW>
__device__ __forceinline__ int mask_ffs(MemberMask<NW> m)
{
    if constexpr (NW > 32) return __ffsll((long long)m);
    else return __ffs(m);
}

template <int NW>
__device__ __forceinline__ int mask_popc(MemberMask<NW> m)
{
    if constexpr (NW > 32) return __popcll(m);
    else return __popc(m);
}

// Recheck of one listed pixel by one warp.  `base` is the warp's shared
// memory (RecheckCfg::PER_WARP bytes, 16-byte aligned).
// F32IN: img and out are float32 B x 3 x M x N and lin = (b M + y) N + x.
// With every member in the mask this is the whole FP64 computation of the
// pixel (the FP64 path of the 7x7 window); agg, when given, receives the
// members' aggregates as the FP64 tile kernel writes them.
template <int R, int FILTER, int DIST, bool F32IN = false, int NORM = NL2, bool ACW = false>
__device__ __forceinline__ void recheck_pixel(const void *img, int M, int N, int lin,
                                              MemberMask<(2 * R + 1) * (2 * R + 1)> mask, void *out, int8_t *idx,
                                              double p, int q, unsigned char *base, int lane, int lam = 0,
                                              double T = 0.0, double *agg = nullptr)
{
    using C = RecheckCfg<R, FILTER, DIST>;
    using PixT = typename std::conditional<F32IN, float4, int4>::type;
    constexpr int W = C::W, NW = C::NW;
    using MaskT = MemberMask<NW>;
    static_assert(!ACW || NW <= 32, "ACWDDF: windows up to 5x5");
    PixT *px = reinterpret_cast<PixT *>(base);
    double *Ma = reinterpret_cast<double *>(base + sizeof(int4) * NW);
    double *Ml = Ma + NW * NW;
    double *fs = Ma + C::MATS * NW * NW;
    const size_t plane = (size_t)M * N;
    const int b = F32IN ? (int)(lin / plane) : 0;
    const int pl = lin - (int)(b * plane);
    const int gy = pl / N, gx = pl % N;
    for (int k = lane; k < NW; k += 32) {
        const int yy = min(max(gy + k / W - R, 0), M - 1);
        const int xx = min(max(gx + k % W - R, 0), N - 1);
        if constexpr (F32IN) {
            const float *s = (const float *)img + (size_t)b * 3 * plane + (size_t)yy * N + xx;
            px[k] = make_float4(s[0], s[plane], s[2 * plane], 0.0f);
        } else {
            const uint8_t *s = (const uint8_t *)img + 3 * ((size_t)yy * N + xx);
            const int x = s[0], y = s[1], z = s[2];
            px[k] = make_int4(x, y, z, x * x + y * y + z * z);
        }
    }
    __syncwarp();
    // rows of the masked members: terms (i, j) for i in mask, all j.  The
    // term functions are symmetric bit for bit, so a pair of two members is
    // computed once (in the row of the lower one) and stored in both rows:
    // the r-th lowest member's row holds every j except the r members below
    // it, NW - r work items.
    constexpr MaskT ALL = (NW == 8 * (int)sizeof(MaskT)) ? ~MaskT(0) : ((MaskT(1) << NW) - 1);
    const int cnt = mask_popc<NW>(mask);
    const int items = cnt * NW - cnt * (cnt - 1) / 2;
    for (int t = lane; t < items; t += 32) {
        int r = 0, start = 0;
        while (start + (NW - r) <= t) {
            start += NW - r;
            ++r;
        }
        MaskT mm = mask;
        for (int s = 0; s < r; ++s) mm &= mm - 1;   // drop the r lowest members
        const int i = mask_ffs<NW>(mm) - 1;
        MaskT row = ALL & ~(mask & ((MaskT(1) << i) - 1));
        for (int s = start; s < t; ++s) row &= row - 1;
        const int j = mask_ffs<NW>(row) - 1;
        double a, l = 0.0;   // VMF: a holds the distance term
        if constexpr (F32IN) {
            a = aterm64f(px[i], px[j]);
            if constexpr (FILTER == DDF) l = l2term64f(px[i], px[j]);
        } else if constexpr (FILTER == VMF) {
            a = lterm64<NORM>(px[i], px[j]);
        } else {
            a = aterm64<DIST>(px[i], px[j], q);
            if constexpr (FILTER == DDF) l = lterm64<NORM>(px[i], px[j]);
        }
        Ma[i * NW + j] = a;
        if constexpr (FILTER == DDF) Ml[i * NW + j] = l;
        if (j != i && ((mask >> j) & 1u)) {
            Ma[j * NW + i] = a;
            if constexpr (FILTER == DDF) Ml[j * NW + i] = l;
        }
    }
    __syncwarp();
    for (int m = lane; m < NW; m += 32) {
        double f = INFINITY;
        if ((mask >> m) & 1u) {
            const int ey = m / W - R;   // window offset (ey, ex), ex = m % W - R
            double sa = 0.0, sl = 0.0;
            // dy order 0, +1, -1, +2, -2, ... restricted to the window's rows
            for (int s = 0; s <= 4 * R; ++s) {
                const int dy = (s == 0) ? 0 : ((s & 1) ? (s + 1) / 2 : -(s / 2));
                if (dy < -R - ey || dy > R - ey) continue;
                // the row sum covers the window's full row (dx = -R-ex .. R-ex)
                const int row = (ey + dy + R) * W;
                double ra = Ma[m * NW + row], rl = 0.0;
                if constexpr (FILTER == DDF) rl = Ml[m * NW + row];
                for (int c = 1; c < W; ++c) {
                    ra += Ma[m * NW + row + c];
                    if constexpr (FILTER == DDF) rl += Ml[m * NW + row + c];
                }
                sa += ra;
                sl += rl;
            }
            if constexpr (FILTER == DDF && DIST == RGB) sa = __fma_rn(kSlope64, sa, (double)NW * kOffset64);
            if (agg) {   // sum_j A, sum_j L (VMF: 0, sum_j L)
                double *ag = agg + ((size_t)lin * NW + m) * 2;
                ag[0] = FILTER == VMF ? 0.0 : sa;
                ag[1] = FILTER == VMF ? sa : sl;
            }
            f = score64<FILTER>(sa, sl, p);
            if constexpr (ACW) fs[NW + m] = sl;   // the member's L2 aggregate
        }
        fs[m] = f;
    }
    __syncwarp();
    if (lane == 0) {
        int sel = select64<FILTER, NW>([&](int k) { return fs[k]; });
        if constexpr (ACW)   // every member is in the mask: the whole of Eq. (9), as the FP64 tile kernel
            sel = acw_decide64<R, DIST>(sel, [&](int k) { return fs[NW + k]; },
                                        [&](int k) { return Ml[k * NW + (NW - 1) / 2]; }, [&](int k) { return px[k]; },
                                        lam, T, q);
        const PixT v = px[sel];
        if constexpr (F32IN) {
            float *o = (float *)out + (size_t)b * 3 * plane + pl;
            o[0] = v.x;
            o[plane] = v.y;
            o[2 * plane] = v.z;
        } else {
            uint8_t *o = (uint8_t *)out + 3 * (size_t)lin;
            o[0] = (uint8_t)v.x;
            o[1] = (uint8_t)v.y;
            o[2] = (uint8_t)v.z;
        }
        if (idx) idx[lin] = (int8_t)sel;
    }
    __syncwarp();
}

template <int R, int FILTER, int DIST, bool F32IN, int NORM, bool ACW>
__global__ void __launch_bounds__(32 * kRecheckWarps) recheck_kernel(const RecheckParams prm)
{
    using C = RecheckCfg<R, FILTER, DIST>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *base = smem + wid * C::PER_WARP;
    const unsigned count = min(prm.ctr[0], prm.cap);
    const int nwarps = gridDim.x * C::WARPS;
    for (unsigned it = blockIdx.x * C::WARPS + wid; it < count; it += nwarps) {
        const int2 ent = prm.list[it];
        // 7x7 windows are listed with every member (the mask field holds -1)
        MemberMask<C::NW> mask = (unsigned)ent.y;
        if constexpr (C::NW > 32) mask = (MemberMask<C::NW>(1) << C::NW) - 1;
        recheck_pixel<R, FILTER, DIST, F32IN, NORM, ACW>(prm.img, prm.M, prm.N, ent.x, mask, prm.out, prm.idx, prm.p,
                                                         prm.q, base, lane, prm.lam, prm.T);
    }
}

template <int R, int FILTER, int DIST, bool F32IN = false, int NORM = NL2, bool ACW = false>
cudaError_t launch_recheck(const RecheckParams &prm, int blocks, cudaStream_t st)
{
    using C = RecheckCfg<R, FILTER, DIST>;
    static std::atomic<bool> configured[kMaxDevices];
    cudaError_t e = once_per_device(configured, [] {
        return cudaFuncSetAttribute(recheck_kernel<R, FILTER, DIST, F32IN, NORM, ACW>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (e != cudaSuccess) return e;
    recheck_kernel<R, FILTER, DIST, F32IN, NORM, ACW><<<blocks, 32 * C::WARPS, C::SMEM, st>>>(prm);
    return cudaGetLastError();
}

}  // namespace vdf
