// vdf_internal.cuh -- pair terms, constants and selection rules shared by the
// CUDA kernels of libvdf (not part of the public ABI).
//
// Paper: M. E. Celebi, "Real-time implementation of order-statistics based
// directional filters".  Section II defines the filters (Eqs. (1)-(3)),
// Section 2.1 Method 1 (Eqs. (4)-(6), Table 1), Section 2.2 Method 2
// (Eq. (7)); Section 3.2 gives the linear map of Eq. (10).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

namespace vdf {

// ------------------------------------------------- per-device set-up ----
// Kernel attributes (the shared-memory opt-in) and device properties belong
// to one device's context, so one-time set-up is tracked per device.
constexpr int kMaxDevices = 64;

// The current device, or -1 (no device, or an ordinal beyond kMaxDevices).
inline int current_device()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    return dev;
}

// Runs set() once per device (again after a failure); `done` is a
// zero-initialised static array.  Concurrent first calls may both run set(),
// which must therefore be idempotent.
template <class F>
inline cudaError_t once_per_device(std::atomic<bool> (&done)[kMaxDevices], F set)
{
    const int dev = current_device();
    if (dev < 0) return cudaErrorInvalidDevice;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    const cudaError_t e = set();
    if (e == cudaSuccess) done[dev].store(true, std::memory_order_release);
    return e;
}

enum Filter { BVDF = 0, DDF = 1, VMF = 2 };
// Minkowski order of the distance term of Eq. (1) (DDF, VMF): 2, 1, or the
// limit of infinite order (the largest component difference).
enum Norm { NL2 = 0, NL1 = 1, NLINF = 2 };
enum Dist { EXACT = 0, MINIMAX = 1, RGB = 2 };

// ------------------------------------------------------------- constants --

// Counter block at the start of every FP32 workspace (256 bytes, 64 words):
// word 0 = pixels listed for the FP64 recheck, word 1 = list overflow flag,
// word kTieCounter = pixels whose near-minimal members the FP32 path proved
// equal (structural ties, settled by the tie rule without a recheck).  The
// batch path keeps its per-group work counters in words 2 .. 2 + groups.
constexpr int kTieCounter = 63;
constexpr size_t kCounterBlockBytes = 256;

// Table 1, Section 2.1: minimax coefficients a_0..a_q for q = 2, 3, 4, padded
// with zeros to degree 4 (a zero leading coefficient leaves Horner's rule
// bit-identical).  ASIN rows are polynomials in tau = sqrt(1 - z) used for
// z >= 1/2 (Eq. (6)); ACOS rows are polynomials in z used for z < 1/2.
static __constant__ double kAsin64[3][5] = {
    {1.829125e-03, 1.371117, 1.480266e-01, 0.0, 0.0},
    {-1.358425e-04, 1.419488, -3.090315e-02, 1.666491e-01, 0.0},
    {2.097797e-05, 1.412840, 1.429881e-02, 6.704361e-02, 6.909677e-02},
};
static __constant__ double kAcos64[3][5] = {
    {1.569882, -9.695260e-01, -1.480266e-01, 0.0, 0.0},
    {1.570864, -1.003730, 3.090318e-02, -2.356775e-01, 0.0},
    {1.570786, -9.990285e-01, -1.429899e-02, -9.481335e-02, -1.381942e-01},
};
static __constant__ float kAsin32[3][5] = {
    {1.829125e-03f, 1.371117f, 1.480266e-01f, 0.0f, 0.0f},
    {-1.358425e-04f, 1.419488f, -3.090315e-02f, 1.666491e-01f, 0.0f},
    {2.097797e-05f, 1.412840f, 1.429881e-02f, 6.704361e-02f, 6.909677e-02f},
};
static __constant__ float kAcos32[3][5] = {
    {1.569882f, -9.695260e-01f, -1.480266e-01f, 0.0f, 0.0f},
    {1.570864f, -1.003730f, 3.090318e-02f, -2.356775e-01f, 0.0f},
    {1.570786f, -9.990285e-01f, -1.429899e-02f, -9.481335e-02f, -1.381942e-01f},
};

// Eq. (10): A ~ 1.436437 B + 0.027664.
constexpr double kSlope64 = 1.436437;
constexpr double kOffset64 = 0.027664;
constexpr float kSlope32 = 1.436437f;
constexpr float kOffset32 = 0.027664f;

constexpr double kHalfPi64 = 1.5707963267948966;   // nearest double to pi/2
constexpr float kHalfPi32 = 1.57079637f;           // nearest float to pi/2

// atan(t) = t * Q(t^2) on [0, 1], Q of degree 6: minimax fit for relative
// error (script gen_atan_poly.py next to this file); float32 Horner
// evaluation error is below 12.8 ulp of the result over the whole range.
// Coefficient k as a constant expression (immediate operands, nothing
// loaded from memory).
constexpr int kAtanDeg = 6;
__host__ __device__ constexpr float atan_q(int k)
{
    return k == 0   ? 0.99999934f
           : k == 1 ? -0.33326516f
           : k == 2 ? 0.19881482f
           : k == 3 ? -0.13487193f
           : k == 4 ? 0.08387123f
           : k == 5 ? -0.037013046f
                    : 0.007863394f;
}

// Relative bounds of the FP32 angle term in units of u = 2^-24 (before the
// safety factor): integer input (angle32: the reciprocal square root, the
// Lagrange c2, the products and 12.8u of polynomial) and float input
// (angle32f: 8u more for its normalised products).
constexpr float kAngleU = 26.0f, kAngleFU = 34.0f;

// ----------------------------------------------------- FP64 pair terms ----
// Inputs are the integer RGB values of two pixels with n2 = |x|^2 in .w.
// Every integer intermediate is exact; each term is a symmetric function of
// its two arguments, bit for bit.

__device__ __forceinline__ double horner4_64(const double *a, double t)
{
    double v = a[4];
    v = __fma_rn(v, t, a[3]);
    v = __fma_rn(v, t, a[2]);
    v = __fma_rn(v, t, a[1]);
    v = __fma_rn(v, t, a[0]);
    return v;
}

// Angular term of the distance mode (BVDF form; for DDF with Method 2 the
// caller applies Eq. (10) to the aggregate).
template <int DIST>
__device__ __forceinline__ double aterm64(const int4 a, const int4 b, int q)
{
    const int d = a.x * b.x + a.y * b.y + a.z * b.z;
    const long long P = (long long)a.w * (long long)b.w;
    if (DIST == EXACT) {
        // Eq. (2): acos(<x,y>/(|x||y|)) = atan2(|x cross y|, <x,y>) for <x,y> >= 0,
        // with |x cross y|^2 = |x|^2 |y|^2 - <x,y>^2 (Lagrange) exact in int64.
        if (P == 0) return kHalfPi64;
        const long long c2 = P - (long long)d * d;
        return atan2(sqrt((double)c2), (double)d);
    } else if (DIST == MINIMAX) {
        // Eqs. (4)-(6): branch on z >= 1/2, i.e. 4 <x,y>^2 >= |x|^2 |y|^2 (exact).
        if (P != 0 && 4LL * d * d >= P) {
            const long long c2 = P - (long long)d * d;
            const double s = sqrt((double)P);
            // 1 - z = |x cross y|^2 / (s (s + <x,y>)), s = |x||y|
            const double t = sqrt((double)c2 / (s * (s + (double)d)));
            return horner4_64(kAsin64[q - 2], t);
        }
        const double z = (P == 0) ? 0.0 : (double)d / sqrt((double)P);
        return horner4_64(kAcos64[q - 2], z);
    } else {
        // Eq. (7): L2 of the chromaticities, sqrt(sum_k (s_y x_k - s_x y_k)^2) / (s_x s_y).
        const int sa = a.x + a.y + a.z, sb = b.x + b.y + b.z;
        if (sa == 0 || sb == 0) {
            if (sa == 0 && sb == 0) return 0.0;
            return sa == 0 ? sqrt((double)b.w) / (double)sb : sqrt((double)a.w) / (double)sa;
        }
        const long long t0 = (long long)sb * a.x - (long long)sa * b.x;
        const long long t1 = (long long)sb * a.y - (long long)sa * b.y;
        const long long t2 = (long long)sb * a.z - (long long)sa * b.z;
        const long long N = t0 * t0 + t1 * t1 + t2 * t2;
        return sqrt((double)N) / ((double)sa * (double)sb);
    }
}

// Eq. (1) at order 2.
__device__ __forceinline__ double l2term64(const int4 a, const int4 b)
{
    const int d = a.x * b.x + a.y * b.y + a.z * b.z;
    return sqrt((double)(a.w + b.w - 2 * d));
}

// Eq. (1) at order 1 or in the limit of infinite order (the largest
// component difference): exact integers.  Order 2 is l2term64.
template <int NORM>
__device__ __forceinline__ double lterm64(const int4 a, const int4 b)
{
    if constexpr (NORM == NL2) {
        return l2term64(a, b);
    } else {
        const int e0 = abs(a.x - b.x), e1 = abs(a.y - b.y), e2 = abs(a.z - b.z);
        if constexpr (NORM == NL1) return (double)(e0 + e1 + e2);
        else return (double)max(e0, max(e1, e2));
    }
}

// FP64 terms for float32 inputs (exact mode only): products of two float32
// values are exact in double; each cross-product component is rounded once.
__device__ __forceinline__ double aterm64f(const float4 a, const float4 b)
{
    const double ax = a.x, ay = a.y, az = a.z, bx = b.x, by = b.y, bz = b.z;
    const double na = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
    const double nb = __dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz));
    if (na == 0.0 || nb == 0.0) return kHalfPi64;
    const double d = __dadd_rn(__dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)), __dmul_rn(az, bz));
    const double c0 = __fma_rn(ay, bz, -__dmul_rn(az, by));
    const double c1 = __fma_rn(az, bx, -__dmul_rn(ax, bz));
    const double c2 = __fma_rn(ax, by, -__dmul_rn(ay, bx));
    const double cc = __dadd_rn(__dadd_rn(__dmul_rn(c0, c0), __dmul_rn(c1, c1)), __dmul_rn(c2, c2));
    return atan2(sqrt(cc), d);
}

__device__ __forceinline__ double l2term64f(const float4 a, const float4 b)
{
    const double e0 = (double)a.x - (double)b.x, e1 = (double)a.y - (double)b.y, e2 = (double)a.z - (double)b.z;
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2)));
}

// ----------------------------------------------------- FP32 pair terms ----
// Inputs: float4 {x, y, z, |x|^2} of integer-valued pixels (all exact in
// float32), plus per-pixel auxiliaries for Methods 1 and 2.  Each term comes
// with a relative (or, for Method 1, absolute) error bound used by the
// certification in select32(); the bounds are derived in the design notes.

constexpr float kU = 5.9604645e-08f;   // 2^-24

struct Aux {
    float a, b;   // Method 1: |x|, 1/|x| (0 for a zero vector); Method 2: sum x_k, |x|/sum x_k
};

// Per-pixel auxiliary values of the FP32 Method 1 / Method 2 terms; v holds
// the integer RGB values with |x|^2 in .w.
template <int DIST>
__device__ __forceinline__ Aux make_aux(const float4 v)
{
    Aux a;
    if constexpr (DIST == MINIMAX) {
        a.a = sqrtf(v.w);
        a.b = v.w > 0.0f ? 1.0f / a.a : 0.0f;
    } else {
        a.a = v.x + v.y + v.z;
        a.b = a.a > 0.0f ? sqrtf(v.w) / a.a : 0.0f;
    }
    return a;
}

// Integer quantities of a pixel pair.  d = <x,y> is exact (< 2^24).
// D = d^2 is split hi + lo by FMA (Dekker: D = Dh + Dl exactly), and so is
// P = |x|^2 |y|^2 (Ph + Pl; Method 1's branch test uses it).
// c2 = |x x y|^2 = P - D (Lagrange) is fma(|x|^2, |y|^2, -Dh) - Dl: the FMA
// gives the integer P - Dh exactly when it is below 2^24 (then c2 has one
// rounding) and with relative error <= u otherwise, where c2 >= 2^24 - 2^11
// dwarfs |Dl| <= 2^11: relative error <= 2u in every case.
struct PairInts {
    float d, Ph, Pl, Dh, Dl, c2;
};

__device__ __forceinline__ PairInts pair_ints(const float4 a, const float4 b)
{
    PairInts r;
    r.d = fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x));
    r.Ph = a.w * b.w;
    r.Pl = fmaf(a.w, b.w, -r.Ph);
    r.Dh = r.d * r.d;
    r.Dl = fmaf(r.d, r.d, -r.Dh);
    r.c2 = fmaf(a.w, b.w, -r.Dh) - r.Dl;
    return r;
}

// theta = atan2(sqrt(c2), d) from c2 = |x x y|^2 and Dh = d^2 via
// t = min(tan, cot): one reciprocal square root of c2 d^2, whose zero is
// guarded by adding `guard` (below every non-zero c2 d^2 that matters).
__device__ __forceinline__ float angle_core(float c2, float Dh, float guard)
{
    const float m = fmaf(c2, Dh, guard);
    const float rs = rsqrtf(m);
    // t = min(tan, cot) = min(sqrt(c2)/d, d/sqrt(c2)) = min(c2, d^2) / sqrt(c2 d^2)
    const float t = fminf(c2, Dh) * rs;
    const float s = t * t;
    float v = atan_q(kAtanDeg);
#pragma unroll
    for (int k = kAtanDeg - 1; k >= 0; --k) v = fmaf(v, s, atan_q(k));
    const float a = t * v;
    // c2 >= d^2: theta >= 45 deg (also a zero vector: both 0, theta = pi/2)
    return (c2 >= Dh) ? (kHalfPi32 - a) : a;
}

// Eq. (2) angle in FP32: theta = atan2(sqrt(c2), d) via t = min(tan, cot).
// Relative error <= kAngleU u (rsqrt 2 ulp, the Lagrange c2, the polynomial).
__device__ __forceinline__ float angle32(const PairInts &r)
{
    // c2 * d^2 is 0 or >= 1 (integers), so adding 1e-30 only guards the zero
    return angle_core(r.c2, r.Dh, 1e-30f);
}

// |x - y| in FP32.  e = |x - y|^2 is an exact integer in [0, 3 * 255^2]; on
// that domain the approximate square root (one SFU operation) is within 2u
// of the exact value (1.67u at worst; every attainable input is checked on
// the GPU by the test suite through vdf_debug_fp32_terms) and exactly 0 at
// 0.  Bound used: 5u.
__device__ __forceinline__ float l2term32(const float4 a, const float4 b, float d)
{
    const float e = fmaf(-2.0f, d, a.w + b.w);
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e));
    return r;
}

// Eq. (1) in FP32 for integer-valued pixels: order 2 as l2term32 (d = <x,y>),
// orders 1 and infinity exact (integer differences; sums below 2^24).
template <int NORM>
__device__ __forceinline__ float lterm32(const float4 a, const float4 b, float d)
{
    if constexpr (NORM == NL2) {
        return l2term32(a, b, d);
    } else {
        const float e0 = fabsf(a.x - b.x), e1 = fabsf(a.y - b.y), e2 = fabsf(a.z - b.z);
        if constexpr (NORM == NL1) return e0 + e1 + e2;
        else return fmaxf(e0, fmaxf(e1, e2));
    }
}

// ------------------------------------------ FP32 terms, float32 input ----
// A float pixel x >= 0 is held exponent-normalised: {x 2^-k, 2^k} with the
// largest component of x 2^-k in [1, 2) (an exact scaling; a zero vector is
// {0, 1}).  Angles are scale-free, and x = (x 2^-k) 2^k exactly, so the L2
// term reads the original values back.  A pixel is "safe" when every
// component is +0 or a positive normal float whose exponent lies within 60
// of the largest one's, and the largest one's exponent lies in [-60, 60];
// pixels that are not (a negative, infinite, NaN or subnormal component, an
// extreme magnitude or spread) are left to the FP64 recheck.  The
// classification reads the bits, so it does not depend on flush-to-zero.

// Normalised pixel, and whether it is safe.
__device__ __forceinline__ float4 normalize_f32(float x, float y, float z, bool &safe)
{
    const int xb = __float_as_int(x), yb = __float_as_int(y), zb = __float_as_int(z);
    const int ex = (xb >> 23) & 0xff, ey = (yb >> 23) & 0xff, ez = (zb >> 23) & 0xff;
    const int em = max(ex, max(ey, ez));   // biased exponent of the largest component (all >= 0)
    auto ok = [em](int bits, int e) {      // +0, or a positive normal within 60 octaves of the largest
        return bits == 0 || (bits > 0 && e >= 1 && e <= 254 && e >= em - 60);
    };
    safe = ok(xb, ex) && ok(yb, ey) && ok(zb, ez) && (em == 0 || (em >= 127 - 60 && em <= 127 + 60));
    if (!safe || em == 0) return make_float4(0.0f, 0.0f, 0.0f, 1.0f);
    const float down = __int_as_float((254 - em) << 23), up = __int_as_float(em << 23);   // 2^-(em-127), 2^(em-127)
    return make_float4(x * down, y * down, z * down, up);
}

// a b - c d by Kahan's algorithm: relative error <= 2u with FMA (Jeannerod,
// Louvet and Muller, Math. Comp. 82 (2013)), barring underflow.
__device__ __forceinline__ float det2(float a, float b, float c, float d)
{
    const float w = c * d;
    const float e = fmaf(-c, d, w);   // w - c d, exactly
    const float f = fmaf(a, b, -w);
    return f + e;
}

// Eq. (2) angle of two normalised safe pixels.  d (three non-negative
// products, FMA chain): <= 3u; each cross component <= 2u (Kahan), so
// |x x y|^2 <= 6u and d^2 <= 7u; the rest as angle32.  Relative error
// <= kAngleFU u (doubled by the bound's safety factor), plus an absolute 2^-58
// where a tiny product underflows; the guard 2^-120 lies below c2 d^2 except
// for angles within 2^-58 of 0 or pi/2.
__device__ __forceinline__ float angle32f(const float4 a, const float4 b)
{
    const float d = fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x));
    const float c0 = det2(a.y, b.z, a.z, b.y), c1 = det2(a.z, b.x, a.x, b.z), c2 = det2(a.x, b.y, a.y, b.x);
    const float cc = fmaf(c2, c2, fmaf(c1, c1, c0 * c0));
    return angle_core(cc, d * d, 0x1p-120f);
}

// |x - y| of two normalised safe pixels: each difference x_k - y_k of the
// original values (exact products by powers of 2) with one rounding, the sum
// of squares <= 4u, the approximate square root <= 2u (checked over every
// float by the test suite): relative error <= 8u, plus an absolute 2^-62
// where a tiny difference underflows.
__device__ __forceinline__ float l2term32f(const float4 a, const float4 b)
{
    const float e0 = fmaf(a.x, a.w, -(b.x * b.w)), e1 = fmaf(a.y, a.w, -(b.y * b.w)), e2 = fmaf(a.z, a.w, -(b.z * b.w));
    const float e = fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e));
    return r;
}

__device__ __forceinline__ float horner4_32(const float *c, float t)
{
    float v = c[4];
    v = fmaf(v, t, c[3]);
    v = fmaf(v, t, c[2]);
    v = fmaf(v, t, c[1]);
    v = fmaf(v, t, c[0]);
    return v;
}

// Method 1 in FP32.  The branch z >= 1/2 is decided exactly:
// 4<x,y>^2 - |x|^2|y|^2 = (4Dh - Ph) + (4Dl - Pl) keeps its sign.
// Absolute error <= 24u.
__device__ __forceinline__ float minimax32(const PairInts &r, const Aux xa, const Aux xb, int q)
{
    const float v = (4.0f * r.Dh - r.Ph) + (4.0f * r.Dl - r.Pl);
    const bool upper = (v >= 0.0f) && (r.Ph > 0.0f);
    const float c2 = r.c2;
    const float np = xa.a * xb.a;                              // |x||y|
    const float tau = c2 * rsqrtf(fmaxf(c2 * np * (np + r.d), 1e-30f));   // sqrt(1 - z)
    const float z = r.d * xa.b * xb.b;                         // 0 for a zero vector
    return upper ? horner4_32(kAsin32[q - 2], tau) : horner4_32(kAcos32[q - 2], z);
}

// Method 2 in FP32: B = sqrt(N) / (s_x s_y), N from exact integer differences.
// Relative error <= 11u.
__device__ __forceinline__ float chroma32(const float4 a, const float4 b, const Aux xa, const Aux xb)
{
    const float ss = xa.a * xb.a;   // exact (< 2^24)
    const float t0 = fmaf(xb.a, a.x, -(xa.a * b.x));
    const float t1 = fmaf(xb.a, a.y, -(xa.a * b.y));
    const float t2 = fmaf(xb.a, a.z, -(xa.a * b.z));
    const float N = fmaf(t2, t2, fmaf(t1, t1, t0 * t0));
    const float D = ss * ss;
    const float B = N * rsqrtf(fmaxf(N * D, 1e-30f));
    return (ss == 0.0f) ? (xa.b + xb.b) : B;
}

// log2 with exact exponent extraction: |error| <= 2^-22.6 + u |result|.
__device__ __forceinline__ float log2_rr(float x)
{
    if (!(x > 0.0f)) return -INFINITY;
    const int bits = __float_as_int(x);
    const int e = ((bits >> 23) & 0xff) - 127;
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);   // [1, 2)
    return (float)e + __log2f(m);
}

}  // namespace vdf
