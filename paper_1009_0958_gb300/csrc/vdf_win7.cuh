// vdf_win7.cuh -- the 7x7 window (R = 3, n = 49 members): one warp per output
// pixel.
//
// Section II defines the filters for any sqrt(n) x sqrt(n) window.  The tile
// kernel's pair reuse across windows keeps (2R+1)-wide register pipelines per
// candidate, which do not fit at R = 3, so the 7x7 window is computed per
// output pixel: the warp stages the 49 clamped members in shared memory and
// forms every member's aggregate over the window directly.
//
//   FP64 (the plain path): recheck_pixel with every member in the mask: each
//     unordered pair once (the term functions are symmetric bit for bit),
//     row sums left to right, rows in the order dy = 0, +1, -1, ..., then
//     select64.  The FP64 recheck of the FP32 path calls the same function,
//     so both give the same result on every pixel.
//   FP32 (certified): lane t takes (member i, window row r) items and sums
//     the row's seven terms left to right; a member's aggregate adds its
//     seven row sums in order (depth 6 + 6 = 4R, the summation depth the
//     FP32 bounds assume).  Scores and certified bounds come from score32;
//     the near set {f - E <= min(f + E)} is found with warp votes (two 32-bit
//     halves of the 49-member mask).  A single near member is the answer;
//     several provably equal ones (identical vectors, collinear ones for
//     BVDF, exact zeros; equal exact scores of the VMF at orders 1 and
//     infinity) are a structural tie (tie rule); otherwise the pixel is
//     listed for the FP64 recheck with every member.
#pragma once

#include "vdf_tile.cuh"

namespace vdf {

struct Win7Params {
    const uint8_t *img;
    uint8_t *out;
    int8_t *idx;
    int2 *list;        // FP32: {pixel id, -1} entries for the FP64 recheck
    unsigned *ctr;     // the workspace's counter block
    unsigned cap;
    int M, N;
    double p;
    int q;
};

constexpr int kWin7Warps = 4;   // output pixels per block (one per warp)

// FP32 term of a uint8 pair: (angle, distance) for the DDF, the angle for
// BVDF, the distance for the VMF, as the FP32 tile kernel computes them.
template <int FILTER, int DIST, int NORM>
__device__ __forceinline__ float2 win7_term32(const float4 a, const float4 b, const Aux xa, const Aux xb, int q)
{
    if constexpr (FILTER == VMF) {
        float d = 0.0f;   // <x,y>, exact; order 2 only
        if constexpr (NORM == NL2) d = fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x));
        return make_float2(lterm32<NORM>(a, b, d), 0.0f);
    } else {
        const PairInts r = pair_ints(a, b);
        float ang;
        if constexpr (DIST == EXACT) ang = angle32(r);
        else if constexpr (DIST == MINIMAX) ang = minimax32(r, xa, xb, q);
        else ang = chroma32(a, b, xa, xb);
        return make_float2(ang, FILTER == DDF ? lterm32<NORM>(a, b, r.d) : 0.0f);
    }
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int FILTER, int DIST, int NORM>
__global__ void __launch_bounds__(32 * kWin7Warps) win7_fp32_kernel(const Win7Params prm)
{
    constexpr int R = 3, W = 7, NW = 49, CENTRE = 24;
    constexpr bool AUX = DIST != EXACT && FILTER != VMF;
    constexpr bool EXACT_SCORES = FILTER == VMF && NORM != NL2;
    __shared__ float4 spx[kWin7Warps][NW];
    __shared__ Aux saux[kWin7Warps][NW];
    __shared__ unsigned skey[kWin7Warps][NW];
    __shared__ float2 srow[kWin7Warps][NW * W];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *px = spx[warp];
    Aux *aux = saux[warp];
    unsigned *key = skey[warp];
    float2 *rs = srow[warp];
    int quarter = -1;   // DDF with p = quarter / 4: the score is Omega^4, else log2 Omega
    if constexpr (FILTER == DDF) {
        const float p4 = 4.0f * (float)prm.p;
        if (p4 == rintf(p4)) quarter = (int)p4;
    }
    const int total = prm.M * prm.N;
    unsigned ties = 0;   // structural ties of this warp's pixels
    for (int lin = blockIdx.x * kWin7Warps + warp; lin < total; lin += gridDim.x * kWin7Warps) {
        const int gy = lin / prm.N, gx = lin - gy * prm.N;
        for (int k = lane; k < NW; k += 32) {
            const int yy = min(max(gy + k / W - R, 0), prm.M - 1);
            const int xx = min(max(gx + k % W - R, 0), prm.N - 1);
            const uint8_t *s = prm.img + 3 * ((size_t)yy * prm.N + xx);
            const int x = s[0], y = s[1], z = s[2];
            const float4 v = make_float4((float)x, (float)y, (float)z, (float)(x * x + y * y + z * z));
            px[k] = v;
            key[k] = (unsigned)x | ((unsigned)y << 8) | ((unsigned)z << 16);
            if constexpr (AUX) aux[k] = make_aux<DIST>(v);
        }
        __syncwarp();
        // row sums: item t = (member i, window row r), dx left to right
        for (int t = lane; t < NW * W; t += 32) {
            const int i = t / W, r = t - i * W;
            const float4 xi = px[i];
            Aux ai{};
            if constexpr (AUX) ai = aux[i];
            float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int c = 0; c < W; ++c) {
                Aux aj{};
                if constexpr (AUX) aj = aux[r * W + c];
                const float2 v = win7_term32<FILTER, DIST, NORM>(xi, px[r * W + c], ai, aj, prm.q);
                s.x = c == 0 ? v.x : s.x + v.x;
                s.y = c == 0 ? v.y : s.y + v.y;
            }
            rs[t] = s;
        }
        __syncwarp();
        // scores and certified bounds of members lane and lane + 32
        float f[2] = {INFINITY, INFINITY}, E[2] = {0.0f, 0.0f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = lane + 32 * h;
            if (m < NW) {
                float sa = rs[m * W].x, sl = rs[m * W].y;
#pragma unroll
                for (int r = 1; r < W; ++r) {
                    sa += rs[m * W + r].x;
                    sl += rs[m * W + r].y;
                }
                float2 v;
                if constexpr (FILTER == VMF) {
                    v = score32<R, VMF, EXACT, false, NORM>(sa, 0.0f, 0.0f, -1);
                } else {
                    if constexpr (FILTER == DDF && DIST == RGB) sa = fmaf(kSlope32, sa, (float)NW * kOffset32);
                    v = score32<R, FILTER, DIST, false, NORM>(sa, sl, (float)prm.p, quarter);
                }
                f[h] = v.x;
                E[h] = v.y;
            }
        }
        const float U = warp_min(fminf(f[0] + E[0], f[1] + E[1]));
        const bool n0 = f[0] - E[0] <= U, n1 = lane + 32 < NW && f[1] - E[1] <= U;
        const unsigned long long near =
            (unsigned long long)__ballot_sync(0xffffffffu, n0) | ((unsigned long long)__ballot_sync(0xffffffffu, n1) << 32);
        int sel;
        bool tied = false;
        if (near == 0ull) {
            sel = CENTRE;   // not reached: the member attaining U is near
        } else if ((near & (near - 1)) == 0ull) {
            sel = __ffsll((long long)near) - 1;
        } else {
            const int first = __ffsll((long long)near) - 1;
            const unsigned kf = key[first];
            const float4 xf = px[first];
            bool same = true, zero = true;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = lane + 32 * h;
                if (m < NW && ((near >> m) & 1ull)) {
                    bool eq = key[m] == kf;
                    if constexpr (FILTER == BVDF) {
                        // same direction: integer cross product 0, both non-zero
                        const float4 xm = px[m];
                        const float c0 = fmaf(xm.y, xf.z, -(xm.z * xf.y));
                        const float c1 = fmaf(xm.z, xf.x, -(xm.x * xf.z));
                        const float c2 = fmaf(xm.x, xf.y, -(xm.y * xf.x));
                        eq = eq || (c0 == 0.0f && c1 == 0.0f && c2 == 0.0f && xm.w > 0.0f && xf.w > 0.0f);
                    }
                    same = same && eq;
                    // exact zeros: a zero score (-inf in the log form) with a zero bound
                    const bool z = E[h] == 0.0f && (f[h] == 0.0f || (FILTER == DDF && f[h] == -INFINITY)) &&
                                   !(FILTER == BVDF && DIST == MINIMAX);
                    zero = zero && z;
                }
            }
            const bool equal = EXACT_SCORES || __all_sync(0xffffffffu, same) || __all_sync(0xffffffffu, zero);
            if (equal) {
                tied = true;
                sel = ((near >> CENTRE) & 1ull) ? CENTRE : first;
            } else {
                // provisional: the smallest score, lowest index first
                const float fm = warp_min(fminf(f[0], f[1]));
                const unsigned long long at = (unsigned long long)__ballot_sync(0xffffffffu, f[0] == fm) |
                                              ((unsigned long long)__ballot_sync(0xffffffffu, f[1] == fm) << 32);
                sel = at ? __ffsll((long long)at) - 1 : CENTRE;
                if (lane == 0) {
                    const unsigned slot = atomicAdd(prm.ctr, 1u);
                    if (slot < prm.cap) prm.list[slot] = make_int2(lin, -1);
                    else atomicOr(prm.ctr + 1, 1u);
                }
            }
        }
        ties += tied ? 1u : 0u;
        if (lane == 0) {
            const float4 v = px[sel];
            uint8_t *o = prm.out + 3 * (size_t)lin;
            o[0] = (uint8_t)v.x;
            o[1] = (uint8_t)v.y;
            o[2] = (uint8_t)v.z;
            if (prm.idx) prm.idx[lin] = (int8_t)sel;
        }
        __syncwarp();
    }
    if (lane == 0 && ties) atomicAdd(prm.ctr + kTieCounter, ties);
}

// FP64 path of the 7x7 window: every pixel through recheck_pixel with every
// member (one warp per block; the shared memory holds the pair matrix).
template <int FILTER, int DIST, int NORM>
__global__ void __launch_bounds__(32) win7_fp64_kernel(const RecheckParams prm, double *agg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const unsigned long long all = (1ull << 49) - 1;
    const int total = prm.M * prm.N;
    for (int lin = blockIdx.x; lin < total; lin += gridDim.x)
        recheck_pixel<3, FILTER, DIST, false, NORM>(prm.img, prm.M, prm.N, lin, all, prm.out, prm.idx, prm.p, prm.q,
                                                     smem, lane, 0, 0.0, agg);
}

}  // namespace vdf
