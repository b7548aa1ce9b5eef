// vdf_backward.cu -- gradient of the directional filters with respect to the
// input image, as a deterministic gather.
//
// The forward pass copies, for every output pixel p, the input vector of one
// window member: y(p) = x(src(p)) with src(p) = clamp(p + off(idx(p))), where
// off(i) = (i / w - R, i % w - R) is the raster offset of member i and clamp
// replaces out-of-image positions by the nearest edge pixel (Section II; the
// border reading of this library).  Away from ties the selection is locally
// constant, so dy/dx is a 0/1 selection matrix and
//     grad_x(q) = sum over p with src(p) = q of grad_y(p).
// Every p with src(p) = q lies within R pixels of q in both directions
// (including at the borders, where clamping only moves sources inward), so
// each thread gathers over the (2R+1)^2 neighbourhood of its own q in a fixed
// order: no atomics, bit-reproducible.
#include "vdf_dispatch.h"

namespace vdf {

namespace {

// A block gathers a kTX x kTY tile: the gradients and indices of the tile
// and a ring around it are first staged in shared memory (entries outside
// the image get index -1).  Then every staged pixel p within R of the tile
// computes its source q = src(p) and, when q lies in the tile, sets bit
// (p - q + (R, R)) in q's source mask (a shared-memory OR).  Finally each
// thread gathers for kQ pixels of one row: it adds the gradients of the set
// bits, lowest first, i.e. in raster order of p.
//
// Staging: with VEC (N a multiple of 4, 16-byte aligned gradients) rows are
// read as float4 / 32-bit words over columns bx - 4 .. bx + kTX + 3 (every
// vector is inside the image or wholly outside it); otherwise element by
// element over bx - R .. bx + kTX + R - 1.
constexpr int kTX = 128, kTY = 8, kQ = 4;

template <int R, bool VEC>
__global__ void __launch_bounds__(256) backward_gather(const float *__restrict__ gy, const int8_t *__restrict__ idx,
                                                       float *__restrict__ gx, int M, int N)
{
    constexpr int W = 2 * R + 1, HY = kTY + 2 * R;
    constexpr int C0 = VEC ? 4 : R;            // staged column of image column bx
    constexpr int HX = kTX + 2 * C0;
    __shared__ __align__(16) float sg[3][HY][HX];
    __shared__ __align__(16) int8_t si[HY][HX];
    __shared__ unsigned qm[kTY][kTX];   // per pixel of the tile: its sources, bit (dy+R) W + (dx+R)
    const int bx = blockIdx.x * kTX, by = blockIdx.y * kTY, b = blockIdx.z;
    const size_t plane = (size_t)M * N;
    const int8_t *ib = idx + (size_t)b * plane;
    const float *g = gy + (size_t)b * 3 * plane;
    const int tid = threadIdx.x;
    for (int e = tid; e < kTY * kTX; e += 256) (&qm[0][0])[e] = 0u;
    if constexpr (VEC) {
        // HY rows x HX / 4 vectors; each thread issues all its loads first
        constexpr int NV = HY * (HX / 4), PER = (NV + 255) / 256;
        float4 v[3][PER];
        int w[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + 256 * k;
            const int r = e / (HX / 4), c4 = e - r * (HX / 4);
            const int py = by - R + r, px = bx - C0 + 4 * c4;
            const bool in = e < NV && py >= 0 && py < M && px >= 0 && px < N;
            const size_t o = in ? (size_t)py * N + px : 0;
            w[k] = in ? __ldg(reinterpret_cast<const int *>(ib + o)) : -1;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                v[c][k] = in ? __ldg(reinterpret_cast<const float4 *>(g + c * plane + o)) : make_float4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + 256 * k;
            if (e >= NV) continue;
            const int r = e / (HX / 4), c4 = e - r * (HX / 4);
            *reinterpret_cast<int *>(&si[r][4 * c4]) = w[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) *reinterpret_cast<float4 *>(&sg[c][r][4 * c4]) = v[c][k];
        }
    } else {
        constexpr int PER = (HY * HX + 255) / 256;
        float v0[PER], v1[PER], v2[PER];
        int vi[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + 256 * k;
            const int r = e / HX, c = e - r * HX;
            const int py = by - R + r, px = bx - C0 + c;
            const bool in = e < HY * HX && py >= 0 && py < M && px >= 0 && px < N;
            const size_t o = in ? (size_t)py * N + px : 0;
            vi[k] = in ? (int)__ldg(ib + o) : -1;
            v0[k] = in ? __ldg(g + o) : 0.0f;
            v1[k] = in ? __ldg(g + plane + o) : 0.0f;
            v2[k] = in ? __ldg(g + 2 * plane + o) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + 256 * k;
            if (e >= HY * HX) continue;
            const int r = e / HX, c = e - r * HX;
            si[r][c] = (int8_t)vi[k];
            sg[0][r][c] = v0[k];
            sg[1][r][c] = v1[k];
            sg[2][r][c] = v2[k];
        }
    }
    __syncthreads();
    // every pixel p within R of the tile marks itself in its source's mask
    constexpr int SW = kTX + 2 * R, NS = HY * SW;
    for (int e = tid; e < NS; e += 256) {
        const int r = e / SW, cc = e - r * SW;            // p at tile row r - R, column cc - R
        const int i = si[r][cc + C0 - R];
        // outside the image (-1), or not a member index of this window size
        // (an index map made with another window): selects nothing
        if ((unsigned)i >= (unsigned)(W * W)) continue;
        const int py = by + r - R, px = bx + cc - R;
        const int qy = min(max(py + i / W - R, 0), M - 1), qx = min(max(px + i % W - R, 0), N - 1);
        const int ty = qy - by, tx = qx - bx;
        if (ty >= 0 && ty < kTY && tx >= 0 && tx < kTX)
            atomicOr(&qm[ty][tx], 1u << ((py - qy + R) * W + (px - qx + R)));
    }
    __syncthreads();
    const int ty = tid / (kTX / kQ), x0 = (tid % (kTX / kQ)) * kQ;   // tile coordinates
    const int y = by + ty, X0 = bx + x0;
    if (y >= M || X0 >= N) return;
    float acc[3][kQ];
#pragma unroll
    for (int j = 0; j < kQ; ++j) {
        unsigned mask = qm[ty][x0 + j];
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
        while (mask) {
            const int n = __ffs(mask) - 1;
            mask &= mask - 1;
            const int r = ty + n / W, c = x0 + j + C0 + n % W - R;
            a0 += sg[0][r][c];
            a1 += sg[1][r][c];
            a2 += sg[2][r][c];
        }
        acc[0][j] = a0;
        acc[1][j] = a1;
        acc[2][j] = a2;
    }
    float *o = gx + (size_t)b * 3 * plane + (size_t)y * N + X0;
    if (VEC && X0 + kQ <= N) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            *reinterpret_cast<float4 *>(o + c * plane) = make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < kQ; ++j)
                if (X0 + j < N) o[c * plane + j] = acc[c][j];
    }
}

}  // namespace

cudaError_t run_backward(const float *gy, const int8_t *idx, float *gx, int B, int M, int N, int R, cudaStream_t st)
{
    // vectors when every row starts on a 16-byte (4-byte for the indices) boundary
    const bool vec = N % 4 == 0 && ((uintptr_t)gy & 15) == 0 && ((uintptr_t)gx & 15) == 0 && ((uintptr_t)idx & 3) == 0;
    dim3 block(256), grid((N + kTX - 1) / kTX, (M + kTY - 1) / kTY, B);
    if (R == 1) {
        if (vec) backward_gather<1, true><<<grid, block, 0, st>>>(gy, idx, gx, M, N);
        else backward_gather<1, false><<<grid, block, 0, st>>>(gy, idx, gx, M, N);
    } else if (R == 2) {
        if (vec) backward_gather<2, true><<<grid, block, 0, st>>>(gy, idx, gx, M, N);
        else backward_gather<2, false><<<grid, block, 0, st>>>(gy, idx, gx, M, N);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vdf
