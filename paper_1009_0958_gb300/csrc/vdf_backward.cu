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

template <int R>
__global__ void __launch_bounds__(256) backward_gather(const float *__restrict__ gy, const int8_t *__restrict__ idx,
                                                       float *__restrict__ gx, int M, int N)
{
    constexpr int W = 2 * R + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int b = blockIdx.z;
    if (x >= N) return;
    const size_t plane = (size_t)M * N;
    const int8_t *ib = idx + (size_t)b * plane;
    const float *g = gy + (size_t)b * 3 * plane;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
        const int py = y + dy;
        if (py < 0 || py >= M) continue;
#pragma unroll
        for (int dx = -R; dx <= R; ++dx) {
            const int px = x + dx;
            if (px < 0 || px >= N) continue;
            const size_t o = (size_t)py * N + px;
            const int i = ib[o];
            const int sy = min(max(py + i / W - R, 0), M - 1);
            const int sx = min(max(px + i % W - R, 0), N - 1);
            if (sy == y && sx == x) {
                a0 += g[o];
                a1 += g[plane + o];
                a2 += g[2 * plane + o];
            }
        }
    }
    float *o = gx + (size_t)b * 3 * plane + (size_t)y * N + x;
    o[0] = a0;
    o[plane] = a1;
    o[2 * plane] = a2;
}

}  // namespace

cudaError_t run_backward(const float *gy, const int8_t *idx, float *gx, int B, int M, int N, int R, cudaStream_t st)
{
    dim3 block(256), grid((N + 255) / 256, M, B);
    if (R == 1) backward_gather<1><<<grid, block, 0, st>>>(gy, idx, gx, M, N);
    else if (R == 2) backward_gather<2><<<grid, block, 0, st>>>(gy, idx, gx, M, N);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace vdf
