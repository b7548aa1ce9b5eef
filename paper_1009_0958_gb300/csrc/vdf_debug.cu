// vdf_debug.cu -- the FP32 pair terms of the tile kernel for given pixel
// pairs (diagnostic entry vdf_debug_fp32_terms).  Built with the same flags
// as the FP32 tile kernels (flush-to-zero), so the values are the ones the
// tile kernel sums.
#include "vdf_dispatch.h"

namespace vdf {

namespace {

__device__ __forceinline__ float4 pixel_of(const int *c)
{
    const float x = (float)c[0], y = (float)c[1], z = (float)c[2];
    return make_float4(x, y, z, (float)(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]));
}

template <int DIST>
__global__ void terms_kernel(const int *pairs, int n, int q, float *angle_out, float *l2_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = pixel_of(pairs + 6 * (size_t)i), b = pixel_of(pairs + 6 * (size_t)i + 3);
    const PairInts r = pair_ints(a, b);
    if (angle_out) {
        float ang;
        if constexpr (DIST == EXACT) ang = angle32(r);
        else if constexpr (DIST == MINIMAX) ang = minimax32(r, make_aux<DIST>(a), make_aux<DIST>(b), q);
        else ang = chroma32(a, b, make_aux<DIST>(a), make_aux<DIST>(b));
        angle_out[i] = ang;
    }
    if (l2_out) l2_out[i] = l2term32(a, b, r.d);
}

}  // namespace

cudaError_t run_debug_terms(const int *pairs, int n, int dist, int q, float *angle_out, float *l2_out,
                            cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int threads = 256, blocks = (n + threads - 1) / threads;
    switch (dist) {
    case EXACT: terms_kernel<EXACT><<<blocks, threads, 0, st>>>(pairs, n, q, angle_out, l2_out); break;
    case MINIMAX: terms_kernel<MINIMAX><<<blocks, threads, 0, st>>>(pairs, n, q, angle_out, l2_out); break;
    default: terms_kernel<RGB><<<blocks, threads, 0, st>>>(pairs, n, q, angle_out, l2_out); break;
    }
    return cudaGetLastError();
}

}  // namespace vdf
