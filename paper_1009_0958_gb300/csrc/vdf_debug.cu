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

// Float pixels (n x 6 floats, raw values): normalised as the tile kernel
// holds them; NaN for a pair with an unsafe pixel.
__global__ void terms_f32_kernel(const float *pairs, int n, float *angle_out, float *l2_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *q = pairs + 6 * (size_t)i;
    bool sa, sb;
    const float4 a = normalize_f32(q[0], q[1], q[2], sa), b = normalize_f32(q[3], q[4], q[5], sb);
    const bool ok = sa && sb;
    if (angle_out) angle_out[i] = ok ? angle32f(a, b) : NAN;
    if (l2_out) l2_out[i] = ok ? l2term32f(a, b) : NAN;
}

// Largest relative error, in units of u = 2^-24, of the approximate square
// root over every positive normal float: r = sqrt.approx(x) is compared with
// the exact root through the exact residual r^2 - x (one FMA rounding):
// (r - sqrt(x)) / sqrt(x) = (r^2 - x) / (x (1 + r / sqrt(x))), evaluated in
// double.
__global__ void sqrt_error_kernel(unsigned *max_err_bits)
{
    float worst = 0.0f;
    for (unsigned bits = 0x00800000u + blockIdx.x * blockDim.x + threadIdx.x; bits < 0x7f800000u;
         bits += gridDim.x * blockDim.x) {
        const float x = __uint_as_float(bits);
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        const double xd = x, rd = r, sd = sqrt(xd);
        const double rel = fabs(rd - sd) / sd;
        worst = fmaxf(worst, (float)(rel * 16777216.0));
    }
    atomicMax(max_err_bits, __float_as_uint(worst));
}

}  // namespace

cudaError_t run_debug_terms_f32(const float *pairs, int n, float *angle_out, float *l2_out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    terms_f32_kernel<<<(n + 255) / 256, 256, 0, st>>>(pairs, n, angle_out, l2_out);
    return cudaGetLastError();
}

cudaError_t run_debug_sqrt_error(unsigned *max_err_bits, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(max_err_bits, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    sqrt_error_kernel<<<152 * 8, 256, 0, st>>>(max_err_bits);
    return cudaGetLastError();
}

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
