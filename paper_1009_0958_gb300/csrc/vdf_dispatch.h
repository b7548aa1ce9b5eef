// vdf_dispatch.h -- internal entry points between the C ABI (vdf_api.cu) and
// the kernel instantiation units (vdf_fp64.cu, vdf_fp32.cu).
#pragma once

#include <cuda_runtime.h>

#include "vdf_tile.cuh"

namespace vdf {

// FP64 tile kernel (uint8 input, or float32 NCHW input when f32in).
cudaError_t run_fp64(const TileParams &prm, int R, int filter, int dist, bool f32in, cudaStream_t st);
// FP32 certified tile kernel (uint8 input), in one of kNumShapes32 tile shapes.
struct TileShape {
    int tw, th;
};
constexpr int kNumShapes32 = 4;
// 28x16 gives a 640-thread block (a multiple of 128), which leaves 96
// registers per thread for DDF 5x5 instead of the 80 of 32x16's 736.  24x12
// (448 threads) fits two blocks per SM where the slots are single values
// (BVDF, VMF, and the DDF's score slots at p = 1/4, 1/2, 3/4), and for the
// DDF's raw slots with one plane buffer.
inline constexpr TileShape kShapes32[kNumShapes32] = {{32, 16}, {32, 8}, {24, 12}, {28, 16}};
cudaError_t run_fp32(const TileParams &prm, int R, int filter, int dist, int shape, cudaStream_t st);
// The exponent a of the FP32 kernel's score slots (TileCfg::SQ: each slot
// holds Omega^4 = SA^a SL^(4-a)), or 0 for raw slots: the DDF 5x5 with the
// exact or chromaticity terms, order 2, at p = a / 4 for a = 1, 2, 3 (p = 1/2
// orders like the plain product of Eq. (3)).  Such configurations have tile-
// shape table entries of their own.
inline int score_slot_exponent(int R, int filter, int dist, int norm, double p)
{
    if (R != 2 || filter != DDF || (dist != EXACT && dist != RGB) || norm != NL2) return 0;
    const float p4 = 4.0f * (float)p;
    return (p4 == 1.0f || p4 == 2.0f || p4 == 3.0f) ? (int)p4 : 0;
}
// The tuned tile shape of a configuration at DDF exponent p (order 2).
int tuned_shape_p(int win, int filter, int dist, double p);
// Gradient gather of the float32 path.
cudaError_t run_backward(const float *gy, const int8_t *idx, float *gx, int B, int M, int N, int R, cudaStream_t st);
// FP32 certified tile kernel for float32 B x 3 x M x N input (exact mode, 32x16 tiles).
cudaError_t run_fp32_f32in(const TileParams &prm, int R, int filter, cudaStream_t st);
// FP64 recheck of the pixels listed by run_fp32 (f32in: by run_fp32_f32in).
cudaError_t run_recheck(const RecheckParams &prm, int R, int filter, int dist, int blocks, cudaStream_t st,
                        bool f32in = false);

// The VMF and the Minkowski orders 1 and infinity (uint8 input, exact
// mode): filter VMF at norm NL2 / NL1 / NLINF, or DDF at NL1 / NLINF.
cudaError_t run_fp32_lp(const TileParams &prm, int R, int filter, int norm, int shape, cudaStream_t st);
cudaError_t run_fp64_lp(const TileParams &prm, int R, int filter, int norm, cudaStream_t st);
cudaError_t run_recheck_lp(const RecheckParams &prm, int R, int filter, int norm, int blocks, cudaStream_t st);

// ACWDDF (Eq. (9)), uint8 input, every distance mode: the FP32 certified tile
// kernel (one of kNumShapes32 shapes), the FP64 tile kernel, and the FP64
// recheck of the pixels the FP32 kernel lists.
cudaError_t run_fp32_acw(const TileParams &prm, int R, int dist, int shape, cudaStream_t st);
cudaError_t run_fp64_acw(const TileParams &prm, int R, int dist, cudaStream_t st);
cudaError_t run_recheck_acw(const RecheckParams &prm, int R, int dist, int blocks, cudaStream_t st);

// The 7x7 window (vdf_win7.cuh): FP32 certified kernel, FP64 path (agg may
// be null) and the FP64 recheck of the pixels the FP32 kernel lists.
struct Win7Params;
cudaError_t run_win7_fp32(const Win7Params &prm, int filter, int dist, int norm, int sms, cudaStream_t st);
cudaError_t run_win7_fp64(const RecheckParams &prm, double *agg, int filter, int dist, int norm, int sms,
                          cudaStream_t st);
cudaError_t run_win7_recheck(const RecheckParams &prm, int filter, int dist, int norm, int blocks, cudaStream_t st);

// The argument checks of vdf_filter's FP32 path, except those of the workspace.
int check_args_no_workspace(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                            int minimax_q, const uint8_t *out, const int8_t *index_out);

// FP32 pair terms of n pixel pairs (n x 6 ints), as the FP32 tile kernel computes them.
cudaError_t run_debug_terms(const int *pairs, int n, int dist, int q, float *angle_out, float *l2_out,
                            cudaStream_t st);
// The same for float pixels (n x 6 floats; NaN where a pixel is unsafe).
cudaError_t run_debug_terms_f32(const float *pairs, int n, float *angle_out, float *l2_out, cudaStream_t st);
// Largest relative error (units of 2^-24, as float bits) of the approximate
// square root over every positive normal float.
cudaError_t run_debug_sqrt_error(unsigned *max_err_bits, cudaStream_t st);

}  // namespace vdf
