// vdf_acw64.cu -- FP64 tile kernel and FP64 recheck of the ACWDDF (Eq. (9)).
// Both in this one translation unit, compiled without floating-point
// contraction (as vdf_fp64.cu), so that a recheck reproduces the FP64 tile
// kernel's aggregates and decisions bit for bit.
#include "vdf_dispatch.h"

namespace vdf {

namespace {

template <int R, int DIST>
cudaError_t go(const TileParams &prm, cudaStream_t st)
{
    // the FP64 DDF tile shapes
    constexpr int TW = R == 1 ? 32 : 16, TH = R == 1 ? 8 : 12;
    return launch_tile<TileCfg<R, DDF, DIST, true, false, TW, TH, NL2, true>>(prm, st);
}

template <int R>
cudaError_t by_dist(const TileParams &prm, int dist, cudaStream_t st)
{
    switch (dist) {
    case EXACT: return go<R, EXACT>(prm, st);
    case MINIMAX: return go<R, MINIMAX>(prm, st);
    case RGB: return go<R, RGB>(prm, st);
    }
    return cudaErrorInvalidValue;
}

template <int R>
cudaError_t recheck_by_dist(const RecheckParams &prm, int dist, int blocks, cudaStream_t st)
{
    switch (dist) {
    case EXACT: return launch_recheck<R, DDF, EXACT, false, NL2, true>(prm, blocks, st);
    case MINIMAX: return launch_recheck<R, DDF, MINIMAX, false, NL2, true>(prm, blocks, st);
    case RGB: return launch_recheck<R, DDF, RGB, false, NL2, true>(prm, blocks, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fp64_acw(const TileParams &prm, int R, int dist, cudaStream_t st)
{
    if (R == 1) return by_dist<1>(prm, dist, st);
    if (R == 2) return by_dist<2>(prm, dist, st);
    return cudaErrorInvalidValue;
}

cudaError_t run_recheck_acw(const RecheckParams &prm, int R, int dist, int blocks, cudaStream_t st)
{
    if (R == 1) return recheck_by_dist<1>(prm, dist, blocks, st);
    if (R == 2) return recheck_by_dist<2>(prm, dist, blocks, st);
    return cudaErrorInvalidValue;
}

}  // namespace vdf
