// vdf_fp32.cu -- FP32 instantiations of the tile kernel (certified scores,
// FP64 recheck list).
#include "vdf_dispatch.h"

namespace vdf {

namespace {

template <int R, int FILTER, int DIST>
cudaError_t go(const TileParams &prm, cudaStream_t st)
{
    return launch_tile<TileCfg<R, FILTER, DIST, false, false, 32, 16>>(prm, st);
}

template <int R, int FILTER>
cudaError_t by_dist(const TileParams &prm, int dist, cudaStream_t st)
{
    switch (dist) {
    case EXACT: return go<R, FILTER, EXACT>(prm, st);
    case MINIMAX: return go<R, FILTER, MINIMAX>(prm, st);
    case RGB: return go<R, FILTER, RGB>(prm, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fp32(const TileParams &prm, int R, int filter, int dist, cudaStream_t st)
{
    if (R == 1) return filter == DDF ? by_dist<1, DDF>(prm, dist, st) : by_dist<1, BVDF>(prm, dist, st);
    if (R == 2) return filter == DDF ? by_dist<2, DDF>(prm, dist, st) : by_dist<2, BVDF>(prm, dist, st);
    return cudaErrorInvalidValue;
}

}  // namespace vdf
