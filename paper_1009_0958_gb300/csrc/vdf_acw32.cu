// vdf_acw32.cu -- FP32 certified tile kernel of the ACWDDF (Eq. (9)): the
// DDF tile kernel whose selection adds the centre-weighted VMF levels and the
// switch, every distance mode, in every tile shape.
#include "vdf_dispatch.h"

namespace vdf {

namespace {

template <int R, int DIST, int S>
cudaError_t go(const TileParams &prm, cudaStream_t st)
{
    return launch_tile<TileCfg<R, DDF, DIST, false, false, kShapes32[S].tw, kShapes32[S].th, NL2, true>>(prm, st);
}

template <int R, int DIST>
cudaError_t by_shape(const TileParams &prm, int shape, cudaStream_t st)
{
    switch (shape) {
    case 0: return go<R, DIST, 0>(prm, st);
    case 1: return go<R, DIST, 1>(prm, st);
    case 2: return go<R, DIST, 2>(prm, st);
    case 3: return go<R, DIST, 3>(prm, st);
    }
    return cudaErrorInvalidValue;
}

template <int R>
cudaError_t by_dist(const TileParams &prm, int dist, int shape, cudaStream_t st)
{
    switch (dist) {
    case EXACT: return by_shape<R, EXACT>(prm, shape, st);
    case MINIMAX: return by_shape<R, MINIMAX>(prm, shape, st);
    case RGB: return by_shape<R, RGB>(prm, shape, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fp32_acw(const TileParams &prm, int R, int dist, int shape, cudaStream_t st)
{
    if (R == 1) return by_dist<1>(prm, dist, shape, st);
    if (R == 2) return by_dist<2>(prm, dist, shape, st);
    return cudaErrorInvalidValue;
}

}  // namespace vdf
