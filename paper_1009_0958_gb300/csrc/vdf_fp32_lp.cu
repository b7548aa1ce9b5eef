// vdf_fp32_lp.cu -- FP32 tile kernel instantiations of the vector median
// filter (Eq. (1)) at orders 2, 1 and infinity, and of the DDF with the
// order-1 or order-infinity distance (exact angles), in every tile shape.
#include "vdf_dispatch.h"

namespace vdf {

namespace {

template <int R, int FILTER, int NORM, int S>
cudaError_t go(const TileParams &prm, cudaStream_t st)
{
    return launch_tile<TileCfg<R, FILTER, EXACT, false, false, kShapes32[S].tw, kShapes32[S].th, NORM>>(prm, st);
}

template <int R, int FILTER, int NORM>
cudaError_t by_shape(const TileParams &prm, int shape, cudaStream_t st)
{
    switch (shape) {
    case 0: return go<R, FILTER, NORM, 0>(prm, st);
    case 1: return go<R, FILTER, NORM, 1>(prm, st);
    case 2: return go<R, FILTER, NORM, 2>(prm, st);
    case 3: return go<R, FILTER, NORM, 3>(prm, st);
    }
    return cudaErrorInvalidValue;
}

template <int R>
cudaError_t by_kind(const TileParams &prm, int filter, int norm, int shape, cudaStream_t st)
{
    if (filter == VMF) {
        switch (norm) {
        case NL2: return by_shape<R, VMF, NL2>(prm, shape, st);
        case NL1: return by_shape<R, VMF, NL1>(prm, shape, st);
        case NLINF: return by_shape<R, VMF, NLINF>(prm, shape, st);
        }
    } else if (filter == DDF) {
        switch (norm) {
        case NL1: return by_shape<R, DDF, NL1>(prm, shape, st);
        case NLINF: return by_shape<R, DDF, NLINF>(prm, shape, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fp32_lp(const TileParams &prm, int R, int filter, int norm, int shape, cudaStream_t st)
{
    if (R == 1) return by_kind<1>(prm, filter, norm, shape, st);
    if (R == 2) return by_kind<2>(prm, filter, norm, shape, st);
    return cudaErrorInvalidValue;
}

}  // namespace vdf
