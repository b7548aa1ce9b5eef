// vdf_fp64_lp.cu -- FP64 tile and recheck kernels of the vector median
// filter (Eq. (1)) at orders 2, 1 and infinity, and of the DDF with the
// order-1 or order-infinity distance (exact angles).  Compiled like
// vdf_fp64.cu, without floating-point contraction, so that a recheck
// reproduces the FP64 tile kernel's aggregates bit for bit.
#include "vdf_dispatch.h"

namespace vdf {

namespace {

// FP64 tile shapes: the VMF has one aggregate per member (as BVDF), the DDF two
template <int R, int FILTER>
struct ShapeLp {
    static constexpr int TW = R == 1 ? 32 : 16;
    static constexpr int TH = R == 1 ? 8 : (FILTER == DDF ? 12 : 16);
};

template <int R, int FILTER, int NORM>
cudaError_t go(const TileParams &prm, cudaStream_t st)
{
    using S = ShapeLp<R, FILTER>;
    return launch_tile<TileCfg<R, FILTER, EXACT, true, false, S::TW, S::TH, NORM>>(prm, st);
}

template <int R>
cudaError_t by_kind(const TileParams &prm, int filter, int norm, cudaStream_t st)
{
    if (filter == VMF) {
        switch (norm) {
        case NL2: return go<R, VMF, NL2>(prm, st);
        case NL1: return go<R, VMF, NL1>(prm, st);
        case NLINF: return go<R, VMF, NLINF>(prm, st);
        }
    } else if (filter == DDF) {
        switch (norm) {
        case NL1: return go<R, DDF, NL1>(prm, st);
        case NLINF: return go<R, DDF, NLINF>(prm, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <int R>
cudaError_t recheck_by_kind(const RecheckParams &prm, int filter, int norm, int blocks, cudaStream_t st)
{
    if (filter == VMF) {
        switch (norm) {
        case NL2: return launch_recheck<R, VMF, EXACT, false, NL2>(prm, blocks, st);
        case NL1: return launch_recheck<R, VMF, EXACT, false, NL1>(prm, blocks, st);
        case NLINF: return launch_recheck<R, VMF, EXACT, false, NLINF>(prm, blocks, st);
        }
    } else if (filter == DDF) {
        switch (norm) {
        case NL1: return launch_recheck<R, DDF, EXACT, false, NL1>(prm, blocks, st);
        case NLINF: return launch_recheck<R, DDF, EXACT, false, NLINF>(prm, blocks, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fp64_lp(const TileParams &prm, int R, int filter, int norm, cudaStream_t st)
{
    if (R == 1) return by_kind<1>(prm, filter, norm, st);
    if (R == 2) return by_kind<2>(prm, filter, norm, st);
    return cudaErrorInvalidValue;
}

cudaError_t run_recheck_lp(const RecheckParams &prm, int R, int filter, int norm, int blocks, cudaStream_t st)
{
    if (R == 1) return recheck_by_kind<1>(prm, filter, norm, blocks, st);
    if (R == 2) return recheck_by_kind<2>(prm, filter, norm, blocks, st);
    return cudaErrorInvalidValue;
}

}  // namespace vdf
