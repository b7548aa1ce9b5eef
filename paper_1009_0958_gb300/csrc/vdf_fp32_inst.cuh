// vdf_fp32_inst.cuh -- instantiation template of the FP32 tile kernel for one
// tile shape; each vdf_fp32_s<k>.cu instantiates one shape (parallel build).
#pragma once

#include "vdf_dispatch.h"

namespace vdf {

// DDF 5x5 at p = 1/4, 1/2 or 3/4 (exact or chromaticity terms) runs with
// score slots (TileCfg::SQ = 4p): the selection decides from the same
// certified Omega^4 scores, formed where the aggregates are emitted (not for
// the diagnostic score dump, which reads raw aggregates).
template <int TW, int TH, int A>
cudaError_t launch_score_slots(const TileParams &prm, int dist, cudaStream_t st)
{
    return dist == EXACT ? launch_tile<TileCfg<2, DDF, EXACT, false, false, TW, TH, NL2, false, A>>(prm, st)
                         : launch_tile<TileCfg<2, DDF, RGB, false, false, TW, TH, NL2, false, A>>(prm, st);
}

template <int TW, int TH>
cudaError_t run_fp32_shape(const TileParams &prm, int R, int filter, int dist, cudaStream_t st)
{
    switch (prm.dbg_fe ? 0 : score_slot_exponent(R, filter, dist, NL2, prm.p)) {
    case 1: return launch_score_slots<TW, TH, 1>(prm, dist, st);
    case 2: return launch_score_slots<TW, TH, 2>(prm, dist, st);
    case 3: return launch_score_slots<TW, TH, 3>(prm, dist, st);
    default: break;
    }
    auto go = [&](auto r, auto f, auto d) {
        return launch_tile<TileCfg<decltype(r)::value, decltype(f)::value, decltype(d)::value, false, false, TW, TH>>(
            prm, st);
    };
    using I = std::integral_constant<int, 0>;
    (void)sizeof(I);
    auto by_dist = [&](auto r, auto f) -> cudaError_t {
        switch (dist) {
        case EXACT: return go(r, f, std::integral_constant<int, EXACT>{});
        case MINIMAX: return go(r, f, std::integral_constant<int, MINIMAX>{});
        case RGB: return go(r, f, std::integral_constant<int, RGB>{});
        }
        return cudaErrorInvalidValue;
    };
    auto by_filter = [&](auto r) -> cudaError_t {
        return filter == DDF ? by_dist(r, std::integral_constant<int, DDF>{})
                             : by_dist(r, std::integral_constant<int, BVDF>{});
    };
    if (R == 1) return by_filter(std::integral_constant<int, 1>{});
    if (R == 2) return by_filter(std::integral_constant<int, 2>{});
    return cudaErrorInvalidValue;
}

}  // namespace vdf
