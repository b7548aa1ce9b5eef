// vdf_fp64.cu -- FP64 instantiations of the tile kernel and the recheck
// kernel.  Both live in this one translation unit, compiled without
// floating-point contraction, so that a recheck reproduces the tile kernel's
// aggregates bit for bit.
#include "vdf_dispatch.h"

namespace vdf {

namespace {

template <int R, int FILTER>
struct Shape64;   // tile shapes: FP64 registers limit the candidates per CTA
template <>
struct Shape64<1, BVDF> { static constexpr int TW = 32, TH = 8; };
template <>
struct Shape64<1, DDF> { static constexpr int TW = 32, TH = 8; };
template <>
struct Shape64<2, BVDF> { static constexpr int TW = 16, TH = 16; };
template <>
struct Shape64<2, DDF> { static constexpr int TW = 16, TH = 12; };

template <int R, int FILTER, int DIST, bool F32IN>
cudaError_t go(const TileParams &prm, cudaStream_t st)
{
    using S = Shape64<R, FILTER>;
    return launch_tile<TileCfg<R, FILTER, DIST, true, F32IN, S::TW, S::TH>>(prm, st);
}

template <int R, int FILTER>
cudaError_t by_dist(const TileParams &prm, int dist, bool f32in, cudaStream_t st)
{
    if (f32in) {
        if (dist != EXACT) return cudaErrorInvalidValue;
        return go<R, FILTER, EXACT, true>(prm, st);
    }
    switch (dist) {
    case EXACT: return go<R, FILTER, EXACT, false>(prm, st);
    case MINIMAX: return go<R, FILTER, MINIMAX, false>(prm, st);
    case RGB: return go<R, FILTER, RGB, false>(prm, st);
    }
    return cudaErrorInvalidValue;
}

template <int R, int FILTER>
cudaError_t recheck_by_dist(const RecheckParams &prm, int dist, bool f32in, int blocks, cudaStream_t st)
{
    if (f32in) {
        if (dist != EXACT) return cudaErrorInvalidValue;
        return launch_recheck<R, FILTER, EXACT, true>(prm, blocks, st);
    }
    switch (dist) {
    case EXACT: return launch_recheck<R, FILTER, EXACT>(prm, blocks, st);
    case MINIMAX: return launch_recheck<R, FILTER, MINIMAX>(prm, blocks, st);
    case RGB: return launch_recheck<R, FILTER, RGB>(prm, blocks, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fp64(const TileParams &prm, int R, int filter, int dist, bool f32in, cudaStream_t st)
{
    if (R == 1) return filter == DDF ? by_dist<1, DDF>(prm, dist, f32in, st) : by_dist<1, BVDF>(prm, dist, f32in, st);
    if (R == 2) return filter == DDF ? by_dist<2, DDF>(prm, dist, f32in, st) : by_dist<2, BVDF>(prm, dist, f32in, st);
    return cudaErrorInvalidValue;
}

cudaError_t run_recheck(const RecheckParams &prm, int R, int filter, int dist, int blocks, cudaStream_t st,
                        bool f32in)
{
    if (R == 1)
        return filter == DDF ? recheck_by_dist<1, DDF>(prm, dist, f32in, blocks, st)
                             : recheck_by_dist<1, BVDF>(prm, dist, f32in, blocks, st);
    if (R == 2)
        return filter == DDF ? recheck_by_dist<2, DDF>(prm, dist, f32in, blocks, st)
                             : recheck_by_dist<2, BVDF>(prm, dist, f32in, blocks, st);
    return cudaErrorInvalidValue;
}

}  // namespace vdf
