// vdf_win7_64.cu -- FP64 path of the 7x7 window and the FP64 recheck of the
// pixels its FP32 kernel lists.  Both run recheck_pixel (every member) in this
// one translation unit, compiled without floating-point contraction, so the
// recheck reproduces the FP64 path bit for bit.
#include <algorithm>

#include "vdf_dispatch.h"
#include "vdf_win7.cuh"

namespace vdf {

namespace {

template <int FILTER, int DIST, int NORM>
cudaError_t go64(const RecheckParams &prm, double *agg, int sms, cudaStream_t st)
{
    using C = RecheckCfg<3, FILTER, DIST>;
    static std::atomic<bool> configured[kMaxDevices];
    cudaError_t e = once_per_device(configured, [] {
        return cudaFuncSetAttribute(win7_fp64_kernel<FILTER, DIST, NORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)C::SMEM);
    });
    if (e != cudaSuccess) return e;
    const long long px = (long long)prm.M * prm.N;
    const int blocks = (int)std::min<long long>(px, (long long)sms * 16);
    win7_fp64_kernel<FILTER, DIST, NORM><<<blocks, 32, C::SMEM, st>>>(prm, agg);
    return cudaGetLastError();
}

template <class F>
cudaError_t by_kind(int filter, int dist, int norm, F go)
{
    if (filter == VMF) {
        switch (norm) {
        case NL2: return go(std::integral_constant<int, VMF>{}, std::integral_constant<int, EXACT>{},
                            std::integral_constant<int, NL2>{});
        case NL1: return go(std::integral_constant<int, VMF>{}, std::integral_constant<int, EXACT>{},
                            std::integral_constant<int, NL1>{});
        case NLINF: return go(std::integral_constant<int, VMF>{}, std::integral_constant<int, EXACT>{},
                              std::integral_constant<int, NLINF>{});
        }
    } else if (filter == DDF && norm != NL2) {
        if (dist != EXACT) return cudaErrorInvalidValue;
        if (norm == NL1)
            return go(std::integral_constant<int, DDF>{}, std::integral_constant<int, EXACT>{},
                      std::integral_constant<int, NL1>{});
        return go(std::integral_constant<int, DDF>{}, std::integral_constant<int, EXACT>{},
                  std::integral_constant<int, NLINF>{});
    } else if (filter == DDF || filter == BVDF) {
        auto by_dist = [&](auto f) -> cudaError_t {
            switch (dist) {
            case EXACT: return go(f, std::integral_constant<int, EXACT>{}, std::integral_constant<int, NL2>{});
            case MINIMAX: return go(f, std::integral_constant<int, MINIMAX>{}, std::integral_constant<int, NL2>{});
            case RGB: return go(f, std::integral_constant<int, RGB>{}, std::integral_constant<int, NL2>{});
            }
            return cudaErrorInvalidValue;
        };
        return filter == DDF ? by_dist(std::integral_constant<int, DDF>{}) : by_dist(std::integral_constant<int, BVDF>{});
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_win7_fp64(const RecheckParams &prm, double *agg, int filter, int dist, int norm, int sms,
                          cudaStream_t st)
{
    return by_kind(filter, dist, norm, [&](auto f, auto d, auto n) {
        return go64<decltype(f)::value, decltype(d)::value, decltype(n)::value>(prm, agg, sms, st);
    });
}

cudaError_t run_win7_recheck(const RecheckParams &prm, int filter, int dist, int norm, int blocks, cudaStream_t st)
{
    return by_kind(filter, dist, norm, [&](auto f, auto d, auto n) {
        return launch_recheck<3, decltype(f)::value, decltype(d)::value, false, decltype(n)::value>(prm, blocks, st);
    });
}

}  // namespace vdf
