// vdf_win7_32.cu -- FP32 certified kernel of the 7x7 window (vdf_win7.cuh),
// every filter kind, distance mode and Minkowski order the library offers.
#include "vdf_dispatch.h"
#include "vdf_win7.cuh"

namespace vdf {

namespace {

template <int FILTER, int DIST, int NORM>
cudaError_t go(const Win7Params &prm, int blocks, cudaStream_t st)
{
    win7_fp32_kernel<FILTER, DIST, NORM><<<blocks, 32 * kWin7Warps, 0, st>>>(prm);
    return cudaGetLastError();
}

}  // namespace

cudaError_t run_win7_fp32(const Win7Params &prm, int filter, int dist, int norm, int sms, cudaStream_t st)
{
    const long long px = (long long)prm.M * prm.N;
    const int blocks = (int)std::min<long long>((px + kWin7Warps - 1) / kWin7Warps, (long long)sms * 16);
    if (filter == VMF) {
        switch (norm) {
        case NL2: return go<VMF, EXACT, NL2>(prm, blocks, st);
        case NL1: return go<VMF, EXACT, NL1>(prm, blocks, st);
        case NLINF: return go<VMF, EXACT, NLINF>(prm, blocks, st);
        }
    } else if (filter == DDF && norm != NL2) {
        if (dist != EXACT) return cudaErrorInvalidValue;
        return norm == NL1 ? go<DDF, EXACT, NL1>(prm, blocks, st) : go<DDF, EXACT, NLINF>(prm, blocks, st);
    } else if (filter == DDF) {
        switch (dist) {
        case EXACT: return go<DDF, EXACT, NL2>(prm, blocks, st);
        case MINIMAX: return go<DDF, MINIMAX, NL2>(prm, blocks, st);
        case RGB: return go<DDF, RGB, NL2>(prm, blocks, st);
        }
    } else if (filter == BVDF) {
        switch (dist) {
        case EXACT: return go<BVDF, EXACT, NL2>(prm, blocks, st);
        case MINIMAX: return go<BVDF, MINIMAX, NL2>(prm, blocks, st);
        case RGB: return go<BVDF, RGB, NL2>(prm, blocks, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace vdf
