// vdf_batch_kernels.cuh -- kernels of the uneven-image batch (vdf_batch.cu),
// templated on the distance mode; each mode is instantiated in a translation
// unit of its own (vdf_batch_d0.cu .. vdf_batch_d2.cu) so they compile in
// parallel.  Not part of the public ABI.
#pragma once

#include <array>
#include <utility>

#include "vdf_dispatch.h"

namespace vdf {

struct BatchDesc {
    const uint8_t *img;
    uint8_t *out;
    int8_t *idx;
    int M, N;
    int tiles_x;
    int tile_base;   // first work item of this image within its group
    int pix_base;    // first batch pixel offset of this image (ascending over the descriptor array)
    int cfg;         // ((win/2 - 1) * 2 + filter) * kNumShapes32 + shape, or for the
                     // DDF 5x5 at p = a/4: kScoreCfg0 + (a - 1) * kNumShapes32 + shape
    double p;
};

struct BatchParams {
    const BatchDesc *desc;   // the group's descriptors (tile kernel) or all of them (recheck kernel)
    int count;
    int total_tiles;         // work items of the group
    unsigned *ctr;           // [0] recheck count, [1] overflow
    unsigned *next_item;     // the group's work counter (persistent form)
    const int *item_image;   // the group's image of every work item (one-CTA-per-item form)
    int2 *list;
    unsigned cap;
    int q;
};

// Configurations: window x filter x tile shape, then the DDF 5x5 at p = a/4
// (a = 1, 2, 3) with score slots (exact and chromaticity terms) in every shape.
constexpr int kScoreCfg0 = 2 * 2 * kNumShapes32;
constexpr int kNumCfgs = kScoreCfg0 + 3 * kNumShapes32;

// The configuration a kernel is instantiated for: Method 1 has no score-slot
// configurations (its plans never use them), so those entries reuse the raw
// DDF 5x5 kernels.
template <int DIST, int CFG>
constexpr int canonical_cfg()
{
    return (CFG >= kScoreCfg0 && DIST == MINIMAX) ? kScoreCfg0 - kNumShapes32 + CFG % kNumShapes32 : CFG;
}

template <int DIST, int CFG>
struct BCfg {
    static constexpr int SHAPE = CFG % kNumShapes32;
    static constexpr bool SCORE = CFG >= kScoreCfg0;
    static_assert(!SCORE || DIST != MINIMAX, "no score slots for Method 1");
    static constexpr int FILTER = SCORE ? DDF : (CFG / kNumShapes32) % 2;
    static constexpr int R = SCORE ? 2 : CFG / (2 * kNumShapes32) + 1;
    using C = TileCfg<R, FILTER, DIST, false, false, kShapes32[SHAPE].tw, kShapes32[SHAPE].th, NL2, false,
                      SCORE ? 1 + (CFG - kScoreCfg0) / kNumShapes32 : -1>;
};

// The persistent tile kernel of one configuration.
template <int DIST, int CFG>
__global__ void __launch_bounds__(BCfg<DIST, CFG>::C::NT, BCfg<DIST, CFG>::C::MINB) batch_kernel(const BatchParams bp)
{
    using C = typename BCfg<DIST, CFG>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    // The CTA's current item and the next one (taken from the queue one item
    // ahead, so the atomic's round trip overlaps the current tile), and the
    // current image: its descriptor and the first item past it.  A CTA's
    // items only increase, so the image index only moves forward; most items
    // fall in the image of the one before and need no descriptor load.
    __shared__ int s_item[2];
    __shared__ int s_img, s_end;
    __shared__ BatchDesc s_desc;
    if (threadIdx.x == 0) {
        s_item[0] = (int)atomicAdd(bp.next_item, 1u);
        s_img = -1;
        s_end = 0;
    }
    for (int it = 0;; it ^= 1) {
        __syncthreads();   // s_item[it] is published; the previous item is done with shared memory
        const int item = s_item[it];
        if (item >= bp.total_tiles) break;
        int next = 0;
        if (threadIdx.x == 0) {
            next = (int)atomicAdd(bp.next_item, 1u);
            if (item >= s_end) {
                int img = s_img, end = s_end;
                while (item >= end) {
                    ++img;
                    end = img + 1 < bp.count ? bp.desc[img + 1].tile_base : bp.total_tiles;
                }
                s_img = img;
                s_end = end;
                s_desc = bp.desc[img];
            }
        }
        __syncthreads();   // s_desc is current
        TileParams prm{};
        prm.img = s_desc.img;
        prm.out = s_desc.out;
        prm.idx = s_desc.idx;
        prm.recheck_list = bp.list;
        prm.recheck_ctr = bp.ctr;
        prm.recheck_cap = bp.cap;
        prm.pix_base = s_desc.pix_base;
        prm.M = s_desc.M;
        prm.N = s_desc.N;
        prm.B = 1;
        prm.p = s_desc.p;
        prm.q = bp.q;
        const int t = item - s_desc.tile_base, tiles_x = s_desc.tiles_x;
        tile_body<C, C::NT>(prm, 0, (t % tiles_x) * C::TW, (t / tiles_x) * C::TH, smem);
        if (threadIdx.x == 0) s_item[it ^ 1] = next;
    }
}

// The same work as one CTA per item: the item's image comes from the
// per-item table, the block scheduler is the queue.  Straight-line code gets
// the register allocation of the single-image tile kernel, which a loop
// around the tile body does not.
template <int DIST, int CFG>
__global__ void __launch_bounds__(BCfg<DIST, CFG>::C::NT, BCfg<DIST, CFG>::C::MINB) batch_item_kernel(const BatchParams bp)
{
    using C = typename BCfg<DIST, CFG>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const int item = blockIdx.x;
    const BatchDesc &d = bp.desc[bp.item_image[item]];
    TileParams prm{};
    prm.img = d.img;
    prm.out = d.out;
    prm.idx = d.idx;
    prm.recheck_list = bp.list;
    prm.recheck_ctr = bp.ctr;
    prm.recheck_cap = bp.cap;
    prm.pix_base = d.pix_base;
    prm.M = d.M;
    prm.N = d.N;
    prm.B = 1;
    prm.p = d.p;
    prm.q = bp.q;
    const int t = item - d.tile_base, tiles_x = d.tiles_x;
    tile_body<C, C::NT>(prm, 0, (t % tiles_x) * C::TW, (t / tiles_x) * C::TH, smem);
}

// Launch of one group's kernel: persistent (one CTA per SM per resident
// CTA), or one CTA per item.
template <int DIST, int CFG>
cudaError_t launch_group(const BatchParams &bp, int sms, cudaStream_t st, bool persistent)
{
    using C = typename BCfg<DIST, CFG>::C;
    if (persistent) batch_kernel<DIST, CFG><<<sms * C::MINB, C::NT, C::SMEM, st>>>(bp);
    else batch_item_kernel<DIST, CFG><<<bp.total_tiles, C::NT, C::SMEM, st>>>(bp);
    return cudaGetLastError();
}

// The shared-memory opt-in of both forms, set once for every configuration
// before any launch (outside graph capture).
template <int DIST, int CFG>
cudaError_t configure_group()
{
    cudaError_t e = cudaFuncSetAttribute(batch_item_kernel<DIST, CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BCfg<DIST, CFG>::C::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<DIST, CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)BCfg<DIST, CFG>::C::SMEM);
    return e;
}

using GroupLaunch = cudaError_t (*)(const BatchParams &, int, cudaStream_t, bool);
using GroupConfigure = cudaError_t (*)();
template <int DIST, int... I>
constexpr std::array<GroupLaunch, sizeof...(I)> group_launchers(std::integer_sequence<int, I...>)
{
    return {&launch_group<DIST, canonical_cfg<DIST, I>()>...};
}
template <int DIST, int... I>
constexpr std::array<GroupConfigure, sizeof...(I)> group_configurers(std::integer_sequence<int, I...>)
{
    return {&configure_group<DIST, canonical_cfg<DIST, I>()>...};
}

// Per-warp shared memory of the largest recheck configuration.
constexpr size_t kRecheckPerWarp = RecheckCfg<2, DDF, EXACT>::PER_WARP;

template <int DIST>
__global__ void __launch_bounds__(32 * kRecheckWarps) batch_recheck_kernel(const BatchParams bp)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *base = smem + wid * kRecheckPerWarp;
    const unsigned count = min(bp.ctr[0], bp.cap);
    const int nwarps = gridDim.x * kRecheckWarps;
    for (unsigned it = blockIdx.x * kRecheckWarps + wid; it < count; it += nwarps) {
        const int2 ent = bp.list[it];
        int lo = 0, hi = bp.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp.desc[mid].pix_base <= ent.x) lo = mid;
            else hi = mid - 1;
        }
        const BatchDesc d = bp.desc[lo];
        const int lin = ent.x - d.pix_base;
        const int rf = d.cfg / kNumShapes32;   // (R - 1) * 2 + filter; 4..6: DDF 5x5 with score slots
        const unsigned mask = (unsigned)ent.y;
        switch (rf) {
        case 0: recheck_pixel<1, BVDF, DIST>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        case 1: recheck_pixel<1, DDF, DIST>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        case 2: recheck_pixel<2, BVDF, DIST>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        default: recheck_pixel<2, DDF, DIST>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        }
    }
}

// The operations of one distance mode, defined in its instantiation unit.
template <int DIST>
struct BatchOps {
    // the tile kernel of configuration cfg over one group's work items
    static cudaError_t launch(int cfg, const BatchParams &bp, int sms, cudaStream_t st, bool persistent);
    // the shared-memory opt-in of every configuration's kernels and of the recheck
    static cudaError_t configure();
    // the FP64 recheck of the batch's listed pixels
    static cudaError_t recheck(const BatchParams &bp, int blocks, cudaStream_t st);
};

// Definitions, included by the instantiation units only.
#ifdef VDF_BATCH_INSTANTIATE
template <int DIST>
cudaError_t BatchOps<DIST>::launch(int cfg, const BatchParams &bp, int sms, cudaStream_t st, bool persistent)
{
    static constexpr auto table = group_launchers<DIST>(std::make_integer_sequence<int, kNumCfgs>{});
    if (cfg < 0 || cfg >= kNumCfgs) return cudaErrorInvalidValue;
    return table[cfg](bp, sms, st, persistent);
}

template <int DIST>
cudaError_t BatchOps<DIST>::configure()
{
    static constexpr auto table = group_configurers<DIST>(std::make_integer_sequence<int, kNumCfgs>{});
    cudaError_t e = cudaFuncSetAttribute(batch_recheck_kernel<DIST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kRecheckPerWarp * kRecheckWarps));
    for (int c = 0; c < kNumCfgs && e == cudaSuccess; ++c) e = table[c]();
    return e;
}

template <int DIST>
cudaError_t BatchOps<DIST>::recheck(const BatchParams &bp, int blocks, cudaStream_t st)
{
    batch_recheck_kernel<DIST><<<blocks, 32 * kRecheckWarps, kRecheckPerWarp * kRecheckWarps, st>>>(bp);
    return cudaGetLastError();
}
#endif

extern template struct BatchOps<EXACT>;
extern template struct BatchOps<MINIMAX>;
extern template struct BatchOps<RGB>;

}  // namespace vdf
