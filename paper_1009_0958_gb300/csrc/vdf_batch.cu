// vdf_batch.cu -- batches of uneven images, one tile-kernel launch per
// configuration present in the batch.
//
// Images are grouped by configuration (window, filter, tile shape from the
// autotuner).  Work items are (image, tile) pairs numbered image by image
// within a group.  A group's tile kernel takes one of two forms:
//   * one CTA per work item (the default): the item's image comes from a
//     per-item table in the workspace and the block scheduler hands out the
//     items;
//   * persistent: as many CTAs as fit on the SMs at the configuration's
//     occupancy, each taking the next item of its group from an atomic
//     counter in the workspace.
// Both run the FP32 tile body of the configuration at its own block size and
// occupancy (two CTAs per SM where shared memory and registers allow).  The
// loop of the persistent form costs registers (DDF 5x5: 500 bytes of spills
// against 44 in straight-line code), which makes it the slower of the two.
// Pixels whose minimum is not certified are appended to one batch-wide
// recheck list, keyed by batch pixel offset, and a persistent kernel
// re-evaluates them in FP64 (one warp each).  No device-side wait exists: the
// work counters are only ever incremented.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/vdf.h"
#include "vdf_dispatch.h"

namespace vdf {

namespace {

struct BatchDesc {
    const uint8_t *img;
    uint8_t *out;
    int8_t *idx;
    int M, N;
    int tiles_x;
    int tile_base;   // first work item of this image within its group
    int pix_base;    // first batch pixel offset of this image (ascending over the descriptor array)
    int cfg;         // ((win/2 - 1) * 2 + filter) * kNumShapes32 + shape
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

template <int CFG>
struct BCfg {
    static constexpr int SHAPE = CFG % kNumShapes32;
    static constexpr int FILTER = (CFG / kNumShapes32) % 2;
    static constexpr int R = CFG / (2 * kNumShapes32) + 1;
    using C = TileCfg<R, FILTER, EXACT, false, false, kShapes32[SHAPE].tw, kShapes32[SHAPE].th>;
};
constexpr int kNumCfgs = 2 * 2 * kNumShapes32;

// The persistent tile kernel of one configuration.
template <int CFG>
__global__ void __launch_bounds__(BCfg<CFG>::C::NT, BCfg<CFG>::C::MINB) batch_kernel(const BatchParams bp)
{
    using C = typename BCfg<CFG>::C;
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
template <int CFG>
__global__ void __launch_bounds__(BCfg<CFG>::C::NT, BCfg<CFG>::C::MINB) batch_item_kernel(const BatchParams bp)
{
    using C = typename BCfg<CFG>::C;
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
template <int CFG>
cudaError_t launch_group(const BatchParams &bp, int sms, cudaStream_t st, bool persistent)
{
    using C = typename BCfg<CFG>::C;
    if (persistent) batch_kernel<CFG><<<sms * C::MINB, C::NT, C::SMEM, st>>>(bp);
    else batch_item_kernel<CFG><<<bp.total_tiles, C::NT, C::SMEM, st>>>(bp);
    return cudaGetLastError();
}

// The shared-memory opt-in of both forms, set once for every configuration
// before any launch (outside graph capture).
template <int CFG>
cudaError_t configure_group()
{
    cudaError_t e = cudaFuncSetAttribute(batch_item_kernel<CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BCfg<CFG>::C::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)BCfg<CFG>::C::SMEM);
    return e;
}

using GroupLaunch = cudaError_t (*)(const BatchParams &, int, cudaStream_t, bool);
using GroupConfigure = cudaError_t (*)();
template <int... I>
constexpr std::array<GroupLaunch, sizeof...(I)> group_launchers(std::integer_sequence<int, I...>)
{
    return {&launch_group<I>...};
}
template <int... I>
constexpr std::array<GroupConfigure, sizeof...(I)> group_configurers(std::integer_sequence<int, I...>)
{
    return {&configure_group<I>...};
}
constexpr auto kGroupLaunch = group_launchers(std::make_integer_sequence<int, kNumCfgs>{});
constexpr auto kGroupConfigure = group_configurers(std::make_integer_sequence<int, kNumCfgs>{});

// Per-warp shared memory of the largest recheck configuration.
constexpr size_t kRecheckPerWarp = RecheckCfg<2, DDF, EXACT>::PER_WARP;

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
        const int rf = d.cfg / kNumShapes32;   // (R - 1) * 2 + filter
        const unsigned mask = (unsigned)ent.y;
        switch (rf) {
        case 0: recheck_pixel<1, BVDF, EXACT>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        case 1: recheck_pixel<1, DDF, EXACT>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        case 2: recheck_pixel<2, BVDF, EXACT>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        default: recheck_pixel<2, DDF, EXACT>(d.img, d.M, d.N, lin, mask, d.out, d.idx, d.p, bp.q, base, lane); break;
        }
    }
}

// recheck count, overflow flag, one work counter per configuration
constexpr size_t kCtrBytes = 256;
static_assert((2 + kNumCfgs) * sizeof(unsigned) <= kCtrBytes && 2 + kNumCfgs <= kTieCounter &&
                  kCtrBytes == kCounterBlockBytes, "counters fit");

size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }

}  // namespace

}  // namespace vdf

struct vdf_plan {
    // images of one configuration: descriptors first .. first + count - 1
    struct Group {
        int cfg, first, count, tiles;
        long long item_first;   // its first entry of item_image
    };
    std::vector<vdf::BatchDesc> desc;   // grouped by configuration
    std::vector<Group> groups;
    std::vector<int> item_image;        // per work item: its image within the group
    int total_tiles = 0;
    long long total_pixels = 0;
    int q = 4;
    int sms = 1;
    std::atomic<bool> persistent{false};   // tile kernels in the persistent work-queue form
    std::mutex mutex;
    cudaGraphExec_t exec = nullptr;
    void *exec_ws = nullptr;
};

namespace {

int plan_num_sms()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Workspace: counters | descriptors | item table | recheck list.
size_t desc_bytes(const vdf_plan *plan) { return vdf::up16(sizeof(vdf::BatchDesc) * plan->desc.size()); }
size_t table_bytes(const vdf_plan *plan) { return vdf::up16(sizeof(int) * plan->item_image.size()); }

size_t plan_ws_bytes(const vdf_plan *plan)
{
    return vdf::kCtrBytes + desc_bytes(plan) + table_bytes(plan) + sizeof(int2) * (size_t)plan->total_pixels;
}

// Parameters of group g's tile kernel, or (g < 0) of the recheck kernel over
// all descriptors.
vdf::BatchParams plan_params(const vdf_plan *plan, void *ws, int g)
{
    vdf::BatchParams bp{};
    char *base = (char *)ws;
    bp.ctr = (unsigned *)base;
    bp.desc = (const vdf::BatchDesc *)(base + vdf::kCtrBytes);
    const int *table = (const int *)(base + vdf::kCtrBytes + desc_bytes(plan));
    bp.list = (int2 *)(base + vdf::kCtrBytes + desc_bytes(plan) + table_bytes(plan));
    bp.count = (int)plan->desc.size();
    bp.cap = (unsigned)plan->total_pixels;
    bp.q = plan->q;
    if (g >= 0) {
        const vdf_plan::Group &gr = plan->groups[g];
        bp.desc += gr.first;
        bp.count = gr.count;
        bp.total_tiles = gr.tiles;
        bp.next_item = bp.ctr + 2 + g;
        bp.item_image = table + gr.item_first;
    }
    return bp;
}

int set_attributes()
{
    static std::atomic<bool> done[vdf::kMaxDevices];
    const cudaError_t err = vdf::once_per_device(done, [] {
        cudaError_t e = cudaFuncSetAttribute(vdf::batch_recheck_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(vdf::kRecheckPerWarp * vdf::kRecheckWarps));
        for (int c = 0; c < vdf::kNumCfgs && e == cudaSuccess; ++c) e = vdf::kGroupConfigure[c]();
        return e;
    });
    return err == cudaSuccess ? VDF_OK : VDF_E_CUDA;
}

bool ws_ok(const vdf_plan *plan, const void *ws, size_t bytes)
{
    return ws && !((uintptr_t)ws & 255) && bytes >= plan_ws_bytes(plan);
}

}  // namespace

extern "C" {

int vdf_plan_create(vdf_plan **plan, const vdf_image_desc *descs, int count, int dist_mode, int minimax_q)
{
    if (!plan || !descs || count < 1) return VDF_E_INVALID;
    *plan = nullptr;
    if (dist_mode != VDF_DIST_EXACT) return VDF_E_UNSUPPORTED;
    vdf_plan *pl = new (std::nothrow) vdf_plan;
    if (!pl) return VDF_E_INVALID;
    pl->q = minimax_q;
    pl->sms = plan_num_sms();
    std::vector<vdf::BatchDesc> all;
    for (int i = 0; i < count; ++i) {
        const vdf_image_desc &d = descs[i];
        const size_t bytes = (size_t)d.M * d.N * 3;
        const bool bad = !d.img || !d.out || d.M < 1 || d.N < 1 || (d.win != 3 && d.win != 5) ||
                         (d.filter != VDF_BVDF && d.filter != VDF_DDF) ||
                         (d.filter == VDF_DDF && !(d.p >= 0.0 && d.p <= 1.0)) ||
                         ((uintptr_t)d.img < (uintptr_t)d.out + bytes && (uintptr_t)d.out < (uintptr_t)d.img + bytes);
        if (bad) {
            delete pl;
            return VDF_E_INVALID;
        }
        const int shape = vdf_get_tuned_shape(d.win, d.filter, dist_mode);
        vdf::BatchDesc bd{};
        bd.img = d.img;
        bd.out = d.out;
        bd.idx = d.index_out;
        bd.M = d.M;
        bd.N = d.N;
        bd.tiles_x = (d.N + vdf::kShapes32[shape].tw - 1) / vdf::kShapes32[shape].tw;
        bd.cfg = ((d.win / 2 - 1) * 2 + d.filter) * vdf::kNumShapes32 + shape;
        bd.p = d.p;
        all.push_back(bd);
    }
    // group by configuration (5x5 first), images in their given order within a group
    long long tiles = 0, pixels = 0;
    for (int cfg = vdf::kNumCfgs - 1; cfg >= 0; --cfg) {
        vdf_plan::Group gr{cfg, (int)pl->desc.size(), 0, 0, (long long)pl->item_image.size()};
        long long gtiles = 0;
        const int th = vdf::kShapes32[cfg % vdf::kNumShapes32].th;
        for (vdf::BatchDesc bd : all) {
            if (bd.cfg != cfg) continue;
            bd.tile_base = (int)gtiles;
            bd.pix_base = (int)pixels;
            const long long nt = (long long)bd.tiles_x * ((bd.M + th - 1) / th);
            gtiles += nt;
            pixels += (long long)bd.M * bd.N;
            if (gtiles > (1LL << 31) - 1 || pixels > (1LL << 31) - 1) {
                delete pl;
                return VDF_E_INVALID;
            }
            pl->item_image.insert(pl->item_image.end(), (size_t)nt, gr.count);
            pl->desc.push_back(bd);
            ++gr.count;
        }
        if (gr.count == 0) continue;
        gr.tiles = (int)gtiles;
        tiles += gtiles;
        pl->groups.push_back(gr);
    }
    pl->total_tiles = (int)std::min<long long>(tiles, (1LL << 31) - 1);
    pl->total_pixels = pixels;
    *plan = pl;
    return VDF_OK;
}

size_t vdf_plan_workspace_bytes(const vdf_plan *plan) { return plan ? plan_ws_bytes(plan) : 0; }

int vdf_plan_upload(vdf_plan *plan, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!plan) return VDF_E_INVALID;
    if (!ws_ok(plan, workspace, workspace_bytes)) return VDF_E_WORKSPACE;
    cudaError_t e = cudaMemcpyAsync((char *)workspace + vdf::kCtrBytes, plan->desc.data(),
                                    sizeof(vdf::BatchDesc) * plan->desc.size(), cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char *)workspace + vdf::kCtrBytes + desc_bytes(plan), plan->item_image.data(),
                            sizeof(int) * plan->item_image.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? VDF_OK : VDF_E_CUDA;
}

int vdf_filter_batch(vdf_plan *plan, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!plan) return VDF_E_INVALID;
    if (!ws_ok(plan, workspace, workspace_bytes)) return VDF_E_WORKSPACE;
    int rc = set_attributes();
    if (rc != VDF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = plan->sms;
    const int ngroups = (int)plan->groups.size();
    cudaError_t e = cudaMemsetAsync(workspace, 0, vdf::kCtrBytes, st);
    for (int g = 0; g < ngroups && e == cudaSuccess; ++g)
        e = vdf::kGroupLaunch[plan->groups[g].cfg](plan_params(plan, workspace, g), sms, st, plan->persistent.load());
    if (e == cudaSuccess) {
        vdf::batch_recheck_kernel<<<sms * 16, 32 * vdf::kRecheckWarps, vdf::kRecheckPerWarp * vdf::kRecheckWarps, st>>>(
            plan_params(plan, workspace, -1));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? VDF_OK : VDF_E_CUDA;
}

int vdf_plan_graph_launch(vdf_plan *plan, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!plan) return VDF_E_INVALID;
    if (!ws_ok(plan, workspace, workspace_bytes)) return VDF_E_WORKSPACE;
    int rc = set_attributes();
    if (rc != VDF_OK) return rc;
    std::lock_guard<std::mutex> lock(plan->mutex);
    if (!plan->exec || plan->exec_ws != workspace) {
        if (plan->exec) {
            cudaGraphExecDestroy(plan->exec);
            plan->exec = nullptr;
        }
        cudaStream_t cs = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return VDF_E_CUDA;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = vdf_filter_batch(plan, workspace, workspace_bytes, cs);
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (rc == VDF_OK && e2 != cudaSuccess) rc = VDF_E_CUDA;
        } else {
            rc = VDF_E_CUDA;
        }
        if (rc == VDF_OK && cudaGraphInstantiate(&plan->exec, graph, 0) != cudaSuccess) rc = VDF_E_CUDA;
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (rc != VDF_OK) {
            plan->exec = nullptr;
            return rc;
        }
        plan->exec_ws = workspace;
    }
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? VDF_OK : VDF_E_CUDA;
}

int vdf_plan_set_persistent(vdf_plan *plan, int persistent)
{
    if (!plan) return VDF_E_INVALID;
    std::lock_guard<std::mutex> lock(plan->mutex);
    if (plan->persistent.load() != (persistent != 0) && plan->exec) {
        cudaGraphExecDestroy(plan->exec);   // the captured graph holds the other form
        plan->exec = nullptr;
        plan->exec_ws = nullptr;
    }
    plan->persistent = persistent != 0;
    return VDF_OK;
}

void vdf_plan_destroy(vdf_plan *plan)
{
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    delete plan;
}

}  // extern "C"
