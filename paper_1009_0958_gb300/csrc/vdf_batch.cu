// vdf_batch.cu -- batches of uneven images in one persistent launch.
//
// Work items are (image, tile) pairs numbered image by image.  The tile
// kernel runs one CTA per SM; each CTA takes the next item from an atomic
// counter in the workspace, finds its image by binary search over the
// images' first item numbers, and runs the FP32 tile body of that image's
// configuration (window, filter, tile shape).  Every CTA has the block size of
// the largest configuration; smaller configurations leave the surplus threads
// idle but still meet every barrier.  Pixels whose minimum is not certified
// are appended to one batch-wide recheck list, keyed by batch pixel offset,
// and a second persistent kernel re-evaluates them in FP64 (one warp each).
// No device-side wait exists: the work counter is only ever incremented.
#include <cuda_runtime.h>
#include <stdint.h>

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
    int tile_base;   // first work item of this image
    int pix_base;    // first batch pixel offset of this image
    int cfg;         // ((win/2 - 1) * 2 + filter) * kNumShapes32 + shape
    double p;
};

struct BatchParams {
    const BatchDesc *desc;
    int count;
    int total_tiles;
    unsigned *ctr;   // [0] recheck count, [1] overflow, [2] next work item
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

template <int... I>
constexpr size_t max_smem(std::integer_sequence<int, I...>)
{
    size_t m = 0;
    ((m = BCfg<I>::C::SMEM > m ? BCfg<I>::C::SMEM : m), ...);
    return m;
}
template <int... I>
constexpr int max_threads(std::integer_sequence<int, I...>)
{
    int m = 0;
    ((m = BCfg<I>::C::NT > m ? BCfg<I>::C::NT : m), ...);
    return m;
}
constexpr size_t kBatchSmem = max_smem(std::make_integer_sequence<int, kNumCfgs>{});
constexpr int kBatchThreads = max_threads(std::make_integer_sequence<int, kNumCfgs>{});

// One configuration's tile body as a call of its own: each body gets its own
// register allocation instead of the union of all twelve.
template <int CFG>
__device__ __noinline__ void run_item(const TileParams prm, int t, int tiles_x)
{
    using C = typename BCfg<CFG>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    tile_body<C, kBatchThreads>(prm, 0, (t % tiles_x) * C::TW, (t / tiles_x) * C::TH, smem);
}

template <int... I>
__device__ __forceinline__ void dispatch_item(int cfg, const TileParams &prm, int t, int tiles_x, unsigned char *smem,
                                              std::integer_sequence<int, I...>)
{
    ((cfg == I ? run_item<I>(prm, t, tiles_x) : void()), ...);
}

__global__ void __launch_bounds__(kBatchThreads, 1) batch_kernel(const BatchParams bp)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(bp.ctr + 2, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= bp.total_tiles) break;
        int lo = 0, hi = bp.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp.desc[mid].tile_base <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchDesc d = bp.desc[lo];
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
        dispatch_item(d.cfg, prm, item - d.tile_base, d.tiles_x, smem, std::make_integer_sequence<int, kNumCfgs>{});
        __syncthreads();   // the next item reuses shared memory and s_item
    }
}

// Per-warp shared memory of the largest recheck configuration.
constexpr size_t kRecheckPerWarp = RecheckCfg<2, DDF, EXACT>::PER_WARP;
constexpr int kRecheckWarps = 4;

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

constexpr size_t kCtrBytes = 256;

size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }

}  // namespace

}  // namespace vdf

struct vdf_plan {
    std::vector<vdf::BatchDesc> desc;
    int total_tiles = 0;
    long long total_pixels = 0;
    int q = 4;
    int sms = 1;
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

size_t plan_ws_bytes(const vdf_plan *plan)
{
    return vdf::kCtrBytes + vdf::up16(sizeof(vdf::BatchDesc) * plan->desc.size()) +
           sizeof(int2) * (size_t)plan->total_pixels;
}

vdf::BatchParams plan_params(const vdf_plan *plan, void *ws)
{
    vdf::BatchParams bp{};
    char *base = (char *)ws;
    bp.ctr = (unsigned *)base;
    bp.desc = (const vdf::BatchDesc *)(base + vdf::kCtrBytes);
    bp.list = (int2 *)(base + vdf::kCtrBytes + vdf::up16(sizeof(vdf::BatchDesc) * plan->desc.size()));
    bp.count = (int)plan->desc.size();
    bp.total_tiles = plan->total_tiles;
    bp.cap = (unsigned)plan->total_pixels;
    bp.q = plan->q;
    return bp;
}

int set_attributes()
{
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(vdf::batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)vdf::kBatchSmem);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(vdf::batch_recheck_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(vdf::kRecheckPerWarp * vdf::kRecheckWarps));
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
    long long tiles = 0, pixels = 0;
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
        const int tw = vdf::kShapes32[shape].tw, th = vdf::kShapes32[shape].th;
        vdf::BatchDesc bd{};
        bd.img = d.img;
        bd.out = d.out;
        bd.idx = d.index_out;
        bd.M = d.M;
        bd.N = d.N;
        bd.tiles_x = (d.N + tw - 1) / tw;
        bd.tile_base = (int)tiles;
        bd.pix_base = (int)pixels;
        bd.cfg = ((d.win / 2 - 1) * 2 + d.filter) * vdf::kNumShapes32 + shape;
        bd.p = d.p;
        tiles += (long long)bd.tiles_x * ((d.M + th - 1) / th);
        pixels += (long long)d.M * d.N;
        if (tiles > (1LL << 31) - 1 || pixels > (1LL << 31) - 1) {
            delete pl;
            return VDF_E_INVALID;
        }
        pl->desc.push_back(bd);
    }
    pl->total_tiles = (int)tiles;
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
    const vdf::BatchParams bp = plan_params(plan, workspace);
    const int sms = plan->sms;
    cudaError_t e = cudaMemsetAsync(bp.ctr, 0, 4 * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        vdf::batch_kernel<<<sms, vdf::kBatchThreads, vdf::kBatchSmem, st>>>(bp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        vdf::batch_recheck_kernel<<<sms * 4, 32 * vdf::kRecheckWarps, vdf::kRecheckPerWarp * vdf::kRecheckWarps, st>>>(
            bp);
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

void vdf_plan_destroy(vdf_plan *plan)
{
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    delete plan;
}

}  // extern "C"
