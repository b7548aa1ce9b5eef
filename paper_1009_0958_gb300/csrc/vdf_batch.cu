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
#include "vdf_batch_kernels.cuh"

namespace vdf {

namespace {

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
    int dist = 0;   // distance mode of every image of the plan
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

// the shared-memory opt-in of the plan's distance mode, once per device
int set_attributes(int dist)
{
    static std::atomic<bool> done[3][vdf::kMaxDevices];
    cudaError_t err = cudaErrorInvalidValue;
    switch (dist) {
    case vdf::EXACT: err = vdf::once_per_device(done[0], [] { return vdf::BatchOps<vdf::EXACT>::configure(); }); break;
    case vdf::MINIMAX:
        err = vdf::once_per_device(done[1], [] { return vdf::BatchOps<vdf::MINIMAX>::configure(); });
        break;
    case vdf::RGB: err = vdf::once_per_device(done[2], [] { return vdf::BatchOps<vdf::RGB>::configure(); }); break;
    }
    return err == cudaSuccess ? VDF_OK : VDF_E_CUDA;
}

cudaError_t launch_group(int dist, int cfg, const vdf::BatchParams &bp, int sms, cudaStream_t st, bool persistent)
{
    switch (dist) {
    case vdf::EXACT: return vdf::BatchOps<vdf::EXACT>::launch(cfg, bp, sms, st, persistent);
    case vdf::MINIMAX: return vdf::BatchOps<vdf::MINIMAX>::launch(cfg, bp, sms, st, persistent);
    case vdf::RGB: return vdf::BatchOps<vdf::RGB>::launch(cfg, bp, sms, st, persistent);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_recheck(int dist, const vdf::BatchParams &bp, int blocks, cudaStream_t st)
{
    switch (dist) {
    case vdf::EXACT: return vdf::BatchOps<vdf::EXACT>::recheck(bp, blocks, st);
    case vdf::MINIMAX: return vdf::BatchOps<vdf::MINIMAX>::recheck(bp, blocks, st);
    case vdf::RGB: return vdf::BatchOps<vdf::RGB>::recheck(bp, blocks, st);
    }
    return cudaErrorInvalidValue;
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
    if (dist_mode < VDF_DIST_EXACT || dist_mode > VDF_DIST_RGB) return VDF_E_INVALID;
    if (dist_mode == VDF_DIST_MINIMAX && (minimax_q < 2 || minimax_q > 4)) return VDF_E_INVALID;
    vdf_plan *pl = new (std::nothrow) vdf_plan;
    if (!pl) return VDF_E_INVALID;
    pl->q = minimax_q;
    pl->dist = dist_mode;
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
        const int shape = vdf::tuned_shape_p(d.win, d.filter, dist_mode, d.p);
        vdf::BatchDesc bd{};
        bd.img = d.img;
        bd.out = d.out;
        bd.idx = d.index_out;
        bd.M = d.M;
        bd.N = d.N;
        bd.tiles_x = (d.N + vdf::kShapes32[shape].tw - 1) / vdf::kShapes32[shape].tw;
        bd.cfg = ((d.win / 2 - 1) * 2 + d.filter) * vdf::kNumShapes32 + shape;
        // DDF 5x5 at p = 1/4 (exact or chromaticity terms): the score-slot kernels
        if (const int a = vdf::score_slot_exponent(d.win / 2, d.filter, dist_mode, vdf::NL2, d.p))
            bd.cfg = vdf::kScoreCfg0 + (a - 1) * vdf::kNumShapes32 + shape;
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
    int rc = set_attributes(plan->dist);
    if (rc != VDF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = plan->sms;
    const int ngroups = (int)plan->groups.size();
    cudaError_t e = cudaMemsetAsync(workspace, 0, vdf::kCtrBytes, st);
    for (int g = 0; g < ngroups && e == cudaSuccess; ++g)
        e = launch_group(plan->dist, plan->groups[g].cfg, plan_params(plan, workspace, g), sms, st,
                         plan->persistent.load());
    if (e == cudaSuccess) e = launch_recheck(plan->dist, plan_params(plan, workspace, -1), sms * 16, st);
    return e == cudaSuccess ? VDF_OK : VDF_E_CUDA;
}

int vdf_plan_graph_launch(vdf_plan *plan, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!plan) return VDF_E_INVALID;
    if (!ws_ok(plan, workspace, workspace_bytes)) return VDF_E_WORKSPACE;
    int rc = set_attributes(plan->dist);
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
