// vdf_frames.cu -- vdf_filter_host_frames: a sequence of host frames through
// the filter, with the copies of each frame overlapping the filtering of its
// neighbours.
//
// Three device slots hold one frame each (input, output, index map and the
// filter's workspace).  Four library-owned streams per device carry the
// stages: host-to-device copy, FP32 pass (or the whole FP64 filter), FP64
// recheck, device-to-host copy.  Frame i uses slot i % 3; its upload waits
// until the download of frame i - 3 (same slot) has finished, and every
// later stage waits for the one before it (events).  So the upload of frame
// i + 1 and the download of frame i - 1 run while frame i is filtered, and
// the recheck of frame i runs beside the FP32 passes of frames i + 1 and
// i + 2 (with two slots the pass of frame i + 2 would wait for it).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/vdf.h"

namespace {

constexpr int kSlots = 3;
constexpr int kMaxDevices = 64;

struct Lanes {
    cudaStream_t up = nullptr, pass = nullptr, recheck = nullptr, down = nullptr;
    cudaEvent_t start = nullptr, fin = nullptr;
    cudaEvent_t loaded[kSlots] = {}, passed[kSlots] = {}, filtered[kSlots] = {}, freed[kSlots] = {};
    bool ready = false;
};

std::mutex g_mutex[kMaxDevices];
Lanes g_lanes[kMaxDevices];

// Streams and events of one device, created on first use and kept until the
// process exits.  Called with the device's mutex held.
cudaError_t lanes_of(int dev, Lanes **out)
{
    Lanes &L = g_lanes[dev];
    if (!L.ready) {
        cudaError_t e = cudaSuccess;
        for (cudaStream_t *s : {&L.up, &L.pass, &L.recheck, &L.down})
            if (e == cudaSuccess && !*s) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
        for (cudaEvent_t *ev : {&L.start, &L.fin})
            if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k)
            for (cudaEvent_t *ev : {&L.loaded[k], &L.passed[k], &L.filtered[k], &L.freed[k]})
                if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        L.ready = true;
    }
    *out = &L;
    return cudaSuccess;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? VDF_OK : VDF_E_CUDA; }

// One slot: vdf_host_buffer_bytes rounded up to 256 bytes, so that every
// slot (and the workspace inside it) keeps the buffer's alignment.
size_t slot_bytes(int M, int N, int precision) { return (vdf_host_buffer_bytes(M, N, precision) + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

size_t vdf_host_frames_buffer_bytes(int M, int N, int precision) { return kSlots * slot_bytes(M, N, precision); }

int vdf_filter_host_frames(const uint8_t *const *img_host, uint8_t *const *out_host, int8_t *const *index_out_host,
                           int count, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
                           int precision, void *dev_buffer, size_t dev_buffer_bytes, void *stream)
{
    if (count < 0 || M < 1 || N < 1 || (count > 0 && (!img_host || !out_host || !dev_buffer))) return VDF_E_INVALID;
    for (int i = 0; i < count; ++i)
        if (!img_host[i] || !out_host[i]) return VDF_E_INVALID;
    const size_t slot = slot_bytes(M, N, precision);
    if (slot == 0) return VDF_E_INVALID;
    if (count == 0) return VDF_OK;
    if (dev_buffer_bytes < kSlots * slot || ((uintptr_t)dev_buffer & 255)) return VDF_E_WORKSPACE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VDF_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex[dev]);
    Lanes *L = nullptr;
    if (lanes_of(dev, &L) != cudaSuccess) return VDF_E_CUDA;

    const size_t px = (size_t)M * N;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const bool fp32 = precision == VDF_PREC_FP32_RECHECK;
    const size_t ws_bytes = vdf_workspace_bytes(M, N, precision);
    cudaStream_t user = (cudaStream_t)stream;

    // everything starts after the work already queued on the caller's stream
    cudaError_t e = cudaEventRecord(L->start, user);
    for (cudaStream_t s : {L->up, L->pass, L->recheck, L->down})
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, L->start, 0);
    int rc = status_of(e);

    for (int i = 0; i < count && rc == VDF_OK; ++i) {
        const int k = i % kSlots;
        uint8_t *d_in = (uint8_t *)dev_buffer + k * slot;
        uint8_t *d_out = d_in + up(3 * px);
        int8_t *d_idx = (int8_t *)(d_out + up(3 * px));
        void *ws = (char *)d_idx + up(px);
        int8_t *idx_host = index_out_host ? index_out_host[i] : nullptr;
        int8_t *idx_dev = idx_host ? d_idx : nullptr;

        if (i >= kSlots) e = cudaStreamWaitEvent(L->up, L->freed[k], 0);   // frame i - 3 is downloaded
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_in, img_host[i], 3 * px, cudaMemcpyHostToDevice, L->up);
        if (e == cudaSuccess) e = cudaEventRecord(L->loaded[k], L->up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(L->pass, L->loaded[k], 0);
        if ((rc = status_of(e)) != VDF_OK) break;
        if (fp32) {
            rc = vdf_fp32_pass(d_in, M, N, win, filter, p, dist_mode, minimax_q, d_out, idx_dev, ws, ws_bytes,
                               L->pass);
            if (rc != VDF_OK) break;
            e = cudaEventRecord(L->passed[k], L->pass);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(L->recheck, L->passed[k], 0);
            if ((rc = status_of(e)) != VDF_OK) break;
            rc = vdf_fp64_recheck(d_in, M, N, win, filter, p, dist_mode, minimax_q, d_out, idx_dev, ws, ws_bytes,
                                  L->recheck);
            if (rc != VDF_OK) break;
            e = cudaEventRecord(L->filtered[k], L->recheck);
        } else {
            rc = vdf_filter(d_in, M, N, win, filter, p, dist_mode, minimax_q, precision, d_out, idx_dev, nullptr,
                            ws, ws_bytes, L->pass);
            if (rc != VDF_OK) break;
            e = cudaEventRecord(L->filtered[k], L->pass);
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(L->down, L->filtered[k], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_host[i], d_out, 3 * px, cudaMemcpyDeviceToHost, L->down);
        if (e == cudaSuccess && idx_host) e = cudaMemcpyAsync(idx_host, d_idx, px, cudaMemcpyDeviceToHost, L->down);
        if (e == cudaSuccess) e = cudaEventRecord(L->freed[k], L->down);
        rc = status_of(e);
    }

    // the caller's stream continues after the last download; the call
    // returns once every stage has finished (also after an error, so that no
    // copy is still using the caller's buffers)
    cudaError_t f = cudaSuccess;
    for (cudaStream_t s : {L->up, L->pass, L->recheck})
        if (f == cudaSuccess && (f = cudaEventRecord(L->fin, s)) == cudaSuccess) f = cudaStreamWaitEvent(L->down, L->fin, 0);
    if (f == cudaSuccess) f = cudaEventRecord(L->fin, L->down);
    if (f == cudaSuccess) f = cudaStreamWaitEvent(user, L->fin, 0);
    if (f == cudaSuccess) f = cudaEventSynchronize(L->fin);
    if (rc == VDF_OK) rc = status_of(f);
    return rc;
}

}  // extern "C"
