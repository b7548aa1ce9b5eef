// vdf_noalloc.cu -- vdf_filter_noalloc: the FP32 certified path without any
// caller-provided scratch.
//
// vdf_filter's FP32 path needs device scratch beyond its inputs and outputs:
// two counters and the list of pixels to re-evaluate in FP64 (one 8-byte
// entry per pixel).  Normally the caller allocates it (vdf_workspace_bytes).  Some
// callers cannot: code that runs where cudaMalloc is forbidden or unsafe
// after start-up (real-time loops that must not block on the allocator or
// synchronise the device), plug-ins whose host owns all device memory and
// hands out only the image buffers, and wrappers that cannot keep a
// workspace alive between calls.  This entry point serves them: its scratch
// is a file-scope device array of fixed size, so it allocates nothing.
//
// Limits and behaviour:
//   - capacity kMaxPixels = 2^21 = 2,097,152 pixels (enough for 1920 x 1080);
//     larger images are rejected with VDF_E_WORKSPACE before any launch;
//   - the array (256 bytes + 16 MiB) is held on every GPU that loads the
//     library, until the process exits;
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress, which may load this library's device code);
//     make that first call before any stream capture.  The address is kept
//     per device for the life of the process: after cudaDeviceReset the
//     kept address belongs to the destroyed context, so this entry point
//     must not be used on that device again;
//   - every call shares the one array and each call clears the counters it
//     needs; calls that overlap on the GPU (different streams, or different
//     host threads without ordering) race on it and must be serialised.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/vdf.h"
#include "vdf_dispatch.h"

namespace {

constexpr size_t kMaxPixels = (size_t)1 << 21;
constexpr size_t kCtrBytes = 256;   // counters, padded like the caller workspace
constexpr size_t kScratchBytes = kCtrBytes + sizeof(int2) * kMaxPixels;   // one {pixel, mask} per pixel
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per
// device; in host code the name g_scratch is only a host-side stand-in).
int scratch_address(void **addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VDF_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return VDF_E_CUDA;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return VDF_OK;
}

}  // namespace

extern "C" int vdf_filter_noalloc(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                                  int minimax_q, uint8_t *out, int8_t *index_out, void *stream)
{
    // every argument check of vdf_filter first, then the capacity
    int rc = vdf::check_args_no_workspace(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out);
    if (rc != VDF_OK) return rc;
    if ((size_t)M * (size_t)N > kMaxPixels) return VDF_E_WORKSPACE;
    void *ws = nullptr;
    rc = scratch_address(&ws);
    if (rc != VDF_OK) return rc;
    rc = vdf_fp32_pass(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, ws, kScratchBytes, stream);
    if (rc != VDF_OK) return rc;
    return vdf_fp64_recheck(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, ws, kScratchBytes,
                            stream);
}
