// vdf_api.cu -- the C ABI of libvdf (declared in include/vdf.h): argument
// checks, workspace layout and the launch sequence of each call.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <mutex>

#include "../../include/vdf.h"
#include "vdf_dispatch.h"
#include "vdf_win7.cuh"

namespace {

thread_local char g_last_cuda[256] = "no error";

int cuda_fail(cudaError_t e)
{
    if (e == cudaSuccess) return VDF_OK;
    strncpy(g_last_cuda, cudaGetErrorString(e), sizeof(g_last_cuda) - 1);
    g_last_cuda[sizeof(g_last_cuda) - 1] = 0;
    return VDF_E_CUDA;
}

// Workspace of the FP32 path: two counters, padding to 256 bytes, then one
// {pixel id, member mask} int2 entry per pixel (the recheck list can never
// overflow).
constexpr size_t kCtrBytes = vdf::kCounterBlockBytes;

bool valid_common(int M, int N, int win, int filter, double p, int dist, int q, int prec)
{
    if (M < 1 || N < 1 || (long long)M * N > (1LL << 31) - 1) return false;
    if (win != 3 && win != 5 && win != 7) return false;
    if (filter != VDF_BVDF && filter != VDF_DDF && filter != VDF_VMF) return false;
    if (filter == VDF_DDF && !(p >= 0.0 && p <= 1.0)) return false;
    if (dist < VDF_DIST_EXACT || dist > VDF_DIST_RGB) return false;
    if (dist == VDF_DIST_MINIMAX && (q < 2 || q > 4)) return false;
    if (prec != VDF_PREC_FP64 && prec != VDF_PREC_FP32_RECHECK) return false;
    return true;
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

// SM count of the current device (looked up once per device)
int num_sms()
{
    static std::atomic<int> sms[vdf::kMaxDevices];
    const int dev = vdf::current_device();
    if (dev < 0) return 1;
    int n = sms[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
        sms[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Blocks of the FP64 recheck kernel: consecutive list entries go to
// different SMs, whose FP64 pipes bound the recheck.
int recheck_blocks() { return num_sms() * 16; }

// Tile shape of the FP32 kernel per (window, filter, distance mode, slot
// kind): shape 0 until vdf_autotune or vdf_set_tuned_shape records another.
// Kinds 1..3 are the score-slot kernels (DDF 5x5 at p = kind / 4), whose
// best shape differs from the raw-slot kernels' of the same configuration;
// kind 4 is the ACWDDF's kernel (its DDF entry).
constexpr int kSlotKinds = 5, kAcwKind = 4;
std::mutex g_tune_mutex;
int g_tuned[2][3][3][kSlotKinds] = {};

int tuned_shape(int win, int filter, int dist, int kind = 0)
{
    if (win != 3 && win != 5) return 0;   // the 7x7 window has no tile shapes
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    return g_tuned[win / 2 - 1][filter][dist][kind];
}

int slot_kind(int win, int filter, int dist, int norm, double p)
{
    return vdf::score_slot_exponent(win / 2, filter, dist, norm, p);
}

void record_tuned_shape(int win, int filter, int dist, int kind, int shape)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[win / 2 - 1][filter][dist][kind] = shape;
}

// Kernel dispatch by filter kind and Minkowski order (internal code): the
// VMF and the orders 1 / infinity have their own instantiation units.
cudaError_t run_tile32(const vdf::TileParams &prm, int R, int filter, int dist, int norm, int shape, cudaStream_t st)
{
    if (filter == VDF_VMF || norm != vdf::NL2) return vdf::run_fp32_lp(prm, R, filter, norm, shape, st);
    return vdf::run_fp32(prm, R, filter, dist, shape, st);
}

cudaError_t run_tile64(const vdf::TileParams &prm, int R, int filter, int dist, int norm, cudaStream_t st)
{
    if (filter == VDF_VMF || norm != vdf::NL2) return vdf::run_fp64_lp(prm, R, filter, norm, st);
    return vdf::run_fp64(prm, R, filter, dist, false, st);
}

cudaError_t run_recheck_any(const vdf::RecheckParams &rp, int R, int filter, int dist, int norm, int blocks,
                            cudaStream_t st)
{
    if (filter == VDF_VMF || norm != vdf::NL2) return vdf::run_recheck_lp(rp, R, filter, norm, blocks, st);
    return vdf::run_recheck(rp, R, filter, dist, blocks, st);
}

}  // namespace

extern "C" {

const char *vdf_strerror(int status)
{
    switch (status) {
    case VDF_OK: return "ok";
    case VDF_E_INVALID: return "invalid argument";
    case VDF_E_CUDA: return "CUDA error";
    case VDF_E_OVERFLOW: return "recheck list overflow";
    case VDF_E_TIMEOUT: return "device-side wait timed out";
    case VDF_E_WORKSPACE: return "workspace missing or too small";
    case VDF_E_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

const char *vdf_last_cuda_error(void) { return g_last_cuda; }

size_t vdf_workspace_bytes(int M, int N, int precision)
{
    if (M < 1 || N < 1) return 0;
    if (precision != VDF_PREC_FP32_RECHECK) return 0;
    return kCtrBytes + sizeof(int2) * (size_t)M * (size_t)N;
}

static int check_filter_args(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                             int minimax_q, int precision, const uint8_t *out, const int8_t *index_out,
                             const double *agg_out, const void *workspace, size_t workspace_bytes)
{
    if (!img || !out || !valid_common(M, N, win, filter, p, dist_mode, minimax_q, precision)) return VDF_E_INVALID;
    const size_t bytes = (size_t)M * N * 3;
    if (overlaps(img, bytes, out, bytes)) return VDF_E_INVALID;
    if (index_out && (overlaps(index_out, (size_t)M * N, img, bytes) || overlaps(index_out, (size_t)M * N, out, bytes)))
        return VDF_E_INVALID;
    if (agg_out && precision != VDF_PREC_FP64) return VDF_E_INVALID;
    const size_t need = vdf_workspace_bytes(M, N, precision);
    if (need && (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255))) return VDF_E_WORKSPACE;
    return VDF_OK;
}

}  // extern "C"

// Argument checks of the FP32 path without its workspace (vdf_filter_noalloc
// supplies its own scratch); dispatch-internal, declared in vdf_dispatch.h.
int vdf::check_args_no_workspace(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                                 int minimax_q, const uint8_t *out, const int8_t *index_out)
{
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;
    if (!valid_common(M, N, win, filter, p, dist_mode, minimax_q, VDF_PREC_FP32_RECHECK)) return VDF_E_INVALID;
    return check_filter_args(img, M, N, win, filter, p, dist_mode, minimax_q, VDF_PREC_FP64, out, index_out, nullptr,
                             nullptr, 0);
}

// The FP32 ACWDDF in one tile shape: counter reset, tile kernel, FP64
// recheck of the listed pixels (arguments already checked).
static cudaError_t acw_pass_shape(const vdf::TileParams &prm, const uint8_t *img, int M, int N, int win,
                                  int dist_mode, int minimax_q, int lambda, double T, int shape, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(prm.recheck_ctr, 0, vdf::kCounterBlockBytes, st);
    if (e == cudaSuccess) e = vdf::run_fp32_acw(prm, win / 2, dist_mode, shape, st);
    if (e == cudaSuccess) {
        vdf::RecheckParams rp{};
        rp.img = img;
        rp.out = prm.out;
        rp.idx = prm.idx;
        rp.list = prm.recheck_list;
        rp.ctr = prm.recheck_ctr;
        rp.cap = prm.recheck_cap;
        rp.M = M;
        rp.N = N;
        rp.p = 0.5;
        rp.q = minimax_q;
        rp.lam = lambda;
        rp.T = T;
        e = vdf::run_recheck_acw(rp, win / 2, dist_mode, recheck_blocks(), st);
    }
    return e;
}

extern "C" {

static vdf::TileParams tile_params(const uint8_t *img, int M, int N, double p, int q, uint8_t *out, int8_t *idx,
                                   double *agg, void *workspace)
{
    vdf::TileParams prm{};
    prm.img = img;
    prm.out = out;
    prm.idx = idx;
    prm.agg = agg;
    prm.M = M;
    prm.N = N;
    prm.B = 1;
    prm.p = p;
    prm.q = q;
    if (workspace) {
        prm.recheck_ctr = (unsigned *)workspace;
        prm.recheck_list = (int2 *)((char *)workspace + kCtrBytes);
        prm.recheck_cap = (unsigned)((size_t)M * N);
    }
    return prm;
}

static int fp32_pass_shape(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                           int minimax_q, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes,
                           int shape, void *stream, int norm = vdf::NL2)
{
    int rc = check_filter_args(img, M, N, win, filter, p, dist_mode, minimax_q, VDF_PREC_FP32_RECHECK, out,
                               index_out, nullptr, workspace, workspace_bytes);
    if (rc != VDF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const vdf::TileParams prm = tile_params(img, M, N, p, minimax_q, out, index_out, nullptr, workspace);
    cudaError_t e = cudaMemsetAsync(prm.recheck_ctr, 0, vdf::kCounterBlockBytes, st);
    if (e == cudaSuccess && win == 7) {
        vdf::Win7Params wp{};
        wp.img = img;
        wp.out = out;
        wp.idx = index_out;
        wp.list = prm.recheck_list;
        wp.ctr = prm.recheck_ctr;
        wp.cap = prm.recheck_cap;
        wp.M = M;
        wp.N = N;
        wp.p = p;
        wp.q = minimax_q;
        e = vdf::run_win7_fp32(wp, filter, dist_mode, norm, num_sms(), st);
    } else if (e == cudaSuccess) {
        e = run_tile32(prm, win / 2, filter, dist_mode, norm, shape, st);
    }
    return cuda_fail(e);
}

static int fp32_pass_norm(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                          int minimax_q, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes,
                          void *stream, int norm)
{
    if (!valid_common(M, N, win, filter, p, dist_mode, minimax_q, VDF_PREC_FP32_RECHECK)) return VDF_E_INVALID;
    const int shape = tuned_shape(win, filter, dist_mode, slot_kind(win, filter, dist_mode, norm, p));
    return fp32_pass_shape(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace,
                           workspace_bytes, shape, stream, norm);
}

static int fp64_recheck_norm(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                             int minimax_q, uint8_t *out, int8_t *index_out, void *workspace,
                             size_t workspace_bytes, void *stream, int norm)
{
    int rc = check_filter_args(img, M, N, win, filter, p, dist_mode, minimax_q, VDF_PREC_FP32_RECHECK, out,
                               index_out, nullptr, workspace, workspace_bytes);
    if (rc != VDF_OK) return rc;
    vdf::RecheckParams rp{};
    rp.img = img;
    rp.out = out;
    rp.idx = index_out;
    rp.list = (const int2 *)((const char *)workspace + kCtrBytes);
    rp.ctr = (const unsigned *)workspace;
    rp.cap = (unsigned)((size_t)M * N);
    rp.M = M;
    rp.N = N;
    rp.p = p;
    rp.q = minimax_q;
    if (win == 7)
        return cuda_fail(vdf::run_win7_recheck(rp, filter, dist_mode, norm, recheck_blocks(), (cudaStream_t)stream));
    return cuda_fail(run_recheck_any(rp, win / 2, filter, dist_mode, norm, recheck_blocks(), (cudaStream_t)stream));
}

int vdf_fp32_pass(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
                  uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes, void *stream)
{
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;
    return fp32_pass_norm(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace,
                          workspace_bytes, stream, vdf::NL2);
}

int vdf_fp64_recheck(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                     int minimax_q, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes,
                     void *stream)
{
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;
    return fp64_recheck_norm(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace,
                             workspace_bytes, stream, vdf::NL2);
}

int vdf_filter_lp(const uint8_t *img, int M, int N, int win, int filter, double p, int minkowski_order,
                  int dist_mode, int minimax_q, int precision, uint8_t *out, int8_t *index_out, double *agg_out,
                  void *workspace, size_t workspace_bytes, void *stream)
{
    int norm;
    switch (minkowski_order) {
    case 2: norm = vdf::NL2; break;
    case 1: norm = vdf::NL1; break;
    case VDF_MINKOWSKI_INF: norm = vdf::NLINF; break;
    default: return VDF_E_INVALID;
    }
    if (filter == VDF_BVDF) norm = vdf::NL2;               // no distance term
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;     // no angular term
    int rc = check_filter_args(img, M, N, win, filter, p, dist_mode, minimax_q, precision, out, index_out, agg_out,
                               workspace, workspace_bytes);
    if (rc != VDF_OK) return rc;
    if (filter == VDF_DDF && norm != vdf::NL2 && dist_mode != VDF_DIST_EXACT) return VDF_E_UNSUPPORTED;
    if (precision == VDF_PREC_FP64 && win == 7) {
        vdf::RecheckParams rp{};
        rp.img = img;
        rp.out = out;
        rp.idx = index_out;
        rp.M = M;
        rp.N = N;
        rp.p = p;
        rp.q = minimax_q;
        return cuda_fail(vdf::run_win7_fp64(rp, agg_out, filter, dist_mode, norm, num_sms(), (cudaStream_t)stream));
    }
    if (precision == VDF_PREC_FP64) {
        const vdf::TileParams prm = tile_params(img, M, N, p, minimax_q, out, index_out, agg_out, nullptr);
        return cuda_fail(run_tile64(prm, win / 2, filter, dist_mode, norm, (cudaStream_t)stream));
    }
    rc = fp32_pass_norm(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace, workspace_bytes,
                        stream, norm);
    if (rc != VDF_OK) return rc;
    return fp64_recheck_norm(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace,
                             workspace_bytes, stream, norm);
}

int vdf_filter_acwddf(const uint8_t *img, int M, int N, int win, int dist_mode, int minimax_q, int lambda, double T,
                      int precision, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes,
                      void *stream)
{
    int rc = check_filter_args(img, M, N, win, VDF_DDF, 0.5, dist_mode, minimax_q, precision, out, index_out,
                               nullptr, workspace, workspace_bytes);
    if (rc != VDF_OK) return rc;
    if (win == 7) return VDF_E_UNSUPPORTED;
    const int d1 = (win * win + 1) / 2;   // 1-based centre index: levels lambda .. lambda+2 must stay <= d
    if (lambda < 1 || lambda > d1 - 2 || !std::isfinite(T)) return VDF_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    vdf::TileParams prm = tile_params(img, M, N, 0.5, minimax_q, out, index_out, nullptr,
                                      precision == VDF_PREC_FP64 ? nullptr : workspace);
    prm.lam = lambda;
    prm.T = T;
    if (precision == VDF_PREC_FP64) return cuda_fail(vdf::run_fp64_acw(prm, win / 2, dist_mode, st));
    return cuda_fail(acw_pass_shape(prm, img, M, N, win, dist_mode, minimax_q, lambda, T,
                                    tuned_shape(win, VDF_DDF, dist_mode, kAcwKind), st));
}


int vdf_filter(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
               int precision, uint8_t *out, int8_t *index_out, double *agg_out, void *workspace,
               size_t workspace_bytes, void *stream)
{
    return vdf_filter_lp(img, M, N, win, filter, p, 2, dist_mode, minimax_q, precision, out, index_out, agg_out,
                         workspace, workspace_bytes, stream);
}

int vdf_workspace_stats(const void *workspace, int64_t *rechecked, int32_t *overflow, void *stream)
{
    if (!workspace) return VDF_E_INVALID;
    unsigned h[2] = {0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (rechecked) *rechecked = h[0];
    if (overflow) *overflow = (int32_t)h[1];
    return VDF_OK;
}

int vdf_read_stats(const void *workspace, vdf_stats *stats, void *stream)
{
    if (!workspace || !stats) return VDF_E_INVALID;
    unsigned h[vdf::kCounterBlockBytes / sizeof(unsigned)] = {};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    stats->rechecked = h[0];
    stats->overflow = (int32_t)h[1];
    stats->structural_ties = h[vdf::kTieCounter];
    return VDF_OK;
}

size_t vdf_host_buffer_bytes(int M, int N, int precision)
{
    if (M < 1 || N < 1) return 0;
    const size_t px = (size_t)M * N;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return up(3 * px) + up(3 * px) + up(px) + vdf_workspace_bytes(M, N, precision);
}

int vdf_filter_host(const uint8_t *img_host, int M, int N, int win, int filter, double p, int dist_mode,
                    int minimax_q, int precision, uint8_t *out_host, int8_t *index_out_host, void *dev_buffer,
                    size_t dev_buffer_bytes, void *stream)
{
    if (!img_host || !out_host || !dev_buffer || M < 1 || N < 1) return VDF_E_INVALID;
    const size_t need = vdf_host_buffer_bytes(M, N, precision);
    if (dev_buffer_bytes < need || ((uintptr_t)dev_buffer & 255)) return VDF_E_WORKSPACE;
    const size_t px = (size_t)M * N;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    uint8_t *d_in = (uint8_t *)dev_buffer;
    uint8_t *d_out = d_in + up(3 * px);
    int8_t *d_idx = (int8_t *)(d_out + up(3 * px));
    void *ws = (char *)d_idx + up(px);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_in, img_host, 3 * px, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = vdf_filter(d_in, M, N, win, filter, p, dist_mode, minimax_q, precision, d_out,
                        index_out_host ? d_idx : nullptr, nullptr, ws, vdf_workspace_bytes(M, N, precision), stream);
    if (rc != VDF_OK) return rc;
    e = cudaMemcpyAsync(out_host, d_out, 3 * px, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && index_out_host) e = cudaMemcpyAsync(index_out_host, d_idx, px, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_fail(e);
}

int vdf_filter_f32(const float *img, int B, int M, int N, int win, int filter, double p, int dist_mode,
                   int minimax_q, int precision, float *out, int8_t *index_out, void *workspace,
                   size_t workspace_bytes, void *stream)
{
    if (!img || !out || B < 1 || B > 65535 || !valid_common(M, N, win, filter, p, dist_mode, minimax_q, precision))
        return VDF_E_INVALID;
    if ((long long)B * M * N > (1LL << 31) - 1) return VDF_E_INVALID;
    const size_t bytes = (size_t)B * M * N * 3 * sizeof(float);
    if (overlaps(img, bytes, out, bytes)) return VDF_E_INVALID;
    if (dist_mode != VDF_DIST_EXACT || filter == VDF_VMF || win == 7) return VDF_E_UNSUPPORTED;
    if (index_out && (overlaps(index_out, (size_t)B * M * N, img, bytes) || overlaps(index_out, (size_t)B * M * N, out, bytes)))
        return VDF_E_INVALID;
    vdf::TileParams prm{};
    prm.img = img;
    prm.out = out;
    prm.idx = index_out;
    prm.M = M;
    prm.N = N;
    prm.B = B;
    prm.p = p;
    prm.q = minimax_q;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == VDF_PREC_FP64) return cuda_fail(vdf::run_fp64(prm, win / 2, filter, dist_mode, true, st));
    // FP32 certified pass over the batch, then the FP64 recheck of the listed
    // pixels (batch pixel ids); the workspace is sized for B * M rows of N
    const size_t need = vdf_workspace_bytes(B * M, N, precision);
    if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) return VDF_E_WORKSPACE;
    prm.recheck_ctr = (unsigned *)workspace;
    prm.recheck_list = (int2 *)((char *)workspace + kCtrBytes);
    prm.recheck_cap = (unsigned)((size_t)B * M * N);
    cudaError_t e = cudaMemsetAsync(prm.recheck_ctr, 0, vdf::kCounterBlockBytes, st);
    if (e == cudaSuccess) e = vdf::run_fp32_f32in(prm, win / 2, filter, st);
    if (e == cudaSuccess) {
        vdf::RecheckParams rp{};
        rp.img = img;
        rp.out = out;
        rp.idx = index_out;
        rp.list = prm.recheck_list;
        rp.ctr = prm.recheck_ctr;
        rp.cap = prm.recheck_cap;
        rp.M = M;
        rp.N = N;
        rp.p = p;
        rp.q = minimax_q;
        e = vdf::run_recheck(rp, win / 2, filter, dist_mode, recheck_blocks(), st, true);
    }
    return cuda_fail(e);
}

int vdf_backward_f32(const float *grad_y, const int8_t *index, int B, int M, int N, int win, float *grad_x,
                     void *stream)
{
    if (!grad_y || !index || !grad_x || B < 1 || B > 65535 || M < 1 || M > 65535 || N < 1) return VDF_E_INVALID;
    if (win != 3 && win != 5) return VDF_E_INVALID;
    const size_t bytes = (size_t)B * M * N * 3 * sizeof(float);
    if (overlaps(grad_y, bytes, grad_x, bytes)) return VDF_E_INVALID;
    return cuda_fail(vdf::run_backward(grad_y, index, grad_x, B, M, N, win / 2, (cudaStream_t)stream));
}

int vdf_num_tile_shapes(void) { return vdf::kNumShapes32; }

int vdf_tile_shape(int shape, int *tile_w, int *tile_h)
{
    if (shape < 0 || shape >= vdf::kNumShapes32) return VDF_E_INVALID;
    if (tile_w) *tile_w = vdf::kShapes32[shape].tw;
    if (tile_h) *tile_h = vdf::kShapes32[shape].th;
    return VDF_OK;
}

int vdf_get_tuned_shape(int win, int filter, int dist_mode)
{
    if ((win != 3 && win != 5) || filter < 0 || filter > 2 || dist_mode < 0 || dist_mode > 2) return VDF_E_INVALID;
    return tuned_shape(win, filter, filter == VDF_VMF ? VDF_DIST_EXACT : dist_mode);
}

int vdf_get_tuned_shape_p(int win, int filter, int dist_mode, double p)
{
    if ((win != 3 && win != 5) || filter < 0 || filter > 2 || dist_mode < 0 || dist_mode > 2) return VDF_E_INVALID;
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;
    return tuned_shape(win, filter, dist_mode, slot_kind(win, filter, dist_mode, vdf::NL2, p));
}

int vdf_set_tuned_shape(int win, int filter, int dist_mode, int shape)
{
    if ((win != 3 && win != 5) || filter < 0 || filter > 2 || dist_mode < 0 || dist_mode > 2) return VDF_E_INVALID;
    if (shape < 0 || shape >= vdf::kNumShapes32) return VDF_E_INVALID;
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;   // one entry: the VMF has no angular term
    for (int kind = 0; kind < kSlotKinds; ++kind) record_tuned_shape(win, filter, dist_mode, kind, shape);
    return VDF_OK;
}

}  // extern "C"

namespace vdf {
int tuned_shape_p(int win, int filter, int dist, double p) { return vdf_get_tuned_shape_p(win, filter, dist, p); }
}  // namespace vdf

extern "C" {

int vdf_autotune(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
                 uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes, int reps, void *stream,
                 int *best_shape, float *best_ms)
{
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;
    int rc = check_filter_args(img, M, N, win, filter, p, dist_mode, minimax_q, VDF_PREC_FP32_RECHECK, out,
                               index_out, nullptr, workspace, workspace_bytes);
    if (rc != VDF_OK) return rc;
    if (win == 7) return VDF_E_UNSUPPORTED;   // one kernel, no tile shapes to choose from
    if (reps < 1) reps = 1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e);
    }
    float best = 3.4e38f;
    int bs = 0;
    for (int s = 0; s < vdf::kNumShapes32 && rc == VDF_OK; ++s) {
        rc = fp32_pass_shape(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace,
                             workspace_bytes, s, stream);
        if (rc != VDF_OK) break;
        e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == VDF_OK && e == cudaSuccess; ++r)
            rc = fp32_pass_shape(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace,
                                 workspace_bytes, s, stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_fail(e);
        if (rc == VDF_OK && ms / reps < best) {
            best = ms / reps;
            bs = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != VDF_OK) return rc;
    record_tuned_shape(win, filter, dist_mode, slot_kind(win, filter, dist_mode, vdf::NL2, p), bs);
    // leave a complete result in out / index_out
    rc = vdf_fp32_pass(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace, workspace_bytes,
                       stream);
    if (rc == VDF_OK)
        rc = vdf_fp64_recheck(img, M, N, win, filter, p, dist_mode, minimax_q, out, index_out, workspace,
                              workspace_bytes, stream);
    if (best_shape) *best_shape = bs;
    if (best_ms) *best_ms = best;
    return rc;
}

int vdf_autotune_acwddf(const uint8_t *img, int M, int N, int win, int dist_mode, int minimax_q, int lambda,
                        double T, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes, int reps,
                        void *stream, int *best_shape, float *best_ms)
{
    int rc = check_filter_args(img, M, N, win, VDF_DDF, 0.5, dist_mode, minimax_q, VDF_PREC_FP32_RECHECK, out,
                               index_out, nullptr, workspace, workspace_bytes);
    if (rc != VDF_OK) return rc;
    if (win == 7) return VDF_E_UNSUPPORTED;
    const int d1 = (win * win + 1) / 2;
    if (lambda < 1 || lambda > d1 - 2 || !std::isfinite(T)) return VDF_E_INVALID;
    if (reps < 1) reps = 1;
    cudaStream_t st = (cudaStream_t)stream;
    vdf::TileParams prm = tile_params(img, M, N, 0.5, minimax_q, out, index_out, nullptr, workspace);
    prm.lam = lambda;
    prm.T = T;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 3.4e38f;
    int bs = 0;
    for (int s = 0; s < vdf::kNumShapes32 && e == cudaSuccess; ++s) {
        e = acw_pass_shape(prm, img, M, N, win, dist_mode, minimax_q, lambda, T, s, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = acw_pass_shape(prm, img, M, N, win, dist_mode, minimax_q, lambda, T, s, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms / reps < best) {
            best = ms / reps;
            bs = s;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e);
    record_tuned_shape(win, VDF_DDF, dist_mode, kAcwKind, bs);
    // leave a complete result in out / index_out
    e = acw_pass_shape(prm, img, M, N, win, dist_mode, minimax_q, lambda, T, bs, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (best_shape) *best_shape = bs;
    if (best_ms) *best_ms = best;
    return cuda_fail(e);
}

int vdf_debug_fp32_scores(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                          int minimax_q, float *fe_out, void *stream)
{
    if (filter == VDF_VMF) dist_mode = VDF_DIST_EXACT;
    if (!img || !fe_out || !valid_common(M, N, win, filter, p, dist_mode, minimax_q, VDF_PREC_FP32_RECHECK))
        return VDF_E_INVALID;
    if (win == 7) return VDF_E_UNSUPPORTED;
    vdf::TileParams prm{};
    prm.img = img;
    prm.dbg_fe = fe_out;
    prm.M = M;
    prm.N = N;
    prm.B = 1;
    prm.p = p;
    prm.q = minimax_q;
    return cuda_fail(run_tile32(prm, win / 2, filter, dist_mode, vdf::NL2, 0, (cudaStream_t)stream));
}

int vdf_debug_fp32_terms(const int *pairs, int n, int dist_mode, int minimax_q, float *angle_out, float *l2_out,
                         void *stream)
{
    if (!pairs || n < 0 || dist_mode < VDF_DIST_EXACT || dist_mode > VDF_DIST_RGB) return VDF_E_INVALID;
    if (dist_mode == VDF_DIST_MINIMAX && (minimax_q < 2 || minimax_q > 4)) return VDF_E_INVALID;
    return cuda_fail(vdf::run_debug_terms(pairs, n, dist_mode, minimax_q, angle_out, l2_out, (cudaStream_t)stream));
}

int vdf_debug_fp32_terms_f32(const float *pairs, int n, float *angle_out, float *l2_out, void *stream)
{
    if (!pairs || n < 0) return VDF_E_INVALID;
    return cuda_fail(vdf::run_debug_terms_f32(pairs, n, angle_out, l2_out, (cudaStream_t)stream));
}

int vdf_debug_sqrt_error(float *max_rel_err_u, void *stream)
{
    if (!max_rel_err_u) return VDF_E_INVALID;
    return cuda_fail(vdf::run_debug_sqrt_error(reinterpret_cast<unsigned *>(max_rel_err_u), (cudaStream_t)stream));
}

}  // extern "C"
