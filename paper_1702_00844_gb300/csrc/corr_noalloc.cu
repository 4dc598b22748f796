// Gain-calibration adjoint for callers that must not allocate device memory.
//
// corr_gain_backward needs a plan, and corr_create allocates (error word,
// workspaces). Some callers cannot do that: a real-time pipeline that forbids
// allocation once observing has started, a plug-in that runs inside another
// framework's memory pool, or code that issues work where a cudaMalloc would
// synchronize the device or fail. This file offers the same computation with
// its scratch memory (the per-channel matrix W' of the input gradient and the
// per-channel loss partials) in a fixed array that the library itself holds.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it until the process exits. Host code cannot use the array's
// name as a device address: on first use on a device, with that device
// current, the address is looked up once with cudaGetSymbolAddress and
// cached.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/corr.h"
#include "corr_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20; // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

corr_status_t scratch_on_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        corr::set_last_error(e);
        return CORR_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return CORR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            corr::set_last_error(e);
            return CORR_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CORR_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

} // namespace

extern "C" size_t corr_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" corr_status_t corr_gain_backward_noalloc(int n_stations, int n_units, int n_samples,
                                                    const void *d_in, const void *d_gain,
                                                    const void *d_vis_model, const void *d_raw_vis,
                                                    void *d_grad_gain, void *d_grad_in,
                                                    float *d_loss, const float *d_grad_scale,
                                                    void *stream)
{
    if (n_stations < 1 || n_units < 1 || n_samples < 0) return CORR_ERR_INVALID_ARG;
    if (!d_gain || !d_vis_model || !d_raw_vis || !d_grad_gain) return CORR_ERR_INVALID_ARG;
    if (d_grad_in && n_samples > 0 && !d_in) return CORR_ERR_INVALID_ARG;
    const void *ptrs[] = {d_in, d_gain, d_vis_model, d_raw_vis, d_grad_gain, d_grad_in, d_loss};
    for (const void *q : ptrs)
        if (q && !aligned16(q)) return CORR_ERR_INVALID_ARG;

    // scratch layout: loss partials (one float per channel), then W'
    const size_t n = 2 * (size_t)n_stations;
    const size_t partial_bytes = d_loss ? ((size_t)n_units * sizeof(float) + 255) / 256 * 256 : 0;
    const size_t w_bytes = d_grad_in ? (size_t)n_units * n * n * sizeof(float2) : 0;
    if (partial_bytes + w_bytes > kScratchBytes) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "corr_gain_backward_noalloc: needs %zu bytes of scratch, the fixed array holds %zu",
                 partial_bytes + w_bytes, kScratchBytes);
        corr::set_last_error(msg);
        return CORR_ERR_UNSUPPORTED;
    }
    void *base = nullptr;
    corr_status_t st = scratch_on_current_device(&base);
    if (st != CORR_OK) return st;
    float *partial = static_cast<float *>(base);
    float2 *W = reinterpret_cast<float2 *>(static_cast<unsigned char *>(base) + partial_bytes);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float2 *R = static_cast<const float2 *>(d_raw_vis);
    const float2 *g = static_cast<const float2 *>(d_gain);
    const float2 *M = static_cast<const float2 *>(d_vis_model);
    cudaError_t e = corr::gain_grad_launch(R, g, M, d_grad_scale, static_cast<float2 *>(d_grad_gain),
                                           d_grad_in ? W : nullptr, n_stations, n_units, s);
    if (e == cudaSuccess && d_grad_in)
        e = corr::input_grad_launch(static_cast<const float2 *>(d_in), W, static_cast<float2 *>(d_grad_in),
                                    n_stations, n_samples, n_units, s);
    if (e == cudaSuccess && d_loss)
        e = corr::gain_loss_launch(R, g, M, nullptr, partial, d_loss, n_stations, n_units, s);
    if (e != cudaSuccess) {
        corr::set_last_error(e);
        return CORR_ERR_CUDA;
    }
    return CORR_OK;
}
