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
// name as a device address: on the first call in a device's context, with
// that device current, the address is looked up with cudaGetSymbolAddress
// and cached together with the context's ID. A later call in another context
// of the device (after cudaDeviceReset, or after the primary context was
// released and created again, when the module is loaded anew and the array
// may move) looks the address up again instead of using a stale one.
#include <cuda.h>
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
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context ID the address belongs to

using CtxGetCurrent = CUresult (*)(CUcontext *);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);

// ID of the calling thread's current context (driver entry points, resolved
// once); 0 if it cannot be read, in which case the address is looked up on
// every call.
unsigned long long current_ctx_id()
{
    static CtxGetCurrent get_current = nullptr;
    static CtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
                cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
                cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrent>(a);
            get_id = reinterpret_cast<CtxGetId>(b);
        }
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

corr_status_t scratch_on_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        corr::set_last_error(e);
        return CORR_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return CORR_ERR_UNSUPPORTED;
    const unsigned long long ctx = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            corr::set_last_error(e);
            return CORR_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
        // the lookup made the device's context current if it was not
        g_scratch_ctx[dev] = current_ctx_id();
    }
    *out = g_scratch_addr[dev];
    return CORR_OK;
}

// The kernels read and write complex values (8 bytes) and floats (4 bytes).
bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

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
    const void *cplx[] = {d_in, d_gain, d_vis_model, d_raw_vis, d_grad_gain, d_grad_in};
    for (const void *q : cplx)
        if (q && !aligned(q, 8)) return CORR_ERR_INVALID_ARG;
    if ((d_loss && !aligned(d_loss, 4)) || (d_grad_scale && !aligned(d_grad_scale, 4)))
        return CORR_ERR_INVALID_ARG;

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
