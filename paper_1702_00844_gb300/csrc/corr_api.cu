// C ABI of the correlator: plan creation, argument checks, work lists and
// kernel dispatch. See include/corr.h for the contract of every entry point.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cerrno>
#include <fcntl.h>
#include <map>
#include <string>
#include <sys/stat.h>
#include <unistd.h>
#include <tuple>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/corr.h"
#include "corr_internal.h"

using namespace corr;

// A tile configuration of the tensor path: the variant of the main work
// list, the variant of the tail list (pair variant with an odd block count:
// narrow tiles for the last block column, or wide tiles for block 0's row)
// and the kernel layout (int8 pair tiles of two pols: 0 with staged
// epilogue groups, 1 with the six-stage operand ring).
struct TileCfg {
    int variant = TC_NARROW;
    int tail = TC_WIDE;
    int layout = 0;
};

struct corr_plan {
    corr_desc_t d{};
    int device = 0;
    int sm_count = 0;
    int path = CORR_PATH_FP32;
    int *d_err = nullptr;
    unsigned long long wait_ns = 2000000000ull;
    // FP32 path
    Fp32Params fp{};
    int fp_threads = 0;
    size_t fp_smem = 0;
    float2 *d_fp_partial = nullptr; // partial sums of a split sample axis
    // tensor path (single problem)
    int4 *d_items = nullptr;   // main list, then the tail list (pair variant)
    int n_items = 0;           // main list
    int n_tail = 0;            // tail list (pair variant, odd block count)
    TileCfg tc;                // tile configuration (autotuned in corr_create)
    int tune_source = 0;       // how it was chosen (corr_tile_config)
    int pair_clusters = 0;     // clusters of the pair variant resident at once (0: unavailable)
    std::vector<TileCfg> tune_cfgs;  // candidates timed in corr_create, and their times
    std::vector<float> tune_ms;
    // int8 power check / redo list (single problem and batches): state =
    // {count, done} of the main and the tail list, then one mark per item
    int *d_redo_state = nullptr;
    int *d_redo_index = nullptr;
    int4 *d_redo_items = nullptr;
    int redo_cap = 0;
    // ragged batches
    std::vector<corr_subarray_t> batch_key;
    TcProblem *d_bprobs = nullptr;
    int4 *d_bitems = nullptr;
    int n_bitems = 0;
    int n_btail = 0;
    TileCfg bc;                // tile configuration of the current batch
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;  // corr_set_kernel_events (not owned)
    std::vector<TileCfg> b_tune_cfgs;  // batch candidates timed and their best times
    std::vector<float> b_tune_ms;
    // host-buffer streaming (CORR_FLAG_HOST_IO)
    int chunk_units = 0;
    void *d_stage_in[2] = {nullptr, nullptr};
    void *d_stage_out[2] = {nullptr, nullptr};
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
    // gain calibration
    float2 *d_R = nullptr;     // recomputed raw visibilities
    float2 *d_W = nullptr;     // W' per channel
    float *d_At = nullptr;     // W' as the tensor-core input gradient's A' tiles
    // FP32 samples on the tensor cores with few tiles: per-chunk partial sums
    float2 *d_tf_partial = nullptr;
    float *d_partial = nullptr;
};

namespace {

thread_local char g_last_error[256] = "";

constexpr int TC_SIDE = TC_RS;

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
// Alignment the gain kernels need: complex float32 values (8 bytes), floats (4).
bool aligned_to(const void *p, uintptr_t a) { return !p || (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

long long n_baselines(long long S) { return S * (S + 1) / 2; }

// Internal path id of a plan with FP32 samples on the tensor cores (path
// CORR_PATH_TENSOR, dtype CORR_CF32 in the descriptor).
constexpr int PATH_TF32 = 3;
constexpr int TF_CHUNK_KB = 16;   // 256 samples per accumulator chunk

// Accumulator chunks of a tf32-split tile over T samples.
long long tf_chunks(int T) { return ((T + 15) / 16 + TF_CHUNK_KB - 1) / TF_CHUNK_KB; }

int tc_blocks(int S) { return (S + TC_SIDE - 1) / TC_SIDE; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// FP32 input as a 4-D tensor: (4 floats of one station and time) x station x
// time x unit, boxes of 4 x 8 stations x tc samples x 1 unit, so that a box
// lands in shared memory as [t][8 stations][4 floats].
// With fewer tiles than two per SM, tf32-split plans spread the chunks of
// each tile over the CTAs (partial sums summed afterwards).
bool tf_use_partial(const corr_plan *h, long long units)
{
    const long long nb = (h->d.n_stations + 63) / 64, ntri = nb * (nb + 1) / 2;
    return h->d_tf_partial && tf_chunks(h->d.n_samples) > 1 && units * ntri < 2LL * h->sm_count;
}

corr_status_t encode_fp32_map(CUtensorMap *m, const void *d_in, int S, int T, int units, int tc)
{
    auto fn = encode_fn();
    if (!fn) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled unavailable");
        return CORR_ERR_CUDA;
    }
    cuuint64_t dims[4] = {4, (cuuint64_t)S, (cuuint64_t)T, (cuuint64_t)units};
    cuuint64_t strides[3] = {(cuuint64_t)T * 16, 16, (cuuint64_t)S * T * 16};
    cuuint32_t box[4] = {4, 8, (cuuint32_t)tc, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(d_in), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return CORR_ERR_CUDA;
    }
    return CORR_OK;
}

// The samples for the tensor-core input gradient as 8-byte elements (one
// complex float each, copied bit for bit): dims (2T per station, stations,
// units, 1), boxes of 2 CORR_IG_BOX elements x 8 stations: one contiguous
// run of CORR_IG_BOX x 16 bytes per station, landing station-major. No swizzle
// mode; the kernel transposes and swizzles.
corr_status_t encode_ig_map(CUtensorMap *m, const void *d_in, int S, int T, long long units)
{
    auto fn = encode_fn();
    if (!fn) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled unavailable");
        return CORR_ERR_CUDA;
    }
    cuuint64_t dims[4] = {2 * (cuuint64_t)T, (cuuint64_t)S, (cuuint64_t)units, 1};
    cuuint64_t strides[3] = {(cuuint64_t)T * 16, (cuuint64_t)S * T * 16, (cuuint64_t)units * S * T * 16};
    cuuint32_t box[4] = {2 * CORR_IG_BOX, CORR_IG_KV / 4, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void *>(d_in), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled (input gradient) failed (%d)", (int)r);
        return CORR_ERR_CUDA;
    }
    return CORR_OK;
}

// The samples for the tf32-split tensor correlator as 8-byte elements (one
// complex float per pol, copied bit for bit): dims (2T per station, stations,
// units, 1), boxes of 32 elements (16 samples x 2 pols) x 64 stations: one
// contiguous 256-byte run per station, landing station-major.
corr_status_t encode_tf32_map(CUtensorMap *m, const void *d_in, int S, int T, long long units)
{
    auto fn = encode_fn();
    if (!fn) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled unavailable");
        return CORR_ERR_CUDA;
    }
    cuuint64_t dims[4] = {2 * (cuuint64_t)T, (cuuint64_t)S, (cuuint64_t)units, 1};
    cuuint64_t strides[3] = {(cuuint64_t)T * 16, (cuuint64_t)S * T * 16, (cuuint64_t)units * S * T * 16};
    cuuint32_t box[4] = {32, 64, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void *>(d_in), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled (tf32 correlator) failed (%d)", (int)r);
        return CORR_ERR_CUDA;
    }
    return CORR_OK;
}

// Stations of the work lists and sub-tile grids: with one pol, pairs of stations
// act as the two pols of one pseudo-station.
int item_stations(int S, int npol) { return npol == 1 ? (S + 1) / 2 : S; }

void fp32_config(corr_plan *h)
{
    // one pol: sub-tiles over pseudo-stations (pairs of stations)
    const int S = item_stations(h->d.n_stations, h->d.n_pols);
    Fp32Params &p = h->fp;
    p.S = S;
    p.S1 = h->d.n_stations;
    p.T = h->d.n_samples;
    p.n_units = h->d.n_channels * h->d.n_integrations;
    // 4 x 2-station sub-tiles up to 64 (pseudo-)stations, else 4 x 4
    // (measured: equal at 64 stations x 2560 units, 12% faster at 64 x 64
    // units, 35-40% slower at 256 and 512 stations); CORR_FP32_TW=2|4 forces
    // one.
    p.tw = S <= 64 ? 2 : 4;
    if (const char *e = std::getenv("CORR_FP32_TW")) p.tw = std::atoi(e) == 2 ? 2 : 4;
    p.nq = (S + 3) / 4;
    p.ncq = (S + p.tw - 1) / p.tw;
    p.nsub = 0;
    for (int i = 0; i < p.nq; ++i) p.nsub += p.ncq - 4 * i / p.tw;
    // at most 192 threads per CTA (4 x 4: two CTAs of 168-register threads
    // fit an SM) or 288 (4 x 2: two CTAs of 112-register threads)
    // A load warp (two pols, TMA staging) replaces the block barrier per
    // stage in the 4 x 2 form. (Measured in the 4 x 4 form, where it takes
    // the place of a sixth compute warp: slower at 128 and 256 stations,
    // faster at 512.)
    p.load_warp = h->d.n_pols == 2 && p.tw == 2 ? 1 : 0;
    int max_threads = p.tw == 4 ? 192 : 288;
    if (const char *e = std::getenv("CORR_FP32_MAXT")) max_threads = std::max(32, std::min(max_threads, std::atoi(e)));
    p.groups = (p.nsub + max_threads - 1) / max_threads;
    p.group_size = (p.nsub + p.groups - 1) / p.groups;
    h->fp_threads = ((p.group_size + 31) / 32) * 32;
    if (p.load_warp) h->fp_threads += 32;
    const int nbox = (S + 7) / 8;
    int tc = 32;
    if (const char *e = std::getenv("CORR_FP32_TC")) tc = std::max(1, std::min(64, std::atoi(e)));
    while (tc > 1 && (size_t)FP32_STAGES * nbox * tc * 128 > 100 * 1024) tc >>= 1;
    p.tc = tc;
    h->fp_smem = (size_t)FP32_STAGES * nbox * tc * 128 + 128;
    // Few units (channels x integrations) leave SMs idle: then the sample
    // axis is split into ranges of whole chunks over more CTAs, and a second
    // kernel sums the partial results in order.
    // CORR_FP32_KSPLIT forces a split count.
    // Both sub-tile forms fit two CTAs per SM. Measured on 64 channels of 64
    // stations, many short CTAs run best (16 CTAs of 2 chunks per channel:
    // 0.144 ms against 0.159 for 4 of 8 and 0.175 for 5 of 7): chunks per
    // CTA are chosen for about four waves of 2 x SMs CTAs, at least 2.
    const int total = std::max(1, (p.T + tc - 1) / tc);
    const long long ctas = (long long)p.n_units * p.groups;
    const long long slots = 2LL * h->sm_count;
    int ks = 1;
    if (p.T > 0 && total > 1 && ctas < slots) {
        const long long per = std::min<long long>(
            total, std::max<long long>(2, ((long long)total * ctas + 4 * slots - 1) / (4 * slots)));
        ks = (int)((total + per - 1) / per);
    }
    if (const char *e = std::getenv("CORR_FP32_KSPLIT")) ks = std::max(1, std::min(total, std::atoi(e)));
    p.kchunks = (total + ks - 1) / ks;
    p.ksplit = (total + p.kchunks - 1) / p.kchunks;
    p.partial = nullptr;
}

// Bytes of one station-time sample of all npol pols.
int sample_bytes(int dtype, int npol) { return npol * (dtype == CORR_CF32 ? 8 : dtype == CORR_CF16 ? 4 : 2); }

size_t in_unit_bytes(const corr_desc_t &d)
{
    return (size_t)d.n_stations * d.n_samples * sample_bytes(d.dtype, d.n_pols);
}

size_t out_unit_bytes(const corr_desc_t &d)
{
    return (size_t)n_baselines(d.n_stations) * d.n_pols * d.n_pols * 8;
}

// Work items of the tensor kernel: {prob, unit, rb, cb0 | ncb << 16}, row
// block rb and column blocks cb0..cb0+ncb-1 of 64 stations, rb <= cb0.
// narrow: every (rb, cb) with rb <= cb; wide: column blocks taken in pairs
// from the row block onward (the last one alone if the count is odd); pair:
// row blocks {rb, rb+1} x column blocks {cb0, cb0+1} for rb <= cb0 over an
// even number of blocks. When the block count nb is odd one block is left
// over (a pair tile there would hold a block without stations), and its
// tiles go to *tail: with tail_kind TC_WIDE the pair tiles cover blocks
// 1 .. nb-1 and block 0's row goes to the tail as wide tiles, the diagonal
// tile (0, 0) and then (0, {c, c+1}) for c = 1, 3, ... (fewer tiles, each
// with N = 256); with TC_NARROW the pair tiles cover blocks 0 .. nb-2 and
// the last block column goes to the tail as narrow tiles (nb of them, with
// double-buffered accumulators). Items are unit-major.
std::vector<int4> tc_items_for(int prob, int S, int units, int variant, std::vector<int4> *tail,
                               int tail_kind = TC_WIDE)
{
    std::vector<int4> v;
    const int nb = tc_blocks(S);
    for (int u = 0; u < units; ++u) {
        if (variant == TC_PAIR && (nb & 1) && tail_kind == TC_NARROW) {
            // pair tiles over blocks 0 .. nb-2, the last block column as narrow tiles
            for (int rb = 0; rb + 1 < nb; rb += 2)
                for (int cb = rb; cb + 1 < nb; cb += 2) v.push_back(make_int4(prob, u, rb, cb | (2 << 16)));
            for (int rb = 0; rb < nb; ++rb) tail->push_back(make_int4(prob, u, rb, (nb - 1) | (1 << 16)));
        } else if (variant == TC_PAIR) {
            const int b0 = nb & 1;   // first block of the pair tiles
            for (int rb = b0; rb < nb; rb += 2)
                for (int cb = rb; cb < nb; cb += 2) v.push_back(make_int4(prob, u, rb, cb | (2 << 16)));
            if (b0) {
                tail->push_back(make_int4(prob, u, 0, 0 | (1 << 16)));
                for (int cb = 1; cb < nb; cb += 2) tail->push_back(make_int4(prob, u, 0, cb | (2 << 16)));
            }
        } else if (variant == TC_WIDE) {
            for (int rb = 0; rb < nb; ++rb)
                for (int cb = rb; cb < nb; cb += 2) {
                    const int ncb = std::min(2, nb - cb);
                    v.push_back(make_int4(prob, u, rb, cb | (ncb << 16)));
                }
        } else {
            for (int cb = 0; cb < nb; ++cb)
                for (int rb = 0; rb <= cb; ++rb) v.push_back(make_int4(prob, u, rb, cb | (1 << 16)));
        }
    }
    return v;
}

int bytes_per_sample(int dtype) { return dtype == CORR_CF32 ? 16 : dtype == CORR_CF16 ? 8 : 4; }



TcProblem make_problem(const void *in, void *out, int S, int T, int units, int dtype, int npol)
{
    TcProblem pr{};
    pr.in = in;
    pr.out = out;
    pr.S = S;
    pr.T = T;
    pr.n_units = units;
    pr.in_unit_bytes = (long long)S * T * sample_bytes(dtype, npol);
    pr.out_unit_elems = n_baselines(S) * npol * npol;
    pr.vec = (((long long)T * sample_bytes(dtype, npol)) % 16 == 0) ? 1 : 0;
    return pr;
}

corr_status_t cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return CORR_OK;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return CORR_ERR_NO_MEMORY;
    return CORR_ERR_CUDA;
}

// Grows the redo buffers to hold n items (allocation: create time or the
// first batched call with a new set, never during a capturable call).
corr_status_t ensure_redo(corr_plan *h, int n)
{
    if (n <= h->redo_cap) return CORR_OK;
    cudaFree(h->d_redo_state);
    cudaFree(h->d_redo_index);
    cudaFree(h->d_redo_items);
    h->d_redo_state = nullptr;
    h->d_redo_index = nullptr;
    h->d_redo_items = nullptr;
    h->redo_cap = 0;
    corr_status_t st;
    // {count, done} of the main list (ctr 0) and the tail list (ctr 1), then
    // the marks; list (redo_off, ctr) uses marks, indices and items from
    // redo_off on. Zeroed once here; each redo launch leaves it zeroed again.
    const size_t state_bytes = ((size_t)n + 4) * sizeof(int);
    if ((st = cuda_status(cudaMalloc(&h->d_redo_state, state_bytes))) != CORR_OK) return st;
    if ((st = cuda_status(cudaMalloc(&h->d_redo_index, (size_t)n * sizeof(int)))) != CORR_OK) return st;
    if ((st = cuda_status(cudaMalloc(&h->d_redo_items, (size_t)n * sizeof(int4)))) != CORR_OK) return st;
    if ((st = cuda_status(cudaMemset(h->d_redo_state, 0, state_bytes))) != CORR_OK) return st;
    if ((st = cuda_status(cudaDeviceSynchronize())) != CORR_OK) return st;
    h->redo_cap = n;
    return CORR_OK;
}

// Launches the tensor kernel for p.items[0 .. p.n_items). int8 with more than
// one 512-sample chunk runs unchunked with the station power check, then a
// chunked launch over the items the check rejected (usually none).
// CTAs of a launch over up to n items: one per SM, or two per cluster of
// the pair variant.
int tc_grid_for(const corr_plan *h, int variant, int n)
{
    if (variant == TC_PAIR) return 2 * std::max(1, std::min(n, h->pair_clusters));
    return std::max(1, std::min(n, h->sm_count));
}

// One item list in one tile variant. The int8 redo list of this launch uses
// the plan's redo entries [redo_off, redo_off + p.n_items) and counter `ctr`.
corr_status_t run_list(corr_plan *h, TcParams p, int dtype, int variant, int layout, int max_T, int redo_off,
                       int ctr, cudaStream_t s)
{
    if (variant == TC_PAIR && h->pair_clusters < 1) {
        set_last_error("the pair tile variant does not fit on this device");
        return CORR_ERR_UNSUPPORTED;
    }
    const int grid = tc_grid_for(h, variant, p.n_items);
    const bool checked = dtype == CORR_CI8 && max_T > TC_INT8_CHUNK_KB * TC_KB_T &&
                         h->redo_cap >= redo_off + p.n_items;
    // measurement hook (corr_set_kernel_events): around the main list's
    // first launch only
    const bool mark = ctr == 0 && h->ev_k0 && h->ev_k1;
    // Both lists' first launches are programmatic dependents, so that their
    // CTAs take SMs as soon as the previous kernel's CTAs leave them. The
    // main list (ctr 0) may read what the kernel before it wrote: its CTAs
    // wait for that kernel after their set-up (dep_wait). The tail list
    // (ctr 1) reads nothing the main list's launches write and needs no
    // wait.
    const bool pdl = true;
    p.dep_wait = ctr == 0 ? 1 : 0;
    if (!checked) {
        p.chunk_kb = dtype == CORR_CI8 ? TC_INT8_CHUNK_KB : 0;
        if (mark) cudaEventRecord(h->ev_k0, s);
        corr_status_t st = cuda_status(tc_launch(dtype, variant, h->d.n_pols, p, grid, s, pdl, layout));
        if (mark) cudaEventRecord(h->ev_k1, s);
        return st;
    }
    // The list is empty when a call starts: the previous redo launch left it
    // so (no memset per call).
    int *count = h->d_redo_state + 2 * ctr;
    TcParams a = p;
    a.chunk_kb = 0;
    a.check_power = 1;
    a.redo_mark = h->d_redo_state + 4 + redo_off;
    a.redo_items = h->d_redo_items + redo_off;
    a.redo_index = h->d_redo_index + redo_off;
    a.redo_count = count;
    a.redo_done = nullptr;
    if (mark) cudaEventRecord(h->ev_k0, s);
    corr_status_t st = cuda_status(tc_launch(dtype, variant, h->d.n_pols, a, grid, s, pdl, layout));
    if (mark) cudaEventRecord(h->ev_k1, s);
    if (st != CORR_OK) return st;
    // the chunked redo launch over the rejected items (usually none), as a
    // programmatic dependent: its CTAs are scheduled while the checked launch
    // ends and wait for it before reading the count, so an empty list costs
    // no launch gap
    TcParams b = a;
    b.items = h->d_redo_items + redo_off;
    b.n_items = p.n_items;          // upper bound; the count is read on the device
    b.n_items_dev = count;
    b.chunk_kb = TC_INT8_CHUNK_KB;
    b.check_power = 0;
    b.redo_done = count + 1;
    b.dep_wait = 0;                 // it waits for the checked launch at its start
    return cuda_status(
        tc_launch(dtype, variant, h->d.n_pols, b, tc_grid_for(h, variant, p.n_items), s, true, layout));
}

// The main list of p in cfg.variant, then (pair variant) the n_tail tail
// items at `tail` in cfg.tail.
corr_status_t run_tensor(corr_plan *h, TcParams p, const int4 *tail, int n_tail, int dtype, const TileCfg &cfg,
                         int max_T, cudaStream_t s)
{
    corr_status_t st = CORR_OK;
    if (p.n_items > 0) st = run_list(h, p, dtype, cfg.variant, cfg.layout, max_T, 0, 0, s);
    if (st == CORR_OK && n_tail > 0) {
        TcParams q = p;
        q.items = tail;
        q.n_items = n_tail;
        st = run_list(h, q, dtype, cfg.tail, 0, max_T, p.n_items, 1, s);
    }
    return st;
}

corr_status_t launch_units(corr_plan *h, const void *d_in, void *d_out, long long units,
                           cudaStream_t s)
{
    const corr_desc_t &d = h->d;
    const size_t out_bytes = (size_t)units * out_unit_bytes(d);
    if (d.n_samples == 0) return cuda_status(cudaMemsetAsync(d_out, 0, out_bytes, s));
    if (h->path == PATH_TF32) {
        CUtensorMap m{};
        corr_status_t st = encode_tf32_map(&m, d_in, d.n_stations, d.n_samples, units);
        if (st != CORR_OK) return st;
        TfParams p{};
        p.out = static_cast<float2 *>(d_out);
        p.S = d.n_stations;
        p.T = d.n_samples;
        p.units = (int)units;
        p.nb = (d.n_stations + 63) / 64;
        p.chunk_kb = TF_CHUNK_KB;
        // fewer tiles than two per SM: every chunk of a tile is a work item
        // of its own, summed by a second kernel
        p.partial = tf_use_partial(h, units) ? h->d_tf_partial : nullptr;
        p.err = h->d_err;
        p.wait_ns = h->wait_ns;
        const bool mark = h->ev_k0 && h->ev_k1;
        if (mark) cudaEventRecord(h->ev_k0, s);
        st = cuda_status(tf32_correlate_launch(&m, p, s));
        if (mark) cudaEventRecord(h->ev_k1, s);
        return st;
    }
    if (h->path == CORR_PATH_FP32) {
        CUtensorMap m{};
        if (d.n_pols == 2) {
            corr_status_t st = encode_fp32_map(&m, d_in, d.n_stations, d.n_samples, (int)units, h->fp.tc);
            if (st != CORR_OK) return st;
        }
        Fp32Params p = h->fp;
        p.n_units = (int)units;
        p.out = static_cast<float2 *>(d_out);
        p.in1 = static_cast<const float2 *>(d_in);
        p.partial = p.ksplit > 1 ? h->d_fp_partial : nullptr;
        p.err = h->d_err;
        p.wait_ns = h->wait_ns;
        const bool mark = h->ev_k0 && h->ev_k1;
        if (mark) cudaEventRecord(h->ev_k0, s);
        corr_status_t st = cuda_status(fp32_launch(&m, p, d.n_pols, h->fp_threads, h->fp_smem, s));
        if (mark) cudaEventRecord(h->ev_k1, s);
        return st;
    }
    TcParams p{};
    p.prob0 = make_problem(d_in, d_out, d.n_stations, d.n_samples, (int)units, d.dtype, d.n_pols);
    p.probs = nullptr;
    // both lists are unit-major, so the first units' items are prefixes
    const long long all_units = (long long)d.n_channels * d.n_integrations;
    p.items = h->d_items;
    p.n_items = (int)((long long)h->n_items / all_units * units);
    p.err = h->d_err;
    p.wait_ns = h->wait_ns;
    return run_tensor(h, p, h->d_items + h->n_items, (int)((long long)h->n_tail / all_units * units),
                      d.dtype, h->tc, d.n_samples, s);
}

corr_status_t launch_correlate(corr_plan *h, const void *d_in, void *d_out, cudaStream_t s)
{
    return launch_units(h, d_in, d_out, (long long)h->d.n_channels * h->d.n_integrations, s);
}


// ------------------------------------------------------------------ autotuner
// The tile configuration of the tensor path (variant, tail kind, kernel
// layout) is chosen per (device, dtype, pols, S, T, units):
//  1. CORR_TC_VARIANT=narrow|wide|pair, CORR_TC_TAIL=narrow|wide and
//     CORR_TC_LAYOUT=0|1 force parts of it (the rest by the size rule);
//  2. CORR_FLAG_NO_AUTOTUNE (or T = 0) takes the size rule: pair tiles from
//     128 stations, a wide tail from 5 blocks, layout 0;
//  3. otherwise a choice cached in this process, or in the cache file, is
//     used; else the candidates the cost model keeps are timed on seeded
//     non-zero samples of the plan's shape and the fastest is kept (in
//     memory and appended to the cache file).
// The cache file is CORR_TUNE_CACHE if set ("off": none), else
// $XDG_CACHE_HOME/corr_gb300/tune.txt or ~/.cache/corr_gb300/tune.txt. A
// line holds the build of this library, the GPU's name and SM count, the
// shape and the choice; lines of other builds are ignored.
enum { TUNE_FORCED = 0, TUNE_RULE = 1, TUNE_TIMED = 2, TUNE_MEMORY = 3, TUNE_FILE = 4 };

struct TuneKey {
    int dev, dtype, npol, S, T;
    long long units; // the choice depends on the waves of work items too
    bool operator<(const TuneKey &o) const
    {
        return std::tie(dev, dtype, npol, S, T, units) < std::tie(o.dev, o.dtype, o.npol, o.S, o.T, o.units);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, TileCfg> g_tune_cache;
const char *const kBuildId = __DATE__ " " __TIME__;

int env_variant(const char *name)
{
    const char *e = std::getenv(name);
    if (!e) return -1;
    if (std::strcmp(e, "wide") == 0) return TC_WIDE;
    if (std::strcmp(e, "narrow") == 0) return TC_NARROW;
    if (std::strcmp(e, "pair") == 0) return TC_PAIR;
    return -1;
}

int forced_variant() { return env_variant("CORR_TC_VARIANT"); }

int forced_layout()
{
    const char *e = std::getenv("CORR_TC_LAYOUT");
    if (!e) return -1;
    return std::atoi(e) == 1 ? 1 : 0;
}

// Layout 1 exists for the int8 pair kernel of two pols only.
bool has_layouts(const corr_desc_t &d) { return d.dtype == CORR_CI8 && d.n_pols == 2; }

// Size rule for S (item) stations: pair tiles from 128 stations when they fit
// (wide otherwise), narrow below; the wide tail from 5 blocks (at 3 blocks
// the narrow tail's double-buffered accumulators measured faster).
TileCfg rule_cfg(const corr_plan *h, int S_items)
{
    TileCfg c;
    c.variant = S_items >= 128 ? (h->pair_clusters > 0 ? TC_PAIR : TC_WIDE) : TC_NARROW;
    c.tail = tc_blocks(S_items) >= 5 ? TC_WIDE : TC_NARROW;
    c.layout = 0;
    return c;
}

TileCfg apply_forced(const corr_plan *h, TileCfg c, bool *any)
{
    const int v = forced_variant(), t = env_variant("CORR_TC_TAIL"), l = forced_layout();
    *any = v >= 0 || t >= 0 || l >= 0;
    if (v >= 0) c.variant = (v == TC_PAIR && h->pair_clusters < 1) ? TC_WIDE : v;
    if (t == TC_NARROW || t == TC_WIDE) c.tail = t;
    if (l >= 0) c.layout = has_layouts(h->d) ? l : 0;
    return c;
}

// Cost model of a tile configuration (in the spirit of Section 2's Table 1:
// work per tile against the operand bytes it moves). A tile's MMAs read
// their operands from shared memory: per tensor-core clock 128 B (narrow,
// M = N = 128), 96 B (wide, N = 256) or 64 B per SM (pair, M = 256 over two
// SMs), of which the tensor core sustains about 72 B/clk (measured MMA-only
// rates: 60 %, 75 %, about 100 %). Predicted time = SM-time of the computed
// station pairs (the lower triangles of diagonal tiles included) over the
// SM count; used only to prune candidates before timing.
double tile_eff(int v) { return v == TC_PAIR ? 1.0 : v == TC_WIDE ? 0.75 : 0.5625; }

double model_items(const std::vector<int4> &items, int variant, int S_items)
{
    double w = 0;
    for (const int4 &it : items) {
        const int ncb = it.w >> 16, cb0 = it.w & 0xFFFF;
        if (variant == TC_PAIR) {
            w += 2.0 * 64.0 * 128.0 / tile_eff(TC_PAIR);
        } else {
            const int last = std::min(TC_SIDE, S_items - (cb0 + ncb - 1) * TC_SIDE);
            const int cols = (ncb - 1) * TC_SIDE + ((2 * last + 15) / 16) * 8;
            w += 64.0 * cols / tile_eff(variant);
        }
    }
    return w;
}

double model_cost(const corr_plan *h, int S_items, int T, long long units, const TileCfg &c)
{
    std::vector<int4> tail;
    const std::vector<int4> items = tc_items_for(0, S_items, 1, c.variant, &tail, c.tail);
    const double w = model_items(items, c.variant, S_items) + model_items(tail, c.tail, S_items);
    return w * (double)T * (double)units / std::max(1, h->sm_count);
}

// Candidates for S (item) stations: narrow, wide and pair tiles (both tail
// kinds when the block count is odd, both layouts where there are two),
// pruned to those the cost model puts within 1.3x of the best.
std::vector<TileCfg> tune_candidates(const corr_plan *h, const std::vector<std::tuple<int, int, long long>> &shapes)
{
    std::vector<TileCfg> all;
    bool odd = false;
    for (const auto &sh : shapes) odd |= (tc_blocks(std::get<0>(sh)) & 1) != 0;
    for (int v = 0; v < TC_N_VARIANTS; ++v) {
        if (v == TC_PAIR && h->pair_clusters < 1) continue;
        for (int t : {TC_WIDE, TC_NARROW}) {
            if (v != TC_PAIR && t != TC_WIDE) continue;   // the tail kind applies to pair tiles only
            if (v == TC_PAIR && !odd && t != TC_WIDE) continue;
            for (int l = 0; l < (v == TC_PAIR && has_layouts(h->d) ? 2 : 1); ++l) {
                TileCfg c;
                c.variant = v;
                c.tail = t;
                c.layout = l;
                all.push_back(c);
            }
        }
    }
    std::vector<double> cost(all.size(), 0.0);
    double best = 1e300;
    for (size_t i = 0; i < all.size(); ++i) {
        for (const auto &sh : shapes)
            cost[i] += model_cost(h, std::get<0>(sh), std::get<1>(sh), std::get<2>(sh), all[i]);
        best = std::min(best, cost[i]);
    }
    std::vector<TileCfg> keep;
    for (size_t i = 0; i < all.size(); ++i)
        if (cost[i] <= 1.3 * best) keep.push_back(all[i]);
    return keep;
}

// Seeded non-zero samples for the timing runs: a counter-based 32-bit hash
// (Wellons' "lowbias32": xorshift-multiply rounds) of each word's index;
// int8 samples uniform in [-55, 55] (the rms of N(0, 32^2) samples, so that
// the station power check behaves as on such data), f16 samples uniform in
// [-1, 1).
__global__ void tune_fill_kernel(uint32_t *w, size_t n, int f16, uint32_t seed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 0x9E3779B9u ^ seed;
        x ^= x >> 16;
        x *= 0x7feb352du;
        x ^= x >> 15;
        x *= 0x846ca68bu;
        x ^= x >> 16;
        uint32_t out = 0;
        if (f16) {
            for (int k = 0; k < 2; ++k) {
                const float v = (float)((int)((x >> (16 * k)) & 0x3FFu) - 512) / 512.0f;
                out |= (uint32_t)__half_as_ushort(__float2half_rn(v)) << (16 * k);
            }
        } else {
            for (int k = 0; k < 4; ++k) {
                const int v = (int)((x >> (8 * k)) & 0xFFu) % 111 - 55;
                out |= (uint32_t)(v & 0xFF) << (8 * k);
            }
        }
        w[i] = out;
    }
}

corr_status_t time_config(corr_plan *h, const TileCfg &cfg, int S, int T, int units, const void *d_in,
                          void *d_out, float *ms_out)
{
    std::vector<int4> tail;
    std::vector<int4> items = tc_items_for(0, item_stations(S, h->d.n_pols), units, cfg.variant, &tail, cfg.tail);
    const int n_main = (int)items.size(), n_tail = (int)tail.size();
    items.insert(items.end(), tail.begin(), tail.end());
    int4 *d_items = nullptr;
    corr_status_t st = cuda_status(cudaMalloc(&d_items, items.size() * sizeof(int4)));
    if (st != CORR_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        if ((st = cuda_status(cudaMemcpy(d_items, items.data(), items.size() * sizeof(int4),
                                         cudaMemcpyHostToDevice))) != CORR_OK)
            break;
        TcParams p{};
        p.prob0 = make_problem(d_in, d_out, S, T, units, h->d.dtype, h->d.n_pols);
        p.items = d_items;
        p.n_items = n_main;
        p.err = h->d_err;
        p.wait_ns = h->wait_ns;
        if (h->d.dtype == CORR_CI8 && (st = ensure_redo(h, n_main + n_tail)) != CORR_OK) break;
        if ((st = cuda_status(cudaEventCreate(&e0))) != CORR_OK) break;
        if ((st = cuda_status(cudaEventCreate(&e1))) != CORR_OK) break;
        for (int i = 0; i < 2 && st == CORR_OK; ++i)
            st = run_tensor(h, p, d_items + n_main, n_tail, h->d.dtype, cfg, T, 0);
        if (st != CORR_OK) break;
        cudaEventRecord(e0, 0);
        for (int i = 0; i < 3 && st == CORR_OK; ++i)
            st = run_tensor(h, p, d_items + n_main, n_tail, h->d.dtype, cfg, T, 0);
        cudaEventRecord(e1, 0);
        if (st != CORR_OK) break;
        if ((st = cuda_status(cudaEventSynchronize(e1))) != CORR_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *ms_out = ms / 3.f;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_items);
    return st;
}

std::string tune_cache_path()
{
    if (const char *e = std::getenv("CORR_TUNE_CACHE")) return std::strcmp(e, "off") == 0 ? std::string() : e;
    std::string base;
    if (const char *x = std::getenv("XDG_CACHE_HOME"); x && *x)
        base = x;
    else if (const char *home = std::getenv("HOME"); home && *home)
        base = std::string(home) + "/.cache";
    else
        return std::string();
    return base + "/corr_gb300/tune.txt";
}

// "<build> <gpu name> <SMs> <dtype> <pols> <S> <T> <units>" (spaces in the
// build and GPU name become '_').
std::string tune_line_key(const corr_plan *h)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, h->device);
    std::string name = prop.name, build = kBuildId;
    for (char &c : name) if (c == ' ') c = '_';
    for (char &c : build) if (c == ' ') c = '_';
    const corr_desc_t &d = h->d;
    char buf[512];
    snprintf(buf, sizeof(buf), "%s %s %d %d %d %d %d %lld", build.c_str(), name.c_str(), h->sm_count, (int)d.dtype,
             d.n_pols, d.n_stations, d.n_samples, (long long)d.n_channels * d.n_integrations);
    return buf;
}

bool tune_file_lookup(const corr_plan *h, TileCfg *out)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return false;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    const std::string key = tune_line_key(h);
    char line[640];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        const size_t n = key.size();
        if (std::strncmp(line, key.c_str(), n) != 0 || line[n] != ' ') continue;
        int v = -1, t = -1, l = -1;
        if (std::sscanf(line + n, "%d %d %d", &v, &t, &l) == 3 && v >= 0 && v < TC_N_VARIANTS &&
            (t == TC_NARROW || t == TC_WIDE) && (l == 0 || l == 1) &&
            !(v == TC_PAIR && h->pair_clusters < 1)) {
            out->variant = v;
            out->tail = t;
            out->layout = has_layouts(h->d) ? l : 0;
            found = true;   // the last matching line wins
        }
    }
    std::fclose(f);
    return found;
}

void tune_file_append(const corr_plan *h, const TileCfg &c)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos && slash > 0) {
        // create the directory (and, one level up, its parent) if missing
        const std::string dir = path.substr(0, slash);
        const size_t up = dir.rfind('/');
        if (up != std::string::npos && up > 0) mkdir(dir.substr(0, up).c_str(), 0755);
        mkdir(dir.c_str(), 0755);
    }
    const std::string line = tune_line_key(h) + " " + std::to_string(c.variant) + " " + std::to_string(c.tail) +
                             " " + std::to_string(c.layout) + "\n";
    // one write() of a short line to a file opened for appending
    const int fd = open(path.c_str(), O_WRONLY | O_CREAT | O_APPEND, 0644);
    if (fd < 0) return;
    const ssize_t w = write(fd, line.data(), line.size());
    (void)w;
    close(fd);
}

corr_status_t tune_tensor_config(corr_plan *h)
{
    const corr_desc_t &d = h->d;
    const int S_items = item_stations(d.n_stations, d.n_pols);
    bool forced = false;
    const TileCfg rule = rule_cfg(h, S_items);
    const TileCfg f = apply_forced(h, rule, &forced);
    if (forced) {
        h->tc = f;
        h->tune_source = TUNE_FORCED;
        return CORR_OK;
    }
    if ((d.flags & CORR_FLAG_NO_AUTOTUNE) || d.n_samples == 0) {
        h->tc = rule;
        h->tune_source = TUNE_RULE;
        return CORR_OK;
    }
    const long long units = (long long)d.n_channels * d.n_integrations;
    const TuneKey key{h->device, d.dtype, d.n_pols, d.n_stations, d.n_samples, units};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->tc = it->second;
            h->tune_source = TUNE_MEMORY;
            return CORR_OK;
        }
    }
    TileCfg cached;
    if (tune_file_lookup(h, &cached)) {
        h->tc = cached;
        h->tune_source = TUNE_FILE;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = cached;
        return CORR_OK;
    }
    const std::vector<TileCfg> cands = tune_candidates(h, {std::make_tuple(S_items, d.n_samples, units)});
    // The plan's own unit count, up to 2 GB of samples and visibilities: the
    // configurations' wave quantisation at the real size decides (the pair
    // variant splits its work over two launches). If that memory is not
    // free, a quarter of it, and otherwise the size rule.
    const long long fit = std::max(1LL, (2048LL << 20) / (long long)(in_unit_bytes(d) + out_unit_bytes(d)));
    int su = (int)std::max(1LL, std::min(units, fit));
    void *d_in = nullptr, *d_out = nullptr;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (cudaMalloc(&d_in, (size_t)su * in_unit_bytes(d)) == cudaSuccess &&
            cudaMalloc(&d_out, (size_t)su * out_unit_bytes(d)) == cudaSuccess)
            break;
        cudaGetLastError();
        cudaFree(d_in);
        d_in = d_out = nullptr;
        su = std::max(1, su / 4);
    }
    if (!d_in || !d_out) {
        h->tc = rule;
        h->tune_source = TUNE_RULE;
        return CORR_OK;
    }
    const size_t words = (size_t)su * in_unit_bytes(d) / 4;
    tune_fill_kernel<<<std::max(1, 4 * h->sm_count), 256>>>(static_cast<uint32_t *>(d_in), words,
                                                            d.dtype == CORR_CF16 ? 1 : 0, 1702844u);
    corr_status_t st = cuda_status(cudaGetLastError());
    h->tune_cfgs.clear();
    h->tune_ms.clear();
    for (const TileCfg &c : cands) {
        if (st != CORR_OK) break;
        float ms = 0.f;
        st = time_config(h, c, d.n_stations, d.n_samples, su, d_in, d_out, &ms);
        if (st == CORR_OK) {
            h->tune_cfgs.push_back(c);
            h->tune_ms.push_back(ms);
        }
    }
    cudaFree(d_in);
    cudaFree(d_out);
    if (st != CORR_OK) return st;
    size_t best = 0;
    for (size_t i = 1; i < h->tune_ms.size(); ++i)
        if (h->tune_ms[i] < h->tune_ms[best]) best = i;
    h->tc = h->tune_cfgs.empty() ? rule : h->tune_cfgs[best];
    h->tune_source = TUNE_TIMED;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = h->tc;
    tune_file_append(h, h->tc);
    return CORR_OK;
}

} // namespace

void corr::set_last_error(cudaError_t e)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

void corr::set_last_error(const char *msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

extern "C" {

const char *corr_status_string(corr_status_t s)
{
    switch (s) {
    case CORR_OK: return "ok";
    case CORR_ERR_INVALID_ARG: return "invalid argument";
    case CORR_ERR_UNSUPPORTED: return "unsupported";
    case CORR_ERR_NO_MEMORY: return "out of memory";
    case CORR_ERR_CUDA: return "CUDA error";
    case CORR_ERR_TIMEOUT: return "kernel gave up waiting (timeout)";
    }
    return "unknown status";
}

const char *corr_last_error_message(void) { return g_last_error; }

void corr_tile_cost(int w, int h, long *flops, long *bytes, long *regs)
{
    if (flops) *flops = 32L * w * h;
    if (bytes) *bytes = 16L * (w + h);
    if (regs) *regs = 4L * (1 + std::min(w, h)) + 8L * w * h;
}

int corr_tc_schedule(int variant, int tail_kind, int n_stations, int cap, int *out)
{
    if (n_stations < 1 || variant < TC_NARROW || variant > TC_PAIR || cap < 0) return -1;
    if (tail_kind != TC_NARROW && tail_kind != TC_WIDE) return -1;
    std::vector<int4> tail;
    const std::vector<int4> items = tc_items_for(0, n_stations, 1, variant, &tail, tail_kind);
    const int n = (int)(items.size() + tail.size());
    if (!out) return n;
    if (n > cap) return -1;
    int k = 0;
    for (int t = 0; t < 2; ++t)
        for (const int4 &it : t ? tail : items) {
            out[4 * k + 0] = it.z;
            out[4 * k + 1] = it.w & 0xFFFF;
            out[4 * k + 2] = it.w >> 16;
            out[4 * k + 3] = t;
            ++k;
        }
    return n;
}

int corr_tc_tiles(int S)
{
    if (S <= 0) return 0;
    const int nb = tc_blocks(S);
    return nb * (nb + 1) / 2;
}

int corr_tc_tile_decode(int S, int k, int *rb, int *cb)
{
    const int nb = tc_blocks(S);
    if (S <= 0 || k < 0 || k >= nb * (nb + 1) / 2) return -1;
    // order of tc_items_for: column block major, row block 0..cb
    int c = 0;
    while (k > c) {
        k -= c + 1;
        ++c;
    }
    if (rb) *rb = k;
    if (cb) *cb = c;
    return 0;
}

int corr_fp32_subtiles(int S)
{
    if (S <= 0) return 0;
    const int nq = (S + 3) / 4;
    return nq * (nq + 1) / 2;
}

int corr_fp32_subtile_decode(int S, int k, int *i, int *j)
{
    const int nq = (S + 3) / 4;
    if (S <= 0 || k < 0 || k >= nq * (nq + 1) / 2) return -1;
    int row = 0, off = 0;
    while (k >= off + (nq - row)) {
        off += nq - row;
        ++row;
    }
    if (i) *i = row;
    if (j) *j = row + (k - off);
    return 0;
}

corr_status_t corr_create(const corr_desc_t *desc, corr_handle_t *out)
{
    if (!out) return CORR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc) return CORR_ERR_INVALID_ARG;
    const corr_desc_t &d = *desc;
    if (d.n_stations < 1 || d.n_channels < 1 || d.n_samples < 0 || d.n_integrations < 1)
        return CORR_ERR_INVALID_ARG;
    if (d.n_pols != 1 && d.n_pols != 2) return CORR_ERR_UNSUPPORTED;
    if (d.dtype < CORR_CF32 || d.dtype > CORR_CI8) return CORR_ERR_INVALID_ARG;
    if (d.path < CORR_PATH_AUTO || d.path > CORR_PATH_TENSOR) return CORR_ERR_INVALID_ARG;
    int path = d.path;
    if (path == CORR_PATH_AUTO) path = d.dtype == CORR_CF32 ? CORR_PATH_FP32 : CORR_PATH_TENSOR;
    if (path == CORR_PATH_FP32 && d.dtype != CORR_CF32) return CORR_ERR_UNSUPPORTED;
    // FP32 samples on the tensor cores: the tf32-split kernel (two pols)
    if (path == CORR_PATH_TENSOR && d.dtype == CORR_CF32) {
        if (d.n_pols != 2) return CORR_ERR_UNSUPPORTED;
        path = PATH_TF32;
    }
    if (d.dtype == CORR_CI8 && d.n_samples > 65535) return CORR_ERR_UNSUPPORTED; // int32 range
    const long long units = (long long)d.n_channels * d.n_integrations;
    if (units > (1LL << 30) || d.n_stations > 65535) return CORR_ERR_UNSUPPORTED;
    if ((d.flags & CORR_FLAG_GAINS) && (d.dtype != CORR_CF32 || d.n_pols != 2)) return CORR_ERR_UNSUPPORTED;

    corr_plan *h = new (std::nothrow) corr_plan();
    if (!h) return CORR_ERR_NO_MEMORY;
    h->d = d;
    h->path = path;
    if (const char *e = std::getenv("CORR_WAIT_LIMIT_NS")) h->wait_ns = std::strtoull(e, nullptr, 10);
    corr_status_t st = CORR_OK;
    do {
        if ((st = cuda_status(cudaGetDevice(&h->device))) != CORR_OK) break;
        if ((st = cuda_status(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount,
                                                     h->device))) != CORR_OK)
            break;
        if ((st = cuda_status(cudaMalloc(&h->d_err, sizeof(int)))) != CORR_OK) break;
        if ((st = cuda_status(cudaMemset(h->d_err, 0, sizeof(int)))) != CORR_OK) break;
        if (path == CORR_PATH_TENSOR) {
            // an odd SM count or a cluster that does not fit leaves the pair
            // variant out (0 clusters)
            int n = 0;
            if (tc_pair_max_clusters(d.dtype, &n) != cudaSuccess) {
                cudaGetLastError();
                n = 0;
            }
            h->pair_clusters = std::min(n, h->sm_count / 2);
        }
        if (path == CORR_PATH_FP32) {
            fp32_config(h);
            if (h->fp.ksplit > 1 &&
                (st = cuda_status(cudaMalloc(&h->d_fp_partial, (size_t)h->fp.ksplit * units *
                                                                   out_unit_bytes(d)))) != CORR_OK)
                break;
        } else if (path == PATH_TF32) {
            const long long nb = (d.n_stations + 63) / 64, ntri = nb * (nb + 1) / 2;
            if (tf_chunks(d.n_samples) > 1 && units * ntri < 2LL * h->sm_count &&
                (st = cuda_status(cudaMalloc(&h->d_tf_partial, (size_t)tf_chunks(d.n_samples) * units *
                                                                   out_unit_bytes(d)))) != CORR_OK)
                break;
        } else if (path == CORR_PATH_TENSOR) {
            if ((st = tune_tensor_config(h)) != CORR_OK) break;
            std::vector<int4> tail;
            std::vector<int4> items =
                tc_items_for(0, item_stations(d.n_stations, d.n_pols), (int)units, h->tc.variant, &tail, h->tc.tail);
            h->n_items = (int)items.size();
            h->n_tail = (int)tail.size();
            items.insert(items.end(), tail.begin(), tail.end());
            if ((st = cuda_status(cudaMalloc(&h->d_items, items.size() * sizeof(int4)))) != CORR_OK)
                break;
            if ((st = cuda_status(cudaMemcpy(h->d_items, items.data(), items.size() * sizeof(int4),
                                             cudaMemcpyHostToDevice))) != CORR_OK)
                break;
            if (d.dtype == CORR_CI8 && (st = ensure_redo(h, h->n_items + h->n_tail)) != CORR_OK) break;
        }
        if (d.flags & CORR_FLAG_HOST_IO) {
            // chunks of about 32 MiB of input (CORR_HOST_CHUNK_MB overrides;
            // at least one channel), and on the FP32 path at least one full
            // wave of its CTAs (two per SM, `groups` per channel): each chunk
            // is its own launch, and a FP32 CTA takes one channel, so small
            // channels would leave most SMs idle
            size_t chunk_mb = 32;
            if (const char *e = std::getenv("CORR_HOST_CHUNK_MB")) chunk_mb = std::max(1ul, std::strtoul(e, nullptr, 10));
            const size_t ub = std::max<size_t>(1, in_unit_bytes(d));
            long long cu = (long long)((chunk_mb << 20) / ub);
            if (h->path == CORR_PATH_FP32)
                cu = std::max<long long>(cu, (2LL * h->sm_count + h->fp.groups - 1) / h->fp.groups);
            if (h->path == PATH_TF32) {   // a tile per CTA and SM: at least one wave of tiles
                const long long nb = (d.n_stations + 63) / 64, ntri = nb * (nb + 1) / 2;
                cu = std::max<long long>(cu, (h->sm_count + ntri - 1) / ntri);
            }
            h->chunk_units = (int)std::max<long long>(1, std::min<long long>(units, cu));
            const size_t ib = (size_t)h->chunk_units * in_unit_bytes(d);
            const size_t ob = (size_t)h->chunk_units * out_unit_bytes(d);
            for (int b = 0; b < 2 && st == CORR_OK; ++b) {
                st = cuda_status(cudaMalloc(&h->d_stage_in[b], std::max<size_t>(ib, 16)));
                if (st == CORR_OK) st = cuda_status(cudaMalloc(&h->d_stage_out[b], ob));
                if (st == CORR_OK) st = cuda_status(cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming));
                if (st == CORR_OK) st = cuda_status(cudaEventCreateWithFlags(&h->ev_comp[b], cudaEventDisableTiming));
                if (st == CORR_OK) st = cuda_status(cudaEventCreateWithFlags(&h->ev_out[b], cudaEventDisableTiming));
            }
            if (st == CORR_OK) st = cuda_status(cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming));
            if (st == CORR_OK) st = cuda_status(cudaStreamCreateWithFlags(&h->s_h2d, cudaStreamNonBlocking));
            if (st == CORR_OK) st = cuda_status(cudaStreamCreateWithFlags(&h->s_d2h, cudaStreamNonBlocking));
            if (st != CORR_OK) break;
        }
        if (d.flags & CORR_FLAG_GAINS) {
            const long long S = d.n_stations, N = 2 * S;
            if ((st = cuda_status(cudaMalloc(&h->d_R, (size_t)(units * n_baselines(S) * 4 * 8)))) != CORR_OK) break;
            if ((st = cuda_status(cudaMalloc(&h->d_W, (size_t)(units * N * N * 8)))) != CORR_OK) break;
            // the tensor-core input gradient's tiles; their padding (rows or
            // columns past 4S) is never written: zeroed once
            const size_t tb = ig_tile_bytes((int)S, units);
            if ((st = cuda_status(cudaMalloc(&h->d_At, tb))) != CORR_OK) break;
            if ((st = cuda_status(cudaMemset(h->d_At, 0, tb))) != CORR_OK) break;
            if ((st = cuda_status(cudaMalloc(&h->d_partial, (size_t)units * sizeof(float)))) != CORR_OK) break;
        }
    } while (0);
    if (st != CORR_OK) {
        corr_destroy(h);
        return st;
    }
    *out = h;
    return CORR_OK;
}

corr_status_t corr_correlate(corr_handle_t h, const void *d_in, void *d_out, void *stream)
{
    if (!h || !d_out || !aligned16(d_out)) return CORR_ERR_INVALID_ARG;
    if (h->d.n_samples > 0 && (!d_in || !aligned16(d_in))) return CORR_ERR_INVALID_ARG;
    return launch_correlate(h, d_in, d_out, static_cast<cudaStream_t>(stream));
}

corr_status_t corr_correlate_host(corr_handle_t h, const void *h_in, void *h_out, void *stream)
{
    if (!h || !h_out || !(h->d.flags & CORR_FLAG_HOST_IO)) return CORR_ERR_INVALID_ARG;
    const corr_desc_t &d = h->d;
    if (d.n_samples > 0 && !h_in) return CORR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long units = (long long)d.n_channels * d.n_integrations;
    const long long cu = h->chunk_units;
    const long long nch = (units + cu - 1) / cu;
    const size_t ib = in_unit_bytes(d), ob = out_unit_bytes(d);
    corr_status_t st = cuda_status(cudaEventRecord(h->ev_start, s));
    if (st == CORR_OK) st = cuda_status(cudaStreamWaitEvent(h->s_h2d, h->ev_start, 0));
    if (st == CORR_OK) st = cuda_status(cudaStreamWaitEvent(h->s_d2h, h->ev_start, 0));
    for (long long i = 0; i < nch && st == CORR_OK; ++i) {
        const int b = (int)(i & 1);
        const long long u0 = i * cu;
        const long long nu = std::min(cu, units - u0);
        // staging buffer b was last read by the kernel of chunk i-2 and its
        // output last copied out by the D2H of chunk i-2
        if (i >= 2) st = cuda_status(cudaStreamWaitEvent(h->s_h2d, h->ev_comp[b], 0));
        if (st == CORR_OK && ib * nu > 0)
            st = cuda_status(cudaMemcpyAsync(h->d_stage_in[b],
                                             static_cast<const char *>(h_in) + (size_t)u0 * ib,
                                             (size_t)nu * ib, cudaMemcpyHostToDevice, h->s_h2d));
        if (st == CORR_OK) st = cuda_status(cudaEventRecord(h->ev_in[b], h->s_h2d));
        if (st == CORR_OK) st = cuda_status(cudaStreamWaitEvent(s, h->ev_in[b], 0));
        if (st == CORR_OK && i >= 2) st = cuda_status(cudaStreamWaitEvent(s, h->ev_out[b], 0));
        if (st == CORR_OK) st = launch_units(h, h->d_stage_in[b], h->d_stage_out[b], nu, s);
        if (st == CORR_OK) st = cuda_status(cudaEventRecord(h->ev_comp[b], s));
        if (st == CORR_OK) st = cuda_status(cudaStreamWaitEvent(h->s_d2h, h->ev_comp[b], 0));
        if (st == CORR_OK)
            st = cuda_status(cudaMemcpyAsync(static_cast<char *>(h_out) + (size_t)u0 * ob,
                                             h->d_stage_out[b], (size_t)nu * ob,
                                             cudaMemcpyDeviceToHost, h->s_d2h));
        if (st == CORR_OK) st = cuda_status(cudaEventRecord(h->ev_out[b], h->s_d2h));
    }
    // the caller's stream completes only after every copy back
    for (int b = 0; b < 2 && st == CORR_OK && b < nch; ++b)
        st = cuda_status(cudaStreamWaitEvent(s, h->ev_out[b], 0));
    return st;
}

} // extern "C"

namespace {

// Work list of a ragged batch in tile variant v: tiles of all sub-arrays,
// heaviest (longest integration) first so that the static round-robin split
// over the persistent CTAs ends evenly; the narrow tail items last.
corr_status_t batch_items(corr_plan *h, int n_sub, const corr_subarray_t *subs, const TileCfg &cfg)
{
    std::vector<int4> items, tail;
    std::vector<int> T(n_sub);
    for (int i = 0; i < n_sub; ++i) {
        T[i] = subs[i].n_samples;
        if (subs[i].n_samples == 0) continue;
        std::vector<int4> u = tc_items_for(i, item_stations(subs[i].n_stations, h->d.n_pols),
                                           subs[i].n_channels, cfg.variant, &tail, cfg.tail);
        items.insert(items.end(), u.begin(), u.end());
    }
    auto heavier = [&](const int4 &a, const int4 &b) { return T[a.x] > T[b.x]; };
    std::stable_sort(items.begin(), items.end(), heavier);
    std::stable_sort(tail.begin(), tail.end(), heavier);
    h->n_btail = (int)tail.size();
    h->n_bitems = (int)items.size();
    items.insert(items.end(), tail.begin(), tail.end());
    cudaFree(h->d_bitems);
    h->d_bitems = nullptr;
    corr_status_t e;
    if (!items.empty()) {
        if ((e = cuda_status(cudaMalloc(&h->d_bitems, items.size() * sizeof(int4)))) != CORR_OK) return e;
        if ((e = cuda_status(cudaMemcpy(h->d_bitems, items.data(), items.size() * sizeof(int4),
                                        cudaMemcpyHostToDevice))) != CORR_OK)
            return e;
    }
    if (h->d.dtype == CORR_CI8 && (e = ensure_redo(h, h->n_bitems + h->n_btail)) != CORR_OK) return e;
    return CORR_OK;
}

corr_status_t run_batch(corr_plan *h, int max_T, cudaStream_t st)
{
    if (h->n_bitems + h->n_btail == 0) return CORR_OK;
    TcParams p{};
    p.probs = h->d_bprobs;
    p.items = h->d_bitems;
    p.n_items = h->n_bitems;
    p.err = h->d_err;
    p.wait_ns = h->wait_ns;
    return run_tensor(h, p, h->d_bitems + h->n_bitems, h->n_btail, h->d.dtype, h->bc, max_T, st);
}

// One warm-up run and one timed run of the current batch work list.
corr_status_t time_batch(corr_plan *h, int max_T, cudaStream_t st, float *ms_out)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    corr_status_t e = CORR_OK;
    do {
        if ((e = cuda_status(cudaEventCreate(&e0))) != CORR_OK) break;
        if ((e = cuda_status(cudaEventCreate(&e1))) != CORR_OK) break;
        if ((e = run_batch(h, max_T, st)) != CORR_OK) break;
        if ((e = cuda_status(cudaEventRecord(e0, st))) != CORR_OK) break;
        if ((e = run_batch(h, max_T, st)) != CORR_OK) break;
        if ((e = cuda_status(cudaEventRecord(e1, st))) != CORR_OK) break;
        if ((e = cuda_status(cudaEventSynchronize(e1))) != CORR_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *ms_out = ms;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

} // namespace

extern "C" {

corr_status_t corr_correlate_batched(corr_handle_t h, int n_sub, const corr_subarray_t *subs,
                                     void *stream)
{
    if (!h || n_sub < 0 || (n_sub > 0 && !subs)) return CORR_ERR_INVALID_ARG;
    if (h->d.dtype == CORR_CF32) return CORR_ERR_UNSUPPORTED;
    if (n_sub == 0) return CORR_OK;
    for (int i = 0; i < n_sub; ++i) {
        const corr_subarray_t &s = subs[i];
        if (s.n_stations < 1 || s.n_channels < 1 || s.n_samples < 0 || s.reserved != 0 ||
            !s.d_out || !aligned16(s.d_out))
            return CORR_ERR_INVALID_ARG;
        if (s.n_samples > 0 && (!s.d_in || !aligned16(s.d_in))) return CORR_ERR_INVALID_ARG;
        if (h->d.dtype == CORR_CI8 && s.n_samples > 65535) return CORR_ERR_UNSUPPORTED;
        if (s.n_stations > 65535) return CORR_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool same = (int)h->batch_key.size() == n_sub;
    for (int i = 0; same && i < n_sub; ++i)
        same = std::memcmp(&h->batch_key[i], &subs[i], sizeof(corr_subarray_t)) == 0;
    int max_T = 0;
    for (int i = 0; i < n_sub; ++i) max_T = std::max(max_T, subs[i].n_samples);
    if (!same) {
        h->batch_key.clear();
        std::vector<TcProblem> probs;
        for (int i = 0; i < n_sub; ++i) {
            const corr_subarray_t &s = subs[i];
            probs.push_back(make_problem(s.d_in, s.d_out, s.n_stations, s.n_samples, s.n_channels,
                                         h->d.dtype, h->d.n_pols));
        }
        cudaFree(h->d_bprobs);
        h->d_bprobs = nullptr;
        corr_status_t e;
        if ((e = cuda_status(cudaMalloc(&h->d_bprobs, probs.size() * sizeof(TcProblem)))) != CORR_OK) return e;
        if ((e = cuda_status(cudaMemcpy(h->d_bprobs, probs.data(), probs.size() * sizeof(TcProblem),
                                        cudaMemcpyHostToDevice))) != CORR_OK)
            return e;
        // One tile configuration serves the whole batch. Parts forced by
        // CORR_TC_VARIANT / CORR_TC_TAIL / CORR_TC_LAYOUT; otherwise the
        // candidates the cost model keeps are timed on this batch (two
        // rounds; each run warms up once and times once; the sub-arrays'
        // outputs are simply overwritten), unless the plan skips tuning or
        // the stream is being captured, where the size rule decides: pair
        // tiles (wide if pairs do not fit) when most of the work is in
        // sub-arrays of >= 128 stations, with the wide tail.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if ((e = cuda_status(cudaStreamIsCapturing(st, &cap))) != CORR_OK) return e;
        const int big_v = h->pair_clusters > 0 ? TC_PAIR : TC_WIDE;
        h->b_tune_cfgs.clear();
        h->b_tune_ms.clear();
        double big = 0, all = 0;
        std::vector<std::tuple<int, int, long long>> shapes;
        for (int i = 0; i < n_sub; ++i) {
            const double w = (double)n_baselines(subs[i].n_stations) * subs[i].n_samples * subs[i].n_channels;
            all += w;
            if (subs[i].n_stations >= 128) big += w;
            if (subs[i].n_samples > 0)
                shapes.emplace_back(item_stations(subs[i].n_stations, h->d.n_pols), subs[i].n_samples,
                                    (long long)subs[i].n_channels);
        }
        TileCfg rule;
        rule.variant = big >= 0.5 * all ? big_v : TC_NARROW;
        rule.tail = TC_WIDE;
        rule.layout = 0;
        bool forced = false;
        h->bc = apply_forced(h, rule, &forced);
        if (!forced && !(h->d.flags & CORR_FLAG_NO_AUTOTUNE) && cap == cudaStreamCaptureStatusNone && max_T > 0) {
            // two rounds over the candidates, each one's best time counts;
            // within 2% of the best, the size rule's choice stays
            const std::vector<TileCfg> cands = tune_candidates(h, shapes);
            h->b_tune_cfgs = cands;
            h->b_tune_ms.assign(cands.size(), 0.f);
            for (int round = 0; round < 2; ++round)
                for (size_t i = 0; i < cands.size(); ++i) {
                    h->bc = cands[i];
                    if ((e = batch_items(h, n_sub, subs, h->bc)) != CORR_OK) return e;
                    float ms = 0.f;
                    if ((e = time_batch(h, max_T, st, &ms)) != CORR_OK) return e;
                    if (round == 0 || ms < h->b_tune_ms[i]) h->b_tune_ms[i] = ms;
                }
            size_t best = cands.size();
            float rule_ms = 0.f;
            for (size_t i = 0; i < cands.size(); ++i)
                if (cands[i].variant == rule.variant && cands[i].tail == rule.tail && cands[i].layout == rule.layout)
                    rule_ms = h->b_tune_ms[i];
            for (size_t i = 0; i < cands.size(); ++i)
                if (best == cands.size() || h->b_tune_ms[i] < h->b_tune_ms[best]) best = i;
            h->bc = (rule_ms > 0.f && h->b_tune_ms[best] >= 0.98f * rule_ms) || best == cands.size() ? rule
                                                                                                     : cands[best];
        }
        if ((e = batch_items(h, n_sub, subs, h->bc)) != CORR_OK) return e;
        h->batch_key.assign(subs, subs + n_sub);
    }
    for (int i = 0; i < n_sub; ++i)
        if (subs[i].n_samples == 0) {
            const size_t bytes = (size_t)subs[i].n_channels * n_baselines(subs[i].n_stations) *
                                 h->d.n_pols * h->d.n_pols * 8;
            corr_status_t e = cuda_status(cudaMemsetAsync(subs[i].d_out, 0, bytes, st));
            if (e != CORR_OK) return e;
        }
    return run_batch(h, max_T, st);
}

corr_status_t corr_gain_loss(corr_handle_t h, const void *d_raw_vis, const void *d_gain,
                             const void *d_vis_model, void *d_vis_out, float *d_loss, void *stream)
{
    if (!h || !d_raw_vis || !d_gain || !d_vis_model) return CORR_ERR_INVALID_ARG;
    if (!(h->d.flags & CORR_FLAG_GAINS)) return CORR_ERR_INVALID_ARG;
    if (!aligned_to(d_raw_vis, 8) || !aligned_to(d_gain, 8) || !aligned_to(d_vis_model, 8) ||
        !aligned_to(d_vis_out, 8) || !aligned_to(d_loss, 4))
        return CORR_ERR_INVALID_ARG;
    const int units = h->d.n_channels * h->d.n_integrations;
    return cuda_status(gain_loss_launch(static_cast<const float2 *>(d_raw_vis),
                                        static_cast<const float2 *>(d_gain),
                                        static_cast<const float2 *>(d_vis_model),
                                        static_cast<float2 *>(d_vis_out), h->d_partial, d_loss,
                                        h->d.n_stations, units, static_cast<cudaStream_t>(stream)));
}

corr_status_t corr_gain_backward(corr_handle_t h, const void *d_in, const void *d_gain,
                                 const void *d_vis_model, const void *d_raw_vis, void *d_grad_gain,
                                 void *d_grad_in, float *d_loss, const float *d_grad_scale,
                                 void *stream)
{
    if (!h || !d_gain || !d_vis_model || !d_grad_gain) return CORR_ERR_INVALID_ARG;
    if (!(h->d.flags & CORR_FLAG_GAINS)) return CORR_ERR_INVALID_ARG;
    if ((!d_raw_vis || d_grad_in) && !d_in) return CORR_ERR_INVALID_ARG;
    if (!aligned_to(d_in, 8) || !aligned_to(d_gain, 8) || !aligned_to(d_vis_model, 8) ||
        !aligned_to(d_raw_vis, 8) || !aligned_to(d_grad_gain, 8) || !aligned_to(d_grad_in, 8) ||
        !aligned_to(d_loss, 4) || !aligned_to(d_grad_scale, 4))
        return CORR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int units = h->d.n_channels * h->d.n_integrations;
    const int S = h->d.n_stations;
    const float2 *R = static_cast<const float2 *>(d_raw_vis);
    if (!R) {
        corr_status_t e = corr_correlate(h, d_in, h->d_R, stream);
        if (e != CORR_OK) return e;
        R = h->d_R;
    }
    const float2 *g = static_cast<const float2 *>(d_gain);
    const float2 *M = static_cast<const float2 *>(d_vis_model);
    // The input gradient on the tensor cores (tf32 split, FP32 accuracy)
    // when the samples and the gradient are 16-byte aligned (TMA loads,
    // 16-byte stores), on CTA pairs when there are two row tiles or more;
    // otherwise, or with CORR_IG_PATH=cuda_core, the FP32 CUDA-core GEMM.
    // CORR_IG_PATH=tc1 keeps the tensor-core path on single CTAs.
    const char *ig = std::getenv("CORR_IG_PATH");
    const bool ig_pair = ig_m_tiles(S) >= 2 && !(ig && std::strcmp(ig, "tc1") == 0);
    const bool tc = d_grad_in && h->d.n_samples > 0 && aligned16(d_in) &&
                    aligned16(d_grad_in) && !(ig && std::strcmp(ig, "cuda_core") == 0);
    CUtensorMap xmap{};
    if (tc) {
        corr_status_t e = encode_ig_map(&xmap, d_in, S, h->d.n_samples, units);
        if (e != CORR_OK) return e;
    }
    corr_status_t e = cuda_status(gain_grad_launch(R, g, M, d_grad_scale, static_cast<float2 *>(d_grad_gain),
                                                   tc ? static_cast<void *>(h->d_At) : (d_grad_in ? h->d_W : nullptr),
                                                   S, units, st, tc ? 1 : 0));
    if (e != CORR_OK) return e;
    if (d_grad_in && tc) {
        IgParams ip{};
        ip.at = h->d_At;
        ip.gx = static_cast<float2 *>(d_grad_in);
        ip.S = S;
        ip.T = h->d.n_samples;
        ip.units = units;
        ip.m_tiles = ig_m_tiles(S);
        ip.m_alloc = ig_m_alloc(S);
        ip.k_blocks = ig_k_blocks(S);
        ip.err = h->d_err;
        ip.wait_ns = h->wait_ns;
        e = cuda_status(input_grad_tc_launch(&xmap, ip, st, ig_pair));
        if (e != CORR_OK) return e;
    } else if (d_grad_in) {
        e = cuda_status(input_grad_launch(static_cast<const float2 *>(d_in), h->d_W,
                                          static_cast<float2 *>(d_grad_in), S, h->d.n_samples, units, st));
        if (e != CORR_OK) return e;
    }
    if (d_loss)
        e = cuda_status(gain_loss_launch(R, g, M, nullptr, h->d_partial, d_loss, S, units, st));
    return e;
}

corr_status_t corr_reorder(int n_stations, int n_channels, int n_samples, int n_integrations,
                           corr_dtype_t dtype, corr_layout_t from, corr_layout_t to,
                           const void *d_in, void *d_out, void *stream)
{
    if (n_stations < 0 || n_channels < 0 || n_samples < 0 || n_integrations < 1)
        return CORR_ERR_INVALID_ARG;
    if (dtype < CORR_CF32 || dtype > CORR_CI8) return CORR_ERR_INVALID_ARG;
    if (from < CORR_LAYOUT_CST || from > CORR_LAYOUT_SCT || to < CORR_LAYOUT_CST || to > CORR_LAYOUT_SCT)
        return CORR_ERR_INVALID_ARG;
    const int eb = bytes_per_sample(dtype);
    const unsigned long long elems =
        (unsigned long long)n_integrations * n_channels * n_stations * n_samples;
    if (elems == 0) return CORR_OK;
    if (!d_in || !d_out) return CORR_ERR_INVALID_ARG;
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
    if (a % eb != 0 || b % eb != 0) return CORR_ERR_INVALID_ARG;
    const unsigned long long bytes = elems * eb;
    if (a < b + bytes && b < a + bytes) return CORR_ERR_INVALID_ARG; // overlap
    int dev = 0, sms = 0;
    corr_status_t st = cuda_status(cudaGetDevice(&dev));
    if (st == CORR_OK) st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (st != CORR_OK) return st;
    return cuda_status(reorder_launch(d_in, d_out, n_stations, n_channels, n_samples, n_integrations,
                                      eb, from, to, sms, static_cast<cudaStream_t>(stream)));
}

int corr_tile_variant(corr_handle_t h)
{
    if (!h) return -1;
    return h->path == CORR_PATH_TENSOR ? h->tc.variant : -1;
}

int corr_batch_tile_variant(corr_handle_t h)
{
    if (!h || h->batch_key.empty()) return -1;
    return h->bc.variant;
}

corr_status_t corr_tile_config(corr_handle_t h, int *variant, int *tail, int *layout, int *source)
{
    if (!h || h->path != CORR_PATH_TENSOR) return CORR_ERR_INVALID_ARG;
    if (variant) *variant = h->tc.variant;
    if (tail) *tail = h->tc.tail;
    if (layout) *layout = h->tc.layout;
    if (source) *source = h->tune_source;
    return CORR_OK;
}

int corr_tune_results(corr_handle_t h, int batch, int cap, int *cfg, float *ms)
{
    if (!h || cap < 0) return -1;
    const std::vector<TileCfg> &c = batch ? h->b_tune_cfgs : h->tune_cfgs;
    const std::vector<float> &t = batch ? h->b_tune_ms : h->tune_ms;
    const int n = (int)c.size();
    for (int i = 0; i < n && i < cap; ++i) {
        if (cfg) {
            cfg[3 * i + 0] = c[i].variant;
            cfg[3 * i + 1] = c[i].tail;
            cfg[3 * i + 2] = c[i].layout;
        }
        if (ms) ms[i] = t[i];
    }
    return n;
}

corr_status_t corr_set_kernel_events(corr_handle_t h, void *ev_start, void *ev_stop)
{
    if (!h || (!ev_start) != (!ev_stop)) return CORR_ERR_INVALID_ARG;
    h->ev_k0 = static_cast<cudaEvent_t>(ev_start);
    h->ev_k1 = static_cast<cudaEvent_t>(ev_stop);
    return CORR_OK;
}

corr_status_t corr_get_error(corr_handle_t h)
{
    if (!h) return CORR_ERR_INVALID_ARG;
    int v = 0;
    corr_status_t e = cuda_status(cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != CORR_OK) return e;
    if (v) {
        e = cuda_status(cudaMemset(h->d_err, 0, sizeof(int)));
        if (e != CORR_OK) return e;
        return CORR_ERR_TIMEOUT;
    }
    return CORR_OK;
}

corr_status_t corr_destroy(corr_handle_t h)
{
    if (!h) return CORR_OK;
    cudaDeviceSynchronize();
    cudaFree(h->d_err);
    cudaFree(h->d_fp_partial);
    cudaFree(h->d_items);
    cudaFree(h->d_redo_state);
    cudaFree(h->d_redo_index);
    cudaFree(h->d_redo_items);
    cudaFree(h->d_bprobs);
    cudaFree(h->d_bitems);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->d_stage_in[b]);
        cudaFree(h->d_stage_out[b]);
        if (h->ev_in[b]) cudaEventDestroy(h->ev_in[b]);
        if (h->ev_comp[b]) cudaEventDestroy(h->ev_comp[b]);
        if (h->ev_out[b]) cudaEventDestroy(h->ev_out[b]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->s_h2d) cudaStreamDestroy(h->s_h2d);
    if (h->s_d2h) cudaStreamDestroy(h->s_d2h);
    cudaFree(h->d_R);
    cudaFree(h->d_W);
    cudaFree(h->d_At);
    cudaFree(h->d_tf_partial);
    cudaFree(h->d_partial);
    delete h;
    return CORR_OK;
}

} // extern "C"
