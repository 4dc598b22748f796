/*
 * C ABI of the GB300 correlator library (libcorr.so).
 *
 * The operation is the X-step of an FX correlator as stated in Section 2 of
 * van Nieuwpoort & Romein, "Correlating Radio Astronomy Signals with
 * Many-Core Hardware": for every frequency channel, every pair of stations
 * s1 <= s2 (autocorrelations included) and every pair of polarisations
 * p1, p2 in {X, Y},
 *
 *     V[ch][baseline(s1,s2)][p1][p2] = sum_t  x[ch][s1][t][p1] * conj(x[ch][s2][t][p2]),
 *
 * with baseline(s1, s2) = s2*(s2+1)/2 + s1 (the order the loop nest of Fig. 2
 * visits the pairs). There are S(S+1)/2 baselines per channel.
 *
 * Memory layouts (all complex values are (re, im) interleaved):
 *   input  : [integration][channel][station][time][pol]
 *            CORR_CF32 -> 2 x float32, CORR_CF16 -> 2 x float16,
 *            CORR_CI8  -> 2 x int8
 *   output : [integration][channel][baseline][pol1][pol2]
 *            complex float32 for CORR_CF32 / CORR_CF16 inputs,
 *            complex int32 for CORR_CI8 inputs (bit-exact).
 *   gains  : [integration][channel][station][pol], complex float32.
 *
 * Ownership: the caller owns every buffer passed in; all pointers named d_*
 * are device pointers on the plan's device and must be 16-byte aligned.
 * The plan owns its work lists, error word and workspaces; it allocates
 * device memory only in corr_create and on the first call of
 * corr_correlate_batched with a new set of sub-arrays.
 *
 * Calls are asynchronous on the given stream (a cudaStream_t passed as
 * void*, NULL = legacy default stream) and do not synchronize, except where
 * stated. Argument errors are detected on the host before any launch and
 * returned as status codes; nothing aborts or exits. A kernel that gives up
 * waiting on an internal pipeline barrier sets the plan's error word, which
 * corr_get_error reports as CORR_ERR_TIMEOUT.
 *
 * The number of polarisations P is 2 (X and Y, as in the paper) or 1; the
 * loop nest of Fig. 2 takes it as a parameter. With P = 1 the pol axes have
 * length 1: the input is [integration][channel][station][time] and the
 * output [integration][channel][baseline], one complex value per baseline.
 * Gain calibration and corr_reorder take P = 2 only.
 */
#ifndef CORR_H
#define CORR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct corr_plan *corr_handle_t;

typedef enum {
    CORR_OK = 0,
    CORR_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or handle */
    CORR_ERR_UNSUPPORTED = 2, /* valid request this library does not implement */
    CORR_ERR_NO_MEMORY = 3,   /* device or host allocation failed */
    CORR_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    CORR_ERR_TIMEOUT = 5      /* a kernel gave up on a pipeline wait */
} corr_status_t;

typedef enum { CORR_CF32 = 0, CORR_CF16 = 1, CORR_CI8 = 2 } corr_dtype_t;

/* Which kernel family computes the products.
 *   CORR_PATH_FP32   : FP32 CUDA-core kernel (4 FMAs per complex multiply-add,
 *                      Section 2); inputs CORR_CF32 only.
 *   CORR_PATH_TENSOR : tcgen05 tensor-core kernel; CORR_CF16 (FP32
 *                      accumulation) or CORR_CI8 (exact, INT32 result); or
 *                      CORR_CF32 with two pols: every sample split into a
 *                      tf32 value and a tf32 remainder, three tf32 products
 *                      per product term, FP32 accumulation (FP32-class
 *                      accuracy). Not for ragged batches.
 *   CORR_PATH_AUTO   : FP32 for CORR_CF32, TENSOR otherwise. */
typedef enum { CORR_PATH_AUTO = 0, CORR_PATH_FP32 = 1, CORR_PATH_TENSOR = 2 } corr_path_t;

/* Plan flags. */
#define CORR_FLAG_GAINS 0x1u      /* allocate the gain-calibration workspace */
#define CORR_FLAG_NO_AUTOTUNE 0x2u /* skip timed tile selection at create */
#define CORR_FLAG_HOST_IO 0x4u     /* allocate staging for corr_correlate_host */

typedef struct {
    int n_stations;     /* S >= 1                                   (Section 2) */
    int n_pols;         /* 2 (X and Y) or 1                  (Section 2, Fig. 2) */
    int n_channels;     /* C >= 1                                   (Section 2) */
    int n_samples;      /* T >= 0, samples per integration          (Section 2) */
    int n_integrations; /* >= 1, integrations stacked before channels           */
    int dtype;          /* corr_dtype_t of the input samples                     */
    int path;           /* corr_path_t                                            */
    unsigned flags;     /* CORR_FLAG_*                                            */
} corr_desc_t;

/* One sub-array of a ragged batch: its own S, C, T, input and output
 * (layouts as above with one integration). */
typedef struct {
    int n_stations;
    int n_channels;
    int n_samples;
    int reserved; /* must be 0 */
    const void *d_in;
    void *d_out;
} corr_subarray_t;

/* Creates a plan for the problem described by *desc on the current CUDA
 * device. Validates the description, allocates the plan's device work list
 * and error word, and (unless CORR_FLAG_NO_AUTOTUNE) times the candidate tile
 * shapes once for this shape (this synchronizes the device). On success
 * *out receives the handle; on failure *out is set to NULL. */
corr_status_t corr_create(const corr_desc_t *desc, corr_handle_t *out);

/* Correlates all integrations and channels of the plan (Section 2, the
 * correlation formula; Fig. 2). d_in: input samples, layout and type as
 * above, n_integrations*n_channels*n_stations*n_samples*P complex values;
 * d_out: visibilities, n_integrations*n_channels*S(S+1)/2*P*P complex
 * values, fully overwritten. d_in may be NULL when n_samples is 0 (the
 * output is then all zeros). Asynchronous on stream (one to four kernel
 * launches and, for int8 with more than 512 samples, small memsets);
 * capturable in a CUDA graph. */
corr_status_t corr_correlate(corr_handle_t h, const void *d_in, void *d_out, void *stream);

/* corr_correlate with HOST buffers (h_in, h_out: same layouts as above, in
 * host memory; page-locked memory gives overlapped copies). The channels
 * are streamed in chunks of about 32 MiB of input: the host-to-device copy
 * of chunk i+1 and the device-to-host copy of chunk i-1 overlap the kernel
 * of chunk i (two plan-owned staging buffers, two plan-owned copy streams).
 * This is the overlap of transfers and correlation that Section 3.6 and
 * Section 4.4 identify as the bound of a correlator fed over a host link.
 * Requires a plan created with CORR_FLAG_HOST_IO. Asynchronous: everything
 * is ordered before later work on stream, so synchronizing stream covers the
 * whole call. The host buffers must stay valid until then. */
corr_status_t corr_correlate_host(corr_handle_t h, const void *h_in, void *h_out, void *stream);

/* Correlates a ragged batch of n_sub independent sub-arrays (each with its
 * own S, C and T, channels independent as in Section 2) in one persistent
 * kernel launch on the tensor path with the plan's dtype (CORR_CF16 or
 * CORR_CI8) and pol count (one launch per tile kind: with the pair variant,
 * pair tiles and, for sub-arrays with an odd number of 64-station blocks,
 * narrow tiles for the last block column). The plan's own S, C and T are
 * ignored. The first call with a
 * new set of sub-arrays (shapes or pointers) builds and uploads the work
 * list and synchronizes; it must not be captured. It also picks the tile
 * variant for this set by timing each variant on the batch itself (one
 * warm-up and one timed run each, whose results the final run overwrites),
 * unless the plan has CORR_FLAG_NO_AUTOTUNE or CORR_TC_VARIANT forces one;
 * corr_batch_tile_variant reports the choice. Later calls with the same set
 * only launch and are capturable. */
corr_status_t corr_correlate_batched(corr_handle_t h, int n_sub, const corr_subarray_t *subs,
                                     void *stream);

/* Gain-calibration loss (not in the paper; the calibration step that
 * consumes the autocorrelations is named in Section 2). With raw
 * visibilities R = corr(x) from corr_correlate, gains g and model M:
 *     V_ab = g_a conj(g_b) R_ab,   L = sum |V_ab - M_ab|^2
 * over channels, baselines and pol pairs. d_raw_vis, d_vis_model: complex
 * float32 [units][B][2][2]; d_gain: complex float32 [units][S][2];
 * d_vis_out (nullable) receives V; d_loss (nullable) receives L (float32).
 * Complex buffers must be 8-byte aligned, d_loss 4-byte aligned
 * (CORR_ERR_INVALID_ARG otherwise). Requires a plan created with
 * CORR_FLAG_GAINS and dtype CORR_CF32. */
corr_status_t corr_gain_loss(corr_handle_t h, const void *d_raw_vis, const void *d_gain,
                             const void *d_vis_model, void *d_vis_out, float *d_loss,
                             void *stream);

/* Adjoint of corr_gain_loss: gradients in the PyTorch convention for a real
 * loss of complex inputs (dL/dRe + i dL/dIm = 2 dL/d conj(z)), scaled by
 * *d_grad_scale (device float, nullable = 1).
 *   d_grad_gain (required): [units][S][2] complex float32,
 *       dL/d conj(g_c) = sum_(c,b) E_cb g_b conj(R_cb) + sum_(a,c) conj(E_ac) g_a R_ac;
 *   d_grad_in (nullable): same layout as d_in (complex float32),
 *       dL/d conj(x_c(t)) = conj(g_c) sum_b W_cb g_b x_b(t),
 *       W_cb = [s_c<=s_b] E_cb + [s_b<=s_c] conj(E_bc), E = V - M;
 *   d_raw_vis (nullable): R from a previous corr_correlate; recomputed if NULL
 *       (d_in must then be 16-byte aligned, as for corr_correlate);
 *   d_loss (nullable): receives L.
 * Complex buffers must be 8-byte aligned, d_loss and d_grad_scale 4-byte
 * aligned (CORR_ERR_INVALID_ARG otherwise).
 * The input gradient is a GEMM per channel (W' = 2 conj(g) W g times the
 * samples). With d_in and d_grad_in 16-byte aligned and n_samples > 0 it
 * runs on the tensor cores in tf32 with
 * every operand split into a tf32 value and a tf32 remainder (three
 * products, FP32 accumulation: about FP32 accuracy); otherwise, or with the
 * environment variable CORR_IG_PATH=cuda_core, as an FP32 GEMM on the CUDA
 * cores. */
corr_status_t corr_gain_backward(corr_handle_t h, const void *d_in, const void *d_gain,
                                 const void *d_vis_model, const void *d_raw_vis,
                                 void *d_grad_gain, void *d_grad_in, float *d_loss,
                                 const float *d_grad_scale, void *stream);

/* Frees the plan and its device memory (synchronizes the plan's device).
 * NULL is accepted. */
corr_status_t corr_destroy(corr_handle_t h);

/* Sample layouts of one integration (integrations are always outermost; an
 * element is both pols of one complex sample, [pol][re, im]):
 *   CORR_LAYOUT_CST  [channel][station][time]: what corr_correlate reads;
 *   CORR_LAYOUT_CTS  [channel][time][station]: all stations of one time step
 *                    together, the transposed layout of Section 4.4 (Fig. 4);
 *   CORR_LAYOUT_SCT  [station][channel][time]: one receiver's stream with all
 *                    its channels, the input of the FX corner turn
 *                    (Section 7). */
typedef enum { CORR_LAYOUT_CST = 0, CORR_LAYOUT_CTS = 1, CORR_LAYOUT_SCT = 2 } corr_layout_t;

/* Permutes samples from layout `from` to layout `to` on the device, bit for
 * bit (Section 4.4's transpose and the local part of Section 7's corner
 * turn). Needs no plan and allocates nothing; asynchronous on `stream`.
 *   d_in, d_out: device buffers of n_integrations * n_channels * n_stations *
 *       n_samples elements of dtype (4 bytes for CORR_CI8, 8 for CORR_CF16,
 *       16 for CORR_CF32), aligned to the element size; they must not
 *       overlap. May be NULL when there are no elements.
 * Errors: CORR_ERR_INVALID_ARG for negative sizes, n_integrations < 1, an
 * unknown dtype or layout, NULL, misaligned or overlapping buffers;
 * CORR_ERR_CUDA if the launch fails. */
corr_status_t corr_reorder(int n_stations, int n_channels, int n_samples, int n_integrations,
                           corr_dtype_t dtype, corr_layout_t from, corr_layout_t to,
                           const void *d_in, void *d_out, void *stream);

/* Tile variant the plan's tensor path uses: 0 = 64x64-station tiles,
 * 1 = 64 x up to 128 stations, 2 = 128x128-station tiles on a cluster of two
 * CTAs (CTA-pair MMAs); -1 for FP32 samples (either path) or NULL. Chosen in corr_create by
 * timing each (see CORR_FLAG_NO_AUTOTUNE); the environment variable
 * CORR_TC_VARIANT=narrow|wide|pair forces one (pair falls back to wide where
 * a cluster of two such CTAs cannot be resident). */
int corr_tile_variant(corr_handle_t h);

/* Measurement hook: with two CUDA events (cudaEvent_t passed as void*), every
 * later corr_correlate / corr_correlate_host chunk on this plan records
 * ev_start on its stream right before the launch of the plan's main kernel
 * (tensor path: the first launch over its main tile list, i.e. the
 * power-checked launch of int8, not the redo or tail launches; FP32 path:
 * the correlation kernel and, for a split sample axis, its reduction; FP32
 * samples on the tensor cores: the correlation kernel and its chunk
 * reduction) and
 * ev_stop right after it, so cudaEventElapsedTime gives that kernel's
 * duration. The plan does not own the events; NULL, NULL turns the hook off.
 * CORR_ERR_INVALID_ARG if only one is NULL. */
corr_status_t corr_set_kernel_events(corr_handle_t h, void *ev_start, void *ev_stop);

/* Tile variant of the plan's current ragged batch (same codes as
 * corr_tile_variant), chosen on the first corr_correlate_batched call with
 * that set of sub-arrays; -1 before any batch or for NULL. */
int corr_batch_tile_variant(corr_handle_t h);

/* The tensor-path plan's tile configuration (Section 2's tiling of the
 * correlation triangle, chosen by corr_create's autotuner): *variant (0
 * narrow, 1 wide, 2 pair), *tail (the tail list's variant for pair tiles
 * with an odd block count: 0 narrow, 1 wide), *layout (0, or 1 for the
 * int8 pair kernel of two pols with the six-stage operand ring instead of
 * staged epilogue groups) and *source: 0 forced by CORR_TC_VARIANT /
 * CORR_TC_TAIL / CORR_TC_LAYOUT, 1 the size rule (CORR_FLAG_NO_AUTOTUNE or
 * no samples), 2 timed in this corr_create, 3 cached earlier in this
 * process, 4 read from the tuning cache file (CORR_TUNE_CACHE, "off" for
 * none; default $XDG_CACHE_HOME/corr_gb300/tune.txt or
 * ~/.cache/corr_gb300/tune.txt; lines of other library builds are ignored).
 * Any output may be NULL. CORR_ERR_INVALID_ARG for a plan of FP32 samples. */
corr_status_t corr_tile_config(corr_handle_t h, int *variant, int *tail, int *layout, int *source);

/* The candidates the autotuner timed (batch = 0: in corr_create; 1: for the
 * current ragged batch) with their times: cfg[3i..3i+2] = {variant, tail,
 * layout}, ms[i] = milliseconds per run (batch: the best of two rounds).
 * Fills up to cap entries (cfg and ms may be NULL) and returns the count
 * (0 when nothing was timed), -1 for a NULL handle. Host-only. */
int corr_tune_results(corr_handle_t h, int batch, int cap, int *cfg, float *ms);

/* Reads and clears the plan's device error word (synchronous copy):
 * CORR_OK or CORR_ERR_TIMEOUT. */
corr_status_t corr_get_error(corr_handle_t h);

/* Static description of a status code. */
const char *corr_status_string(corr_status_t s);

/* Text of the last CUDA failure seen by this thread inside the library
 * (empty if none). Valid until the next failing call on this thread. */
const char *corr_last_error_message(void);

/* corr_gain_backward without a plan and without any allocation.
 *
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc, such as a real-time pipeline that forbids allocation once
 * observing has started, a plug-in running inside another framework's
 * memory pool, or code issuing work where an allocation would synchronize
 * the device. It computes what corr_gain_backward computes (same gradient
 * convention and layouts) for n_units channels of n_stations stations and
 * n_samples samples, with d_raw_vis (R from corr_correlate) required.
 *
 * Scratch (the input-gradient matrix W', 32*S*S*n_units bytes when
 * d_grad_in is given, and one float per channel when d_loss is given) lives
 * in a fixed array of corr_noalloc_scratch_bytes() bytes (16 MiB) that the
 * library holds on every GPU that loads it, until the process exits. Larger
 * problems are rejected with CORR_ERR_UNSUPPORTED and a message in
 * corr_last_error_message. Nothing in the array needs to start at zero;
 * every call overwrites what it uses. The first call in a device's context
 * looks up the array's device address with that device current (a
 * synchronous runtime call), so make it before any stream capture; the
 * address is cached with the context's ID and looked up again in a new
 * context of the device (after cudaDeviceReset, for example). Complex
 * buffers must be 8-byte aligned, d_loss and d_grad_scale 4-byte aligned
 * (CORR_ERR_INVALID_ARG otherwise). All calls share the
 * one array: calls whose kernels overlap on the GPU (different streams
 * without ordering) race and give wrong results. No cudaMalloc, cudaFree or
 * allocating library routine is called. Asynchronous on stream. */
corr_status_t corr_gain_backward_noalloc(int n_stations, int n_units, int n_samples,
                                         const void *d_in, const void *d_gain,
                                         const void *d_vis_model, const void *d_raw_vis,
                                         void *d_grad_gain, void *d_grad_in, float *d_loss,
                                         const float *d_grad_scale, void *stream);

/* Size in bytes of the fixed scratch array of corr_gain_backward_noalloc. */
size_t corr_noalloc_scratch_bytes(void);

/* Host-only helpers (no GPU needed), used by the plan and by tests. */

/* Tile cost model of Section 2 (Table 1) for a w x h station tile:
 * flops = 32wh, bytes = 16(w+h), minimum registers = 4(1+min(w,h)) + 8wh. */
void corr_tile_cost(int w, int h, long *flops, long *bytes, long *regs);

/* Number of tensor-path work tiles for S stations (upper triangle of
 * 64-station blocks, diagonal included) and the decode of tile k into its
 * row and column block (rb <= cb). Returns -1 for k out of range. */
int corr_tc_tiles(int n_stations);
int corr_tc_tile_decode(int n_stations, int k, int *rb, int *cb);

/* The tensor path's work tiles for one channel of n_stations stations in
 * tile variant `variant` (0 narrow, 1 wide, 2 pair), in launch order: for
 * tile k, out[4k..4k+3] = {row block, first column block, column blocks,
 * list} over 64-station blocks, list 0 for the main launch and 1 for the
 * second launch. The second list exists for the pair variant with an odd
 * block count, in variant tail_kind: 0 (narrow) = the last block column as
 * narrow tiles, pair tiles over blocks 0 .. nb-2; 1 (wide) = block 0's row
 * as wide tiles, pair tiles over blocks 1 .. nb-1. A tile's row blocks are
 * {rb} (narrow, wide) or {rb, rb+1} (pair); its column blocks cb0 .. cb0 +
 * count - 1. With out == NULL returns the tile count; otherwise fills out
 * and returns the count, or -1 if it exceeds cap (tiles) or the arguments
 * are invalid. */
int corr_tc_schedule(int variant, int tail_kind, int n_stations, int cap, int *out);

/* Number of 4x4-station register tiles of the FP32 path per channel
 * (upper triangle, diagonal included) and the decode of tile k into its
 * row and column index (i <= j). Returns -1 for k out of range. The FP32
 * kernel uses this map above 64 stations; up to 64 it uses 4x2-station
 * tiles, row i holding column pairs j = 2i .. ceil(S/2) - 1. */
int corr_fp32_subtiles(int n_stations);
int corr_fp32_subtile_decode(int n_stations, int k, int *i, int *j);

#ifdef __cplusplus
}
#endif

#endif /* CORR_H */
