// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace corr {

// ---------------------------------------------------------------- tensor path
// One correlation problem for the tcgen05 kernel: n_units independent
// channels (integrations x channels) of S stations and T samples.
struct TcProblem {
    const void *in;           // [unit][S][T][P pols] complex f16 or int8
    void *out;                // [unit][S(S+1)/2][P][P] complex f32 or int32
    long long in_unit_bytes;  // S*T*P*sizeof(complex sample)
    long long out_unit_elems; // S(S+1)/2 * P*P complex values
    int S, T, n_units, vec;   // vec: 16-byte vector loads are aligned
};

struct TcParams {
    TcProblem prob0;          // used when probs == nullptr
    const TcProblem *probs;   // device array (ragged batches)
    const int4 *items;        // {problem, unit, row block, col block | n blocks << 16}
    int n_items;
    const int *n_items_dev;   // if set, the item count is read from device memory
    int chunk_kb;             // K-blocks per exact accumulation chunk (0 = all)
    // int8 without chunks: producers bound every partial sum of a tile by the
    // largest station power sum_t |x|^2 of its stations (Cauchy-Schwarz); a
    // tile whose bound exceeds 2^24 is appended once to the redo list, which
    // a second, chunked launch recomputes (overwriting its output).
    int check_power;
    int *redo_mark;           // per item: 0, or 1 once appended (zeroed per call)
    int4 *redo_items;
    int *redo_count;
    int *err;                 // device error word
    unsigned long long wait_ns;
};

// Tile variants of the tensor kernel: narrow = 64x64-station tiles (N=128,
// double-buffered accumulators); wide = 64 x up to 128 stations (N=256);
// pair = 128x128-station tiles on a cluster of two CTAs (CTA-pair MMAs,
// M=256, N=256).
enum TcVariant { TC_NARROW = 0, TC_WIDE = 1, TC_PAIR = 2 };
constexpr int TC_N_VARIANTS = 3;

constexpr int TC_RS = 64;      // stations per tile side
constexpr int TC_KB_T = 32;    // time samples per K-block
constexpr int TC_THREADS = 13 * 32;
constexpr int TC_INT8_CHUNK_KB = 16; // 512 samples: |partial| <= 2^24

// grid: CTAs (even for TC_PAIR: two per cluster). npol: 1 or 2 polarisations
// (with 1, the items are over pseudo-stations of two stations each).
cudaError_t tc_launch(int dtype, int variant, int npol, const TcParams &p, int grid, cudaStream_t s);
// Clusters of the pair variant that fit on the device at once.
cudaError_t tc_pair_max_clusters(int dtype, int *n);

// ------------------------------------------------------------------ FP32 path
struct Fp32Params {
    float2 *out;
    int S, T, n_units;                // S: (pseudo-)stations of the sub-tile grid
    int tw;                           // sub-tiles of 4 x tw stations (tw = 4 or 2)
    int nq, ncq;                      // row groups (4 stations) and column groups (tw)
    int nsub, groups, group_size;     // sub-tiles per unit and their grouping over CTAs
    int tc;                           // samples per pipeline stage
    int *err;
    unsigned long long wait_ns;
    // one polarisation: the samples [unit][station][time] complex64, and the
    // real station count (S = ceil(S1 / 2) pseudo-stations)
    const float2 *in1;
    int S1;
    // split of the sample axis over CTAs (few units): ksplit ranges of
    // kchunks chunks each, partial sums in partial[ksplit][n_units][...],
    // summed in a fixed order by a second kernel (nullptr when ksplit = 1)
    int ksplit, kchunks;
    float2 *partial;
};
constexpr int FP32_STAGES = 3;
// npol 2: samples through the TMA map tmap; npol 1: through p.in1.
cudaError_t fp32_launch(const void *tmap, const Fp32Params &p, int npol, int threads, size_t smem,
                        cudaStream_t s);

// -------------------------------------------------------------- gain adjoint
cudaError_t gain_loss_launch(const float2 *R, const float2 *g, const float2 *M, float2 *V,
                             float *partial, float *loss, int S, int units, cudaStream_t s);
cudaError_t gain_grad_launch(const float2 *R, const float2 *g, const float2 *M,
                             const float *scale, float2 *grad_g, int S, int units,
                             cudaStream_t s);
cudaError_t input_grad_launch(const float2 *x, const float2 *R, const float2 *g,
                              const float2 *M, const float *scale, float2 *W,
                              float2 *grad_x, int S, int T, int units, cudaStream_t s);

// ------------------------------------------------------------ layouts
// Permutes n_integrations x (C x S x T) elements of elem_bytes (4, 8 or 16)
// from layout `from` to layout `to` (corr_layout_t).
cudaError_t reorder_launch(const void *in, void *out, int S, int C, int T, long long n_integrations,
                           int elem_bytes, int from, int to, int sm_count, cudaStream_t s);

// Records the text returned by corr_last_error_message on this thread.
void set_last_error(cudaError_t e);
void set_last_error(const char *msg);

} // namespace corr
