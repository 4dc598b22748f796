// Internal declarations of the tensor-core path (corr_tc.cu and its host
// side), kept apart so that the tensor kernel's sources are exactly
// corr_tc.cu, this header and ptx.cuh.
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
    // The list cleans up after itself: the redo launch's last CTA clears the
    // marks of the items it held and zeroes the count, so no call needs a
    // memset first.
    int check_power;
    int *redo_mark;           // per item: 0, or 1 once appended
    int4 *redo_items;
    int *redo_index;          // item index of each appended entry
    int *redo_count;
    int *redo_done;           // redo launch only: CTAs finished (the last one resets the list)
    int *err;                 // device error word
    unsigned long long wait_ns;
    // launched as a programmatic dependent of whatever kernel precedes it on
    // the stream: every CTA sets up its barriers and TMEM, then waits for
    // that kernel's completion before it touches global memory
    int dep_wait;
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
// pdl: launched as a programmatic dependent of the previous kernel on the
// stream: the redo launch (the kernel waits for that kernel's completion
// before it reads the redo count), a main launch with dep_wait set (it waits
// after its set-up), or a tail list (it reads nothing the kernels before it
// in the same call write, and those began after everything earlier on the
// stream had completed).
// layout: 0, or 1 for the int8 pair kernel of two pols in its second
// instantiation (six operand stages, no staged epilogue groups); ignored
// elsewhere.
cudaError_t tc_launch(int dtype, int variant, int npol, const TcParams &p, int grid, cudaStream_t s,
                      bool pdl = false, int layout = 0);
// Clusters of the pair variant that fit on the device at once.
cudaError_t tc_pair_max_clusters(int dtype, int *n);

} // namespace corr
