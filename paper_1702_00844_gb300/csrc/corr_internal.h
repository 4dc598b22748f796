// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "corr_tc_internal.h"

namespace corr {

// ------------------------------------------------------------------ FP32 path
struct Fp32Params {
    float2 *out;
    int S, T, n_units;                // S: (pseudo-)stations of the sub-tile grid
    int tw;                           // sub-tiles of 4 x tw stations (tw = 4 or 2)
    int load_warp;                    // 1: an extra warp issues the TMA loads (two pols only)
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
#ifndef CORR_FP32_STAGES
#define CORR_FP32_STAGES 3
#endif
constexpr int FP32_STAGES = CORR_FP32_STAGES;
// npol 2: samples through the TMA map tmap; npol 1: through p.in1.
cudaError_t fp32_launch(const void *tmap, const Fp32Params &p, int npol, int threads, size_t smem,
                        cudaStream_t s);

// -------------------------------------------------------------- gain adjoint
cudaError_t gain_loss_launch(const float2 *R, const float2 *g, const float2 *M, float2 *V,
                             float *partial, float *loss, int S, int units, cudaStream_t s);
// dL/d conj(g); with W (units x 2S x 2S complex64) also the matrix W' of the
// input gradient, from the same residuals.
// Input gradient on the tensor cores (corr_gain_tc.cu): A' tiles written
// by gain_grad_launch in tile mode, samples through a TMA map of boxes of
// 4 floats x CORR_IG_KV / 4 stations x up to 128 times.
struct IgParams {
    const float *at;          // A' tiles [unit][m tile][k block]([hi, lo] unless CORR_IG_A_FP32)[128 x CORR_IG_KV floats]
    float2 *gx;               // [unit][S][T][2] complex
    int S, T, units, m_tiles, k_blocks;
    int m_alloc;              // row tiles per unit in the A' buffer (m_tiles rounded up to even)
    int *err;
    unsigned long long wait_ns;
};
// Times per tile of the tensor-core input gradient (its N) and operand
// stages of its ring. A TMA box of samples holds at most CORR_IG_BOX times
// (2 x CORR_IG_BOX 8-byte elements <= 256); wider tiles take several.
#ifndef CORR_IG_N
#define CORR_IG_N 128
#endif
// Reduction values (re and im of a station's two pols: 4 per station) per
// K-block: 32 (rows of 128 bytes of tf32 in the 128-byte swizzled layout, 8
// stations) or 16 (rows of 64 bytes in the 64-byte swizzled layout, 4
// stations: stages half as large, twice as many in flight; measured slower,
// the kernel's cost is per K-block rather than per byte in flight).
#ifndef CORR_IG_KV
#define CORR_IG_KV 32
#endif
#ifndef CORR_IG_STAGES
#define CORR_IG_STAGES (CORR_IG_KV == 16 ? 6 : 3)
#endif
#define CORR_IG_BOX (CORR_IG_N < 128 ? CORR_IG_N : 128)
// Warps that split the operands into tf32 hi and lo.
#ifndef CORR_IG_SPLIT_WARPS
#define CORR_IG_SPLIT_WARPS 4
#endif
// 1: A' tiles hold W' in FP32 and the kernel splits them in shared memory;
// 0: the gain-gradient kernel writes them already split (hi and lo tiles).
#ifndef CORR_IG_A_FP32
#define CORR_IG_A_FP32 0
#endif
// FP32 samples on the tensor cores (corr_tf32.cu): tf32 value + remainder
// split, three products, FP32 accumulation; two pols, complex64 samples
// [unit][S][T][2] read through a TMA map of 8-byte elements.
struct TfParams {
    float2 *out;              // [unit][baseline][2][2] complex
    int S, T, units, nb;      // nb = blocks of 64 stations
    int chunk_kb;             // K-blocks of 16 samples per accumulator chunk
    // nullable: with few tiles, each chunk of a tile is its own work item
    // writing partial[chunk][unit][baseline][2][2], summed afterwards
    float2 *partial;
    int *err;
    unsigned long long wait_ns;
};
cudaError_t tf32_correlate_launch(const void *xmap, const TfParams &p, cudaStream_t s);

// Row tiles (128 rows of M' = 4S) and K blocks (CORR_IG_KV of K' = 4S) of
// the tiles.
__host__ __device__ inline int ig_m_tiles(int S) { return (4 * S + 127) / 128; }
__host__ __device__ inline int ig_k_blocks(int S) { return (4 * S + CORR_IG_KV - 1) / CORR_IG_KV; }
// A CTA pair takes two row tiles; with an odd count the second of the last
// pair reads a zero tile.
__host__ __device__ inline int ig_m_alloc(int S) { return (ig_m_tiles(S) + 1) & ~1; }
inline size_t ig_tile_bytes(int S, long long units)
{
    return (size_t)units * ig_m_alloc(S) * ig_k_blocks(S) * (CORR_IG_A_FP32 ? 1 : 2) * (128 * 4 * CORR_IG_KV);
}
// pair: tiles of two row tiles on CTA pairs (cta_group::2)
cudaError_t input_grad_tc_launch(const void *xmap, const IgParams &p, cudaStream_t s, bool pair);
// tiles = 1: W is the A' tile buffer (zeroed once, its padding never written)
cudaError_t gain_grad_launch(const float2 *R, const float2 *g, const float2 *M,
                             const float *scale, float2 *grad_g, void *W, int S, int units,
                             cudaStream_t s, int tiles = 0);
// dL/d conj(x) = W' x per channel (W' from gain_grad_launch).
cudaError_t input_grad_launch(const float2 *x, const float2 *W, float2 *grad_x, int S, int T, int units,
                              cudaStream_t s);

// ------------------------------------------------------------ layouts
// Permutes n_integrations x (C x S x T) elements of elem_bytes (4, 8 or 16)
// from layout `from` to layout `to` (corr_layout_t).
cudaError_t reorder_launch(const void *in, void *out, int S, int C, int T, long long n_integrations,
                           int elem_bytes, int from, int to, int sm_count, cudaStream_t s);

// Records the text returned by corr_last_error_message on this thread.
void set_last_error(cudaError_t e);
void set_last_error(const char *msg);

} // namespace corr
