// Sample-layout permutations (corr_reorder).
//
// The correlator reads [channel][station][time][pol] (CST). Section 4.4 keeps,
// for the GPU kernel, the samples of all stations of one time step together
// ([channel][time][station][pol], CTS, the "transposed" layout), and Section 7
// describes the FX corner turn: every receiver delivers all channels of one
// station ([station][channel][time][pol], SCT) and the correlator needs one
// channel of all stations. Each kernel launch here moves one integration's
// elements (an element = both pols of one complex sample: 4, 8 or 16 bytes)
// from one of these layouts to another, bit for bit.
//
// Work unit: a tile of stations x time steps of one channel. Threads read the
// tile along the input's fastest axis (time for CST and SCT, stations for
// CTS) into shared memory and write it along the output's fastest axis, so
// both sides are coalesced. The kernels are bound by HBM: every element is
// read once and written once.
#include <algorithm>

#include "../../include/corr.h"
#include "corr_internal.h"

namespace corr {

namespace {

constexpr int RT = 32;          // tile side (stations and time steps)
constexpr int RTHREADS = 256;   // 8 rows of 32 threads

// Offset of element (c, s, t) of one integration in layout L.
__device__ __forceinline__ long long layout_offset(int L, int S, int C, int T, int c, int s, int t)
{
    if (L == CORR_LAYOUT_CTS) return ((long long)c * T + t) * S + s;
    if (L == CORR_LAYOUT_SCT) return ((long long)s * C + c) * T + t;
    return ((long long)c * S + s) * T + t; // CORR_LAYOUT_CST
}

template <typename E>
__global__ void __launch_bounds__(RTHREADS) reorder_kernel(const E *__restrict__ in, E *__restrict__ out,
                                                           int S, int C, int T, int from, int to,
                                                           long long n_tiles)
{
    __shared__ E tile[RT][RT + 1]; // [station][time], padded against bank conflicts
    const int n_st = (S + RT - 1) / RT, n_tt = (T + RT - 1) / RT;
    const int tx = threadIdx.x & (RT - 1), ty = threadIdx.x / RT;
    const bool in_s_fast = from == CORR_LAYOUT_CTS, out_s_fast = to == CORR_LAYOUT_CTS;
    const long long per_integration = (long long)S * C * T;
    for (long long k = blockIdx.x; k < n_tiles; k += gridDim.x) {
        const int tt = (int)(k % n_tt);
        long long r = k / n_tt;
        const int st = (int)(r % n_st);
        r /= n_st;
        const int c = (int)(r % C);
        const long long base = (r / C) * per_integration;
        const int s0 = st * RT, t0 = tt * RT;
#pragma unroll
        for (int i = 0; i < RT; i += RTHREADS / RT) {
            // thread (tx, ty + i) along the fast axis of the input
            const int s = s0 + (in_s_fast ? tx : ty + i);
            const int t = t0 + (in_s_fast ? ty + i : tx);
            if (s < S && t < T) tile[s - s0][t - t0] = in[base + layout_offset(from, S, C, T, c, s, t)];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RT; i += RTHREADS / RT) {
            const int s = s0 + (out_s_fast ? tx : ty + i);
            const int t = t0 + (out_s_fast ? ty + i : tx);
            if (s < S && t < T) out[base + layout_offset(to, S, C, T, c, s, t)] = tile[s - s0][t - t0];
        }
        __syncthreads();
    }
}

// Vectorised form: 16-byte global loads and stores (V = 16 / sizeof(E)
// elements along each side's contiguous axis), tiles of TILE x TILE
// elements, elements moved one by one through shared memory. Needs both
// contiguous axes to be multiples of V and 16-byte aligned buffers.
template <typename E, int TILE>
__global__ void __launch_bounds__(RTHREADS) reorder_vec_kernel(const E *__restrict__ in, E *__restrict__ out,
                                                               int S, int C, int T, int from, int to,
                                                               long long n_tiles)
{
    constexpr int V = 16 / (int)sizeof(E);   // elements per 16-byte vector
    constexpr int NV = TILE / V;             // vectors along a tile row
    constexpr int PER = TILE * NV / RTHREADS;
    static_assert(PER * RTHREADS == TILE * NV, "tile / thread count");
    __shared__ E tile[TILE][TILE + 1];       // [station][time]
    const int n_st = (S + TILE - 1) / TILE, n_tt = (T + TILE - 1) / TILE;
    const bool in_s_fast = from == CORR_LAYOUT_CTS, out_s_fast = to == CORR_LAYOUT_CTS;
    const long long per_integration = (long long)S * C * T;
    // tile k -> (integration base, channel c, first station s0, first time t0)
    auto tile_of = [&](long long k, long long &base, int &c, int &s0, int &t0) {
        const int tt = (int)(k % n_tt);
        long long r = k / n_tt;
        const int st = (int)(r % n_st);
        r /= n_st;
        c = (int)(r % C);
        base = (r / C) * per_integration;
        s0 = st * TILE;
        t0 = tt * TILE;
    };
    auto load = [&](long long k, uint4 (&buf)[PER]) {
        long long base;
        int c, s0, t0;
        tile_of(k, base, c, s0, t0);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int id = threadIdx.x + j * RTHREADS;
            const int v = id % NV, row = id / NV;
            const int s = s0 + (in_s_fast ? v * V : row);
            const int t = t0 + (in_s_fast ? row : v * V);
            buf[j] = (s < S && t < T)
                         ? __ldg(reinterpret_cast<const uint4 *>(in + base + layout_offset(from, S, C, T, c, s, t)))
                         : make_uint4(0, 0, 0, 0);
        }
    };
    // The loads of the CTA's next tile are issued before the stores of the
    // current one, so that both are in flight together.
    uint4 cur[PER], nxt[PER];
    long long k = blockIdx.x;
    if (k < n_tiles) load(k, cur);
    for (; k < n_tiles; k += gridDim.x) {
        long long base;
        int c, s0, t0;
        tile_of(k, base, c, s0, t0);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int id = threadIdx.x + j * RTHREADS;
            const int v = id % NV, row = id / NV;
            const E *e = reinterpret_cast<const E *>(&cur[j]);
#pragma unroll
            for (int q = 0; q < V; ++q) {
                if (in_s_fast)
                    tile[v * V + q][row] = e[q];
                else
                    tile[row][v * V + q] = e[q];
            }
        }
        __syncthreads();
        if (k + gridDim.x < n_tiles) load(k + gridDim.x, nxt);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int id = threadIdx.x + j * RTHREADS;
            const int v = id % NV, row = id / NV;
            const int s = s0 + (out_s_fast ? v * V : row);
            const int t = t0 + (out_s_fast ? row : v * V);
            if (s < S && t < T) {
                uint4 w;
                E *e = reinterpret_cast<E *>(&w);
#pragma unroll
                for (int q = 0; q < V; ++q)
                    e[q] = out_s_fast ? tile[v * V + q][row] : tile[row][v * V + q];
                *reinterpret_cast<uint4 *>(out + base + layout_offset(to, S, C, T, c, s, t)) = w;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PER; ++j) cur[j] = nxt[j];
    }
}

template <typename E>
cudaError_t launch_reorder(const void *in, void *out, int S, int C, int T, long long units_i,
                           int from, int to, int sm_count, cudaStream_t s)
{
    constexpr int V = 16 / (int)sizeof(E);
    constexpr int TILE = sizeof(E) == 16 ? 32 : 64;
    const int fast_in = from == CORR_LAYOUT_CTS ? S : T, fast_out = to == CORR_LAYOUT_CTS ? S : T;
    const bool vec = fast_in % V == 0 && fast_out % V == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
                     reinterpret_cast<uintptr_t>(out) % 16 == 0;
    const int tile = vec ? TILE : RT;
    const long long n_tiles =
        units_i * C * (long long)((S + tile - 1) / tile) * ((T + tile - 1) / tile);
    if (n_tiles == 0) return cudaSuccess;
    const long long grid = std::min<long long>(n_tiles, (long long)sm_count * 8);
    if (vec)
        reorder_vec_kernel<E, TILE><<<(unsigned)grid, RTHREADS, 0, s>>>(
            static_cast<const E *>(in), static_cast<E *>(out), S, C, T, from, to, n_tiles);
    else
        reorder_kernel<E><<<(unsigned)grid, RTHREADS, 0, s>>>(static_cast<const E *>(in), static_cast<E *>(out),
                                                               S, C, T, from, to, n_tiles);
    return cudaGetLastError();
}

} // namespace

cudaError_t reorder_launch(const void *in, void *out, int S, int C, int T, long long n_integrations,
                           int elem_bytes, int from, int to, int sm_count, cudaStream_t s)
{
    if (elem_bytes == 16) return launch_reorder<uint4>(in, out, S, C, T, n_integrations, from, to, sm_count, s);
    if (elem_bytes == 8) return launch_reorder<uint2>(in, out, S, C, T, n_integrations, from, to, sm_count, s);
    return launch_reorder<uint32_t>(in, out, S, C, T, n_integrations, from, to, sm_count, s);
}

} // namespace corr
