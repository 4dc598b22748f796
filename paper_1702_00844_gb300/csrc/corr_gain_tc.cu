// Sample gradient of the gain-calibration loss on the tensor cores.
//
// Per channel, grad_x[c][t] = sum_b W'[c][b] x[b][t] over c, b = (station,
// pol), W' = 2 conj(g) W g (see corr_gain.cu for W). As a real GEMM with the
// real and imaginary parts interleaved along both axes (rows 2c, 2c+1 and
// reduction index k = 2b, 2b+1):
//     A'[2c][2b] = Re W'cb,   A'[2c][2b+1] = -Im W'cb,
//     A'[2c+1][2b] = Im W'cb, A'[2c+1][2b+1] = Re W'cb,
//     B'[t][2b] = Re x_b(t),  B'[t][2b+1] = Im x_b(t),
// so D = A' B'^T holds Re grad_x in row 2c and Im in row 2c+1 (M' = K' = 4S,
// N = T).
//
// FP32 accuracy from tf32 tensor cores (tcgen05 kind::tf32): every operand
// is split into hi = its value rounded to tf32 (11 significant bits) and
// lo = (value - hi), exact in FP32 (rounded to tf32 for A', by the
// gain-gradient kernel; for the samples the MMA uses its tf32 bits), and
//     A'B' ~ A_hi B_hi + A_hi B_lo + A_lo B_hi
// accumulated in FP32 (the dropped A_lo B_lo and lo's lost bits are at most
// about 2^-21 of each product).
//
// Tiles of (channel, 128-row tile of M', IG_N-time tile of N), spread over
// one persistent CTA per SM; or, with two row tiles or more, tiles of two
// row tiles x 2 IG_N times on CTA pairs (a cluster of two, cta_group::2
// MMAs of M = 256, N = 2 IG_N): each CTA stages its own row tile of A' and
// its own IG_N times of the samples, so per SM the MMA does twice the work
// for the same shared-memory operand traffic. Per K-block of IG_KV = 32
// reduction values (8 stations x 2 pols x re/im; 16 and 4 stations with
// CORR_IG_KV = 16), through a ring of operand stages that runs on across
// the CTA's tiles:
//   - one thread issues the loads: A' as bulk copies (16 KB, or 8 KB) of
//     tiles that the gain-gradient kernel wrote already swizzled, split into
//     hi and lo (or in FP32 with CORR_IG_A_FP32, split here in shared
//     memory), and the samples with TMA boxes of IG_BOX times (16 bytes
//     each, 2 IG_BOX 8-byte elements: one contiguous run) x the K-block's
//     stations, landing station-major in the lo tile;
//   - IG_SW warps split the samples into hi and lo and transpose them into
//     K-major rows (one time each) of the K-block's stations x 16 bytes, the
//     chunk of station j in row t at 16-byte position j ^ (t mod 8): the
//     128-byte swizzled layout the MMA reads (j ^ ((t / 2) mod 4), the
//     64-byte one, with 16 values);
//   - one thread (of the even CTA of a pair) issues IG_KV / 8 K-steps x 3 MMAs
//     (K = 8) into one of two TMEM accumulators, alternating per tile; in a
//     pair one thread of the odd CTA forwards each of its stages' "split
//     done" phases to the even CTA with one cluster-scope arrival;
// and four more warps store each finished accumulator (TMEM -> registers ->
// a per-warp transpose in shared memory -> 16-byte stores of (XX, YY)
// complex pairs of one station and time) while the next tile's MMAs run in
// the other one.
// Every wait is bounded (mbar_wait_bounded); a pair leaves together after a
// cluster barrier that every thread reaches once its bounded loops end.
#include <cuda.h>

#include "corr_internal.h"
#include "ptx.cuh"

namespace corr {

namespace {

// warp 0 loads, warps 1 .. SW split, the next four store (each a different
// TMEM lane quarter, warp % 4), the last allocates TMEM and issues the MMAs
// (in the odd CTA of a pair: relays its split phases)
constexpr int IG_SW = CORR_IG_SPLIT_WARPS;
constexpr int IG_SPLIT_THREADS = 32 * IG_SW;
constexpr int IG_EPI_WARP0 = 1 + IG_SW, IG_MMA_WARP = IG_EPI_WARP0 + 4;
constexpr int IG_THREADS = 32 * (IG_MMA_WARP + 1);
constexpr int IG_A_PARTS = CORR_IG_A_FP32 ? 1 : 2;   // A' tiles per K block in global memory
constexpr int IG_M = 128, IG_N = CORR_IG_N;    // per CTA: rows of M' x times
constexpr int IG_STAGES = CORR_IG_STAGES;
constexpr int IG_KV = CORR_IG_KV;                // reduction values per K-block
constexpr int IG_KS = IG_KV / 4;                 // stations per K-block
constexpr uint32_t IG_ROW = 4 * IG_KV;           // bytes per operand row: 128 or 64
constexpr uint32_t IG_A_BYTES = IG_M * IG_ROW;   // 128 rows x IG_KV tf32
constexpr uint32_t IG_B_BYTES = IG_N * IG_ROW;   // IG_N rows x IG_KV tf32
static_assert(IG_KV == 16 || IG_KV == 32, "K-blocks of 16 or 32 reduction values");
constexpr uint32_t IG_STAGE_BYTES = 2 * IG_A_BYTES + 2 * IG_B_BYTES;   // A hi, A lo, B hi, B lo
constexpr uint32_t IG_EPI_BYTES = 4 * 32 * 17 * 4;                       // per-warp transpose
constexpr int IG_BOX = CORR_IG_BOX;              // times per TMA box of samples
static_assert(IG_N == 64 || IG_N == 128 || IG_N == 256, "input-gradient tile width");
static_assert(IG_N % IG_BOX == 0 && 2 * IG_BOX <= 256, "a TMA box row holds at most 256 elements");

// MMA width, TMEM columns (two accumulators) of a CTA
template <bool PAIR> constexpr int ig_mma_n() { return PAIR ? 2 * IG_N : IG_N; }
template <bool PAIR> constexpr uint32_t ig_tmem_cols() { return 2 * ig_mma_n<PAIR>(); }

// Shared-memory descriptor of a K-major operand tile in the 64-byte swizzled
// layout (as smem_desc_sw128 in ptx.cuh, for rows of 64 bytes): 8-row groups
// 512 bytes apart, layout 4, tile base 512-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Operand descriptors and the swizzled position of 16-byte chunk c of row r:
// the 128-byte swizzle (c ^ (r mod 8)) for 32 values per row, the 64-byte
// swizzle (c ^ ((r / 2) mod 4)) for 16.
__device__ __forceinline__ uint64_t ig_desc(uint32_t saddr)
{
    return IG_KV == 32 ? smem_desc_sw128(saddr) : smem_desc_sw64(saddr);
}
__device__ __forceinline__ uint32_t ig_swz(int r, int c)
{
    return (uint32_t)(r * (int)IG_ROW + (IG_KV == 32 ? (c ^ (r & 7)) : (c ^ ((r >> 1) & 3))) * 16);
}

struct IgBars {
    uint64_t raw[IG_STAGES];     // loads landed (transaction bytes)
    uint64_t rd[IG_STAGES];      // raw samples read into registers (one arrival per split thread)
    uint64_t full[IG_STAGES];    // operands split (one arrival per split thread; + 1 relayed in a pair)
    uint64_t empty[IG_STAGES];   // MMAs of the stage done (commit)
    uint64_t acc_full[2];        // a tile's MMAs done (commit)
    uint64_t acc_empty[2];       // a tile's accumulator read out (4 warps; + 4 remote in a pair)
    uint64_t done;               // every MMA issued has completed (commit)
    uint32_t tmem_base;
    int abort_flag;
};

constexpr size_t ig_smem_bytes() { return IG_STAGES * IG_STAGE_BYTES + IG_EPI_BYTES + sizeof(IgBars) + 1024; }
static_assert(ig_smem_bytes() <= 227 * 1024, "input-gradient tiles must fit in shared memory");

struct IgTile {
    int t0, mt, unit;   // first time of this CTA's samples, row tile, unit
    int tt0;            // first time of the tile's accumulator columns
};

// Tile `tile` of the flattened (unit, row tile or row-tile pair, time tile)
// space, time tiles fastest (consecutive tiles share their A' tiles).
template <bool PAIR>
__device__ __forceinline__ IgTile ig_tile(long long tile, int n_times, int rank, const IgParams &p)
{
    const int m_groups = PAIR ? (p.m_tiles + 1) / 2 : p.m_tiles;
    IgTile r;
    const int nt = (int)(tile % n_times);
    const long long rest = tile / n_times;
    const int mg = (int)(rest % m_groups);
    r.unit = (int)(rest / m_groups);
    r.mt = PAIR ? 2 * mg + rank : mg;
    r.tt0 = nt * ig_mma_n<PAIR>();
    r.t0 = r.tt0 + rank * IG_N;
    return r;
}

template <bool PAIR>
__device__ __forceinline__ void ig_body(const CUtensorMap &xmap, const IgParams &p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t base = smem_u32(smem);
    float *epi = reinterpret_cast<float *>(smem + IG_STAGES * IG_STAGE_BYTES);
    IgBars *bars = reinterpret_cast<IgBars *>(smem + IG_STAGES * IG_STAGE_BYTES + IG_EPI_BYTES);
    volatile int *abort_flag = &bars->abort_flag;
    constexpr int MN = ig_mma_n<PAIR>();
    constexpr uint32_t TMEM_COLS = ig_tmem_cols<PAIR>();

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rank = PAIR ? (int)cluster_ctarank() : 0;
    const int KB = p.k_blocks;
    const int n_times = (p.T + MN - 1) / MN;
    const int m_groups = PAIR ? (p.m_tiles + 1) / 2 : p.m_tiles;
    const long long n_tiles = (long long)n_times * m_groups * p.units;
    // this CTA's (or pair's) tiles: g0, g0 + G, ...
    const long long g0 = PAIR ? blockIdx.x / 2 : blockIdx.x;
    const long long G = PAIR ? gridDim.x / 2 : gridDim.x;
    const int my_tiles = (int)((n_tiles - g0 + G - 1) / G);

    if (tid == 0) {
        prefetch_tmap(&xmap);
        for (int s = 0; s < IG_STAGES; ++s) {
            mbar_init(&bars->raw[s], 1);
            mbar_init(&bars->rd[s], IG_SPLIT_THREADS);
            mbar_init(&bars->full[s], IG_SPLIT_THREADS + (PAIR && rank == 0 ? 1 : 0));
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], PAIR ? 8 : 4);
        }
        mbar_init(&bars->done, 1);
        bars->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == IG_MMA_WARP) {
        if constexpr (PAIR) {
            tmem_alloc_pair(&bars->tmem_base, TMEM_COLS);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(&bars->tmem_base, TMEM_COLS);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();   // both CTAs' barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    auto a_hi = [&](int s) { return base + (uint32_t)s * IG_STAGE_BYTES; };
    auto a_lo = [&](int s) { return a_hi(s) + IG_A_BYTES; };
    auto b_hi = [&](int s) { return a_hi(s) + 2 * IG_A_BYTES; };
    auto b_lo = [&](int s) { return b_hi(s) + IG_B_BYTES; };

    if (warp == 0) {
        // ----------------------------------------------------------- loads
        if (lane == 0) {
            long long g = 0;   // K blocks issued so far (over all tiles)
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const IgTile tl = ig_tile<PAIR>(g0 + (long long)i * G, n_times, rank, p);
                // A' tiles of this (unit, row tile): [k block][parts][128 rows x 128 B];
                // p.m_alloc row tiles per unit (a pair's missing odd one is zero)
                const uint8_t *a_tiles = reinterpret_cast<const uint8_t *>(p.at) +
                                         ((size_t)tl.unit * p.m_alloc + tl.mt) * (size_t)KB * IG_A_PARTS * IG_A_BYTES;
                for (int kb = 0; kb < KB; ++kb, ++g) {
                    const int s = (int)(g % IG_STAGES);
                    if (g >= IG_STAGES && !mbar_wait_bounded(&bars->empty[s], (uint32_t)((g / IG_STAGES) - 1) & 1,
                                                             abort_flag, p.err, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&bars->raw[s], IG_A_PARTS * IG_A_BYTES + IG_B_BYTES);
                    bulk_load_g2s(a_hi(s), a_tiles + (size_t)kb * IG_A_PARTS * IG_A_BYTES, IG_A_BYTES,
                                  &bars->raw[s]);
                    if (IG_A_PARTS == 2)
                        bulk_load_g2s(a_lo(s), a_tiles + ((size_t)kb * 2 + 1) * IG_A_BYTES, IG_A_BYTES,
                                      &bars->raw[s]);
                    // the IG_KS stations of this K block, IG_N times from this
                    // CTA's first (zero outside), into the lo tile: boxes of
                    // IG_BOX times, each landing station-major
#pragma unroll
                    for (int h = 0; h < IG_N / IG_BOX; ++h)
                        tma_load_4d(smem + (size_t)s * IG_STAGE_BYTES + 2 * IG_A_BYTES + IG_B_BYTES +
                                        (size_t)h * IG_BOX * IG_KS * 16,
                                    &xmap, &bars->raw[s], 2 * (tl.t0 + h * IG_BOX), kb * IG_KS, tl.unit, 0);
                }
            }
            // on a give-up, let the copies in flight land before the CTA (and
            // its shared memory) goes away; fixed 2 s bound per stage
            if (*abort_flag) {
                int dummy = 0;
                for (long long q = g > IG_STAGES ? g - IG_STAGES : 0; q < g; ++q)
                    mbar_wait_bounded(&bars->raw[q % IG_STAGES], (uint32_t)(q / IG_STAGES) & 1, &dummy, p.err,
                                      2000000000ull);
            }
        }
        __syncwarp();
    } else if (warp <= IG_SW) {
        // ------------------------------------------------------------ split
        const int pt = tid - 32;   // 0 .. IG_SPLIT_THREADS - 1
        long long g = 0;
        bool ok = true;
        for (int i = 0; i < my_tiles && ok; ++i) {
            for (int kb = 0; kb < KB; ++kb, ++g) {
                const int s = (int)(g % IG_STAGES);
                // each wait's outcome is taken by the whole warp, so that a
                // warp leaves together and its lanes meet again below
                const bool landed =
                    mbar_wait_bounded(&bars->raw[s], (uint32_t)(g / IG_STAGES) & 1, abort_flag, p.err, p.wait_ns);
                if (!__all_sync(0xffffffffu, landed)) {
                    ok = false;
                    break;
                }
                // chunk i = q * IG_SPLIT_THREADS + pt of the raw boxes
                // (landed in the lo tile, box after box) is (station
                // (i / IG_BOX) % 8, time of its box i % IG_BOX): consecutive
                // threads read consecutive times of one station. Once all
                // split threads hold their chunks (rd), each writes hi and lo
                // into row t at 16-byte position (station ^ (t mod 8)).
                constexpr int CH = IG_N * IG_KS / IG_SPLIT_THREADS;   // chunks per thread
                uint4 v[CH];
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    v[q] = lds128(b_lo(s) + (uint32_t)((q * IG_SPLIT_THREADS + pt) * 16));
                mbar_arrive(&bars->rd[s]);
                // meanwhile, with FP32 A' tiles, A': each thread splits its
                // own 16-byte chunks in place (hi) and into the lo tile at the
                // same offset
#pragma unroll
                for (int q = 0; q < (IG_A_PARTS == 1 ? (int)(IG_A_BYTES / 16) / IG_SPLIT_THREADS : 0); ++q) {
                    const uint32_t off = (uint32_t)((q * IG_SPLIT_THREADS + pt) * 16);
                    const uint4 a = lds128(a_hi(s) + off);
                    const float4 f = make_float4(__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z),
                                                 __uint_as_float(a.w));
                    const float4 hf =
                        make_float4(tf32_round(f.x), tf32_round(f.y), tf32_round(f.z), tf32_round(f.w));
                    sts128(a_hi(s) + off, make_uint4(__float_as_uint(hf.x), __float_as_uint(hf.y),
                                                     __float_as_uint(hf.z), __float_as_uint(hf.w)));
                    sts128(a_lo(s) + off, make_uint4(__float_as_uint(tf32_round(f.x - hf.x)),
                                                     __float_as_uint(tf32_round(f.y - hf.y)),
                                                     __float_as_uint(tf32_round(f.z - hf.z)),
                                                     __float_as_uint(tf32_round(f.w - hf.w))));
                }
                const bool read =
                    mbar_wait_bounded(&bars->rd[s], (uint32_t)(g / IG_STAGES) & 1, abort_flag, p.err, p.wait_ns);
                if (!__all_sync(0xffffffffu, read)) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    // box h = i / (8 IG_BOX), station, time h IG_BOX + i % IG_BOX
                    const int i = q * IG_SPLIT_THREADS + pt, st = (i / IG_BOX) % IG_KS,
                              t = (i / (IG_KS * IG_BOX)) * IG_BOX + i % IG_BOX;
                    const float4 f = make_float4(__uint_as_float(v[q].x), __uint_as_float(v[q].y),
                                                 __uint_as_float(v[q].z), __uint_as_float(v[q].w));
                    const float4 hf =
                        make_float4(tf32_round(f.x), tf32_round(f.y), tf32_round(f.z), tf32_round(f.w));
                    const uint4 h = make_uint4(__float_as_uint(hf.x), __float_as_uint(hf.y), __float_as_uint(hf.z),
                                               __float_as_uint(hf.w));
                    // lo: the exact remainder, of which the MMA uses the tf32 bits
                    const uint4 l = make_uint4(__float_as_uint(f.x - hf.x), __float_as_uint(f.y - hf.y),
                                               __float_as_uint(f.z - hf.z), __float_as_uint(f.w - hf.w));
                    const uint32_t sw = ig_swz(t, st);
                    sts128(b_hi(s) + sw, h);
                    sts128(b_lo(s) + sw, l);
                }
                fence_proxy_async_smem();
                mbar_arrive(&bars->full[s]);
            }
        }
    } else if (warp < IG_MMA_WARP) {
        // --------------------------------------------------------- epilogue
        // TMEM lanes of this warp: 32 * (warp % 4) ..; lane r of the tile
        // is row m = 128 mt + r of M': c = m / 2 = (station, pol), and re
        // (r even) or im. A quad of lanes holds (X re, X im, Y re, Y im) of
        // one station. Column j of the accumulator is time tt0 + j.
        const int quarter = warp & 3;
        float *w = epi + (size_t)quarter * 32 * 17;
        const int k = lane & 3, quad = lane & ~3;
        for (int i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            // the warp leaves together (the TMEM loads below are warp-wide)
            const bool got =
                mbar_wait_bounded(&bars->acc_full[b], (uint32_t)(i >> 1) & 1, abort_flag, p.err, p.wait_ns);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const IgTile tl = ig_tile<PAIR>(g0 + (long long)i * G, n_times, rank, p);
            const int station = (IG_M * tl.mt + quarter * 32) / 4 + (lane >> 2);
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * MN);
            for (int cg = 0; cg < MN / 16; ++cg) {
                uint32_t v[16];
                tmem_ld_32x32b_x16(taddr + cg * 16, v);
                tmem_wait_ld();
                if (cg == MN / 16 - 1) {
                    // the accumulator is read out: the next tile but one may
                    // start its MMAs in it (in a pair, the even CTA's MMA
                    // thread counts both CTAs' epilogue warps)
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (PAIR && rank == 1)
                            mbar_arrive_cluster(mapa_shared(smem_u32(&bars->acc_empty[b]), 0));
                        else
                            mbar_arrive(&bars->acc_empty[b]);
                    }
                }
#pragma unroll
                for (int m = 0; m < 16; ++m) w[lane * 17 + m] = __uint_as_float(v[m]);
                __syncwarp();
                // lane k of the quad stores times m = k, k + 4, k + 8, k + 12
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int m = k + 4 * q;
                    const int t = tl.tt0 + cg * 16 + m;
                    const float4 o = make_float4(w[(quad + 0) * 17 + m], w[(quad + 1) * 17 + m],
                                                 w[(quad + 2) * 17 + m], w[(quad + 3) * 17 + m]);
                    if (station < p.S && t < p.T)
                        *reinterpret_cast<float4 *>(p.gx + (((size_t)tl.unit * p.S + station) * p.T + t) * 2) = o;
                }
                __syncwarp();
            }
        }
    } else if (!PAIR || rank == 0) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            constexpr uint32_t ID = idesc_tf32_f32(PAIR ? 2 * IG_M : IG_M, MN);
            auto mma = [&](uint32_t d, uint64_t a, uint64_t bdesc, uint32_t acc) {
                if constexpr (PAIR)
                    tc_mma_tf32_pair(d, a, bdesc, ID, acc);
                else
                    tc_mma_tf32(d, a, bdesc, ID, acc);
            };
            auto commit = [&](uint64_t *bar) {
                if constexpr (PAIR)
                    tc_commit_pair(bar, 3);   // the barrier at this offset in both CTAs
                else
                    tc_commit(bar);
            };
            long long g = 0;
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int b = i & 1;
                if (i >= 2 && !mbar_wait_bounded<PAIR>(&bars->acc_empty[b], (uint32_t)((i >> 1) - 1) & 1, abort_flag,
                                                 p.err, p.wait_ns))
                    break;
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * MN);
                for (int kb = 0; kb < KB; ++kb, ++g) {
                    const int s = (int)(g % IG_STAGES);
                    if (!mbar_wait_bounded<PAIR>(&bars->full[s], (uint32_t)(g / IG_STAGES) & 1, abort_flag, p.err,
                                           p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < IG_KV / 8; ++ks) {
                        const uint32_t o = 32u * ks;   // 8 tf32 of K per step
                        mma(acc, ig_desc(a_hi(s) + o), ig_desc(b_hi(s) + o), (kb | ks) ? 1u : 0u);
                        mma(acc, ig_desc(a_hi(s) + o), ig_desc(b_lo(s) + o), 1u);
                        mma(acc, ig_desc(a_lo(s) + o), ig_desc(b_hi(s) + o), 1u);
                    }
                    commit(&bars->empty[s]);
                }
                if (ok) commit(&bars->acc_full[b]);
            }
            // before TMEM is freed every MMA issued must have completed
            // (fixed 2 s bound)
            commit(&bars->done);
            int dummy = 0;
            mbar_wait_bounded(&bars->done, 0, &dummy, p.err, 2000000000ull);
        }
        __syncwarp();
    } else {
        // --------------------------------------- relay (odd CTA of a pair)
        // This CTA's split threads arrive on its own "full" barriers (CTA
        // scope); one thread follows the MMA thread's order and forwards
        // each completed phase to the even CTA with one cluster-scope
        // arrival.
        if (lane == 0) {
            long long g = 0;
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i)
                for (int kb = 0; kb < KB; ++kb, ++g) {
                    const int s = (int)(g % IG_STAGES);
                    if (!mbar_wait_bounded(&bars->full[s], (uint32_t)(g / IG_STAGES) & 1, abort_flag, p.err,
                                           p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(smem_u32(&bars->full[s]), 0));
                }
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    // a pair leaves together: the even CTA has seen its MMAs complete, and
    // the odd CTA's remote arrivals have all been made
    if constexpr (PAIR) cluster_sync();
    if (warp == IG_MMA_WARP) {
        tc_fence_after();
        if constexpr (PAIR)
            tmem_dealloc_pair(tmem, TMEM_COLS);
        else
            tmem_dealloc(tmem, TMEM_COLS);
    }
}

__global__ void __launch_bounds__(IG_THREADS, 1)
    input_grad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const IgParams p)
{
    ig_body<false>(xmap, p);
}

#if CORR_IG_N <= 128   // a pair's MMA is 2 IG_N wide, at most 256
#define CORR_IG_HAVE_PAIR 1
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(IG_THREADS, 1)
    input_grad_tc_pair_kernel(const __grid_constant__ CUtensorMap xmap, const IgParams p)
{
    ig_body<true>(xmap, p);
}
#else
#define CORR_IG_HAVE_PAIR 0
#endif

} // namespace

cudaError_t input_grad_tc_launch(const void *xmap, const IgParams &p, cudaStream_t s, bool pair)
{
    if (p.T <= 0 || p.units <= 0) return cudaSuccess;
    pair = pair && CORR_IG_HAVE_PAIR;
    const size_t smem = ig_smem_bytes();
#if CORR_IG_HAVE_PAIR
    const void *fn = pair ? (const void *)input_grad_tc_pair_kernel : (const void *)input_grad_tc_kernel;
#else
    const void *fn = (const void *)input_grad_tc_kernel;
#endif
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const CUtensorMap &m = *static_cast<const CUtensorMap *>(xmap);
#if CORR_IG_HAVE_PAIR
    if (pair) {
        const long long n_tiles =
            (long long)((p.T + 2 * IG_N - 1) / (2 * IG_N)) * ((p.m_tiles + 1) / 2) * p.units;
        const unsigned clusters = (unsigned)std::min<long long>(n_tiles, std::max(1, sms / 2));
        input_grad_tc_pair_kernel<<<2 * clusters, IG_THREADS, smem, s>>>(m, p);
        return cudaGetLastError();
    }
#endif
    {
        const long long n_tiles = (long long)((p.T + IG_N - 1) / IG_N) * p.m_tiles * p.units;
        const unsigned grid = (unsigned)std::min<long long>(n_tiles, std::max(1, sms));
        input_grad_tc_kernel<<<grid, IG_THREADS, smem, s>>>(m, p);
    }
    return cudaGetLastError();
}

} // namespace corr
