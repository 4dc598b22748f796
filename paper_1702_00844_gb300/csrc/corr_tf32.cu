// FP32 samples correlated on the tensor cores at FP32-class accuracy.
//
// The X-step of Section 2, V_ab = sum_t x_a(t) conj(x_b(t)) for a = (s1, p1),
// b = (s2, p2), s1 <= s2, written as real GEMMs over the time axis. Each
// operand row (station, pol) holds, per K-block of 16 samples, the 16 real
// parts and then the 16 imaginary parts (32 values, one 128-byte swizzle
// row), so with K-steps k0, k1 over the real parts and k2, k3 over the
// imaginary parts:
//     Re V += A[k0]B[k0] + A[k1]B[k1] + A[k2]B[k2] + A[k3]B[k3]
//     Im V += A[k2]B[k0] + A[k3]B[k1] - A[k0]B[k2] - A[k1]B[k3]   (negate-A bit)
// with A = the row block's stations and B = the column block's (the same
// tiles on a diagonal tile): 8 flops per complex multiply-add, the
// correlator's op count.
//
// tcgen05 has no FP32 MMA. Every operand value is split into hi = the value
// rounded to tf32 and lo = (value - hi), exact in FP32, of which the MMA
// uses the tf32 bits, and each product above is A_hi B_hi + A_hi B_lo +
// A_lo B_hi (kind::tf32, FP32 accumulation in TMEM; the dropped A_lo B_lo
// and lo's lost bits are at most about 2^-21 of each product): three MMAs
// per product, 24 per K-block.
//
// The tensor core adds each MMA's result to the FP32 accumulator with an
// error of about half an ulp of the running sum, biased toward zero, so a
// sum of n MMAs is off by about n/2 ulp: 0.75 T MMAs per output over T
// samples would reach 1.5e-5 of an autocorrelation at T = 768. So a tile
// accumulates in chunks of chunk_kb K-blocks (the first stored, the others
// added by the epilogue in FP32 with round to nearest): at 256 samples per
// chunk, 192 MMAs, about 6e-6.
//
// Tiles of (unit, 64-station row block rb, 64-station column block cb >= rb)
// over one persistent CTA per SM, each tile M = 128 rows (station, pol) x
// N = 128 columns, Re and Im in two TMEM column ranges, two accumulators
// alternating per chunk. Per K-block, through a ring of operand stages that
// runs on across the CTA's tiles:
//   - one thread issues TMA boxes of 16 samples x 64 stations (8-byte
//     elements, one complex per pol: one contiguous 256-byte run per
//     station) for the row block and, off the diagonal, the column block;
//     each lands station-major in its operand's lo tile;
//   - TF_SW warps read the raw samples (a pair of stations per warp and
//     iteration, conflict-free), meet on an mbarrier, transpose each quad of
//     lanes' 4 times x (X re, X im, Y re, Y im) in two shuffle rounds, and write hi
//     and lo chunks into the 128-byte swizzled K-major rows (chunk q of row
//     r at q ^ (r mod 8));
//   - one thread issues the 24 MMAs;
// and four warps store each finished accumulator (TMEM -> registers ->
// 16-byte stores of V[unit][baseline][p1][0..1]: per column station a warp
// writes 512 contiguous bytes) while the next tile's MMAs run in the other.
// Every wait is bounded (mbar_wait_bounded).
#include <cuda.h>

#include "corr_internal.h"
#include "ptx.cuh"

namespace corr {

namespace {

#ifndef CORR_TF_SPLIT_WARPS
#define CORR_TF_SPLIT_WARPS 8
#endif
// warp 0 loads, warps 1 .. SW split, the next four store (each a different
// TMEM lane quarter, warp % 4), the last allocates TMEM and issues the MMAs
constexpr int TF_SW = CORR_TF_SPLIT_WARPS;
constexpr int TF_SPLIT = 32 * TF_SW;     // split threads
constexpr int TF_MMA_WARP = TF_SW + 5;
constexpr int TF_THREADS = 32 * (TF_MMA_WARP + 1);
constexpr int TF_RS = 64;                // stations per block
constexpr int TF_KT = 16;                // samples per K-block
constexpr uint32_t TF_TILE = 128 * 128;  // 16 KB: 128 rows x 32 tf32
constexpr uint32_t TF_STAGE = 4 * TF_TILE;   // A hi, A lo, B hi, B lo
constexpr int TF_STAGES = 3;
constexpr uint32_t TF_TMEM_COLS = 512;   // 2 accumulators x (Re 128 + Im 128)

struct TfBars {
    uint64_t raw[TF_STAGES];     // loads landed (transaction bytes)
    uint64_t rd[TF_STAGES];      // raw samples read into registers (one arrival per split thread)
    uint64_t full[TF_STAGES];    // operands split (one arrival per split thread)
    uint64_t empty[TF_STAGES];   // MMAs of the stage done (commit)
    uint64_t acc_full[2];        // a tile's MMAs done (commit)
    uint64_t acc_empty[2];       // a tile's accumulator read out (4 warps)
    uint64_t done;               // every MMA issued has completed (commit)
    uint32_t tmem_base;
    int abort_flag;
};

constexpr size_t tf_smem_bytes() { return TF_STAGES * TF_STAGE + sizeof(TfBars) + 1024; }
static_assert(tf_smem_bytes() <= 227 * 1024, "tf32 correlator stages must fit in shared memory");

struct TfTile {
    int unit, rb, cb;
    int c0, c1;   // the item's accumulator chunks [c0, c1)
};

// Work item `item`: a tile of the flattened (unit, column block, row block
// <= column block) space with all its chunks, or (with p.partial) one chunk
// of a tile.
__device__ __forceinline__ TfTile tf_tile(long long item, int nch, const TfParams &p)
{
    const int ntri = p.nb * (p.nb + 1) / 2;
    TfTile r;
    long long tile = item;
    r.c0 = 0;
    r.c1 = nch;
    if (p.partial) {
        tile = item / nch;
        r.c0 = (int)(item % nch);
        r.c1 = r.c0 + 1;
    }
    r.unit = (int)(tile / ntri);
    int k = (int)(tile % ntri), cb = 0;
    while (k > cb) {
        k -= cb + 1;
        ++cb;
    }
    r.cb = cb;
    r.rb = k;
    return r;
}

__global__ void __launch_bounds__(TF_THREADS, 1)
    tf32_correlate_kernel(const __grid_constant__ CUtensorMap xmap, const TfParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t base = smem_u32(smem);
    TfBars *bars = reinterpret_cast<TfBars *>(smem + TF_STAGES * TF_STAGE);
    volatile int *abort_flag = &bars->abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KB = (p.T + TF_KT - 1) / TF_KT;
    const int nch = (KB + p.chunk_kb - 1) / p.chunk_kb;   // accumulator chunks per tile
    const long long n_items = (long long)p.units * (p.nb * (p.nb + 1) / 2) * (p.partial ? nch : 1);
    const int my_tiles = (int)((n_items - blockIdx.x + gridDim.x - 1) / gridDim.x);

    if (tid == 0) {
        prefetch_tmap(&xmap);
        for (int s = 0; s < TF_STAGES; ++s) {
            mbar_init(&bars->raw[s], 1);
            mbar_init(&bars->rd[s], TF_SPLIT);
            mbar_init(&bars->full[s], TF_SPLIT);
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], 4);
        }
        mbar_init(&bars->done, 1);
        bars->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == TF_MMA_WARP) {
        tmem_alloc(&bars->tmem_base, TF_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    auto a_hi = [&](int s) { return base + (uint32_t)s * TF_STAGE; };
    auto a_lo = [&](int s) { return a_hi(s) + TF_TILE; };
    auto b_hi = [&](int s) { return a_hi(s) + 2 * TF_TILE; };
    auto b_lo = [&](int s) { return a_hi(s) + 3 * TF_TILE; };

    if (warp == 0) {
        // ----------------------------------------------------------- loads
        if (lane == 0) {
            long long g = 0;   // K blocks issued so far (over all tiles)
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const TfTile tl = tf_tile(blockIdx.x + (long long)i * gridDim.x, nch, p);
                const bool diag = tl.rb == tl.cb;
                const int kb1 = min(KB, tl.c1 * p.chunk_kb);
                for (int kb = tl.c0 * p.chunk_kb; kb < kb1; ++kb, ++g) {
                    const int s = (int)(g % TF_STAGES);
                    if (g >= TF_STAGES && !mbar_wait_bounded(&bars->empty[s], (uint32_t)((g / TF_STAGES) - 1) & 1,
                                                             abort_flag, p.err, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&bars->raw[s], diag ? TF_TILE : 2 * TF_TILE);
                    // 16 samples x 2 pols (32 elements) x 64 stations from
                    // (time kb * 16, station rb * 64); zero outside
                    tma_load_4d(smem + (size_t)s * TF_STAGE + TF_TILE, &xmap, &bars->raw[s], 2 * kb * TF_KT,
                                tl.rb * TF_RS, tl.unit, 0);
                    if (!diag)
                        tma_load_4d(smem + (size_t)s * TF_STAGE + 3 * TF_TILE, &xmap, &bars->raw[s],
                                    2 * kb * TF_KT, tl.cb * TF_RS, tl.unit, 0);
                }
            }
            // on a give-up, let the copies in flight land before the CTA (and
            // its shared memory) goes away; fixed 2 s bound per stage
            if (*abort_flag) {
                int dummy = 0;
                for (long long q = g > TF_STAGES ? g - TF_STAGES : 0; q < g; ++q)
                    mbar_wait_bounded(&bars->raw[q % TF_STAGES], (uint32_t)(q / TF_STAGES) & 1, &dummy, p.err,
                                      2000000000ull);
            }
        }
        __syncwarp();
    } else if (warp <= TF_SW) {
        // ------------------------------------------------------------ split
        const int j = lane & 3;              // this lane's component after the transpose
        long long g = 0;
        bool ok = true;
        for (int i = 0; i < my_tiles && ok; ++i) {
            const TfTile tl = tf_tile(blockIdx.x + (long long)i * gridDim.x, nch, p);
            const int nops = tl.rb == tl.cb ? 1 : 2;
            const int kb1 = min(KB, tl.c1 * p.chunk_kb);
            for (int kb = tl.c0 * p.chunk_kb; kb < kb1; ++kb, ++g) {
                const int s = (int)(g % TF_STAGES);
                if (!mbar_wait_bounded(&bars->raw[s], (uint32_t)(g / TF_STAGES) & 1, abort_flag, p.err, p.wait_ns)) {
                    ok = false;
                    break;
                }
                // Each warp takes a pair of stations per iteration (pair
                // q * TF_SW + w); its lanes read 16-byte raw elements (station,
                // time) = (X re, X im, Y re, Y im) in quads of 4 consecutive
                // times. Lane l: quarter h = l / 8 takes station 2 pair +
                // h / 2 and the time quads {0, 3} (h even) or {1, 2} (h odd),
                // a pairing that keeps every quarter-warp's reads and its
                // swizzled writes on 8 distinct 16-byte bank groups.
                constexpr int NE = 32 / TF_SW;   // station pairs per warp and operand
                const int w = warp - 1, h = lane >> 3, m = (lane >> 2) & 1;
                const int st_off = h >> 1, tq = (h & 1) ? 1 + m : 3 * m;
                const int t = 4 * tq + (lane & 3);
                uint4 v[2][NE];
#pragma unroll
                for (int o = 0; o < 2; ++o)
                    if (o < nops) {
                        const uint32_t raw = o == 0 ? a_lo(s) : b_lo(s);
#pragma unroll
                        for (int q = 0; q < NE; ++q) {
                            const int st = 2 * (q * TF_SW + w) + st_off;
                            v[o][q] = lds128(raw + (uint32_t)((st * 16 + t) * 16));
                        }
                    }
                mbar_arrive(&bars->rd[s]);
                if (!mbar_wait_bounded(&bars->rd[s], (uint32_t)(g / TF_STAGES) & 1, abort_flag, p.err, p.wait_ns)) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int o = 0; o < 2; ++o)
                    if (o < nops) {
                        const uint32_t hi = o == 0 ? a_hi(s) : b_hi(s), lo = o == 0 ? a_lo(s) : b_lo(s);
#pragma unroll
                        for (int q = 0; q < NE; ++q) {
                            // 4 x 4 transpose within the quad (lane j: time j,
                            // components c0..c3) in two exchange rounds: with
                            // the partner across bit 0 keep components of
                            // parity j & 1 for both times of the pair, then with
                            // the partner across bit 1 keep component j for all
                            // four times
                            const uint4 c = v[o][q];
                            const bool b0 = (j & 1) != 0, b1 = (j & 2) != 0;
                            const uint32_t r0 = __shfl_xor_sync(0xffffffffu, b0 ? c.x : c.y, 1);
                            const uint32_t r1 = __shfl_xor_sync(0xffffffffu, b0 ? c.z : c.w, 1);
                            const uint32_t u0 = b0 ? r0 : c.x, u1 = b0 ? c.y : r0;
                            const uint32_t u2 = b0 ? r1 : c.z, u3 = b0 ? c.w : r1;
                            const uint32_t q0 = __shfl_xor_sync(0xffffffffu, b1 ? u0 : u2, 2);
                            const uint32_t q1 = __shfl_xor_sync(0xffffffffu, b1 ? u1 : u3, 2);
                            const float out[4] = {__uint_as_float(b1 ? q0 : u0), __uint_as_float(b1 ? q1 : u1),
                                                  __uint_as_float(b1 ? u2 : q0), __uint_as_float(b1 ? u3 : q1)};
                            const int st = 2 * (q * TF_SW + w) + st_off;
                            const int row = 2 * st + (j >> 1);
                            const int chunk = (j & 1) * 4 + tq;
                            const uint32_t sw = (uint32_t)(row * 128 + ((chunk ^ (row & 7)) * 16));
                            // hi = the tf32 rounding; lo = the exact remainder,
                            // whose bits below tf32 the MMA does not use (an
                            // error of at most 2^-21 of the value)
                            float hv[4], lv[4];
#pragma unroll
                            for (int mm = 0; mm < 4; ++mm) {
                                hv[mm] = tf32_round(out[mm]);
                                lv[mm] = out[mm] - hv[mm];
                            }
                            sts128(hi + sw, make_uint4(__float_as_uint(hv[0]), __float_as_uint(hv[1]),
                                                       __float_as_uint(hv[2]), __float_as_uint(hv[3])));
                            sts128(lo + sw, make_uint4(__float_as_uint(lv[0]), __float_as_uint(lv[1]),
                                                       __float_as_uint(lv[2]), __float_as_uint(lv[3])));
                        }
                    }
                fence_proxy_async_smem();
                mbar_arrive(&bars->full[s]);
            }
        }
    } else if (warp < TF_MMA_WARP) {
        // --------------------------------------------------------- epilogue
        // TMEM lanes of this warp: 32 * (warp % 4) ..; lane r of the tile is
        // row (station rb * 64 + r / 2, pol r % 2); column c is (station
        // cb * 64 + c / 2, pol c % 2), Re at column c, Im at 128 + c. A
        // tile's chunks arrive in order; the first is stored, the others
        // are added to what this same thread stored (FP32, round to
        // nearest).
        const int quarter = warp & 3;
        const long long B = (long long)p.S * (p.S + 1) / 2;
        uint32_t it = 0;   // accumulator items (tile chunks) so far
        bool ok = true;
        for (int i = 0; i < my_tiles && ok; ++i) {
            const TfTile tl = tf_tile(blockIdx.x + (long long)i * gridDim.x, nch, p);
            const int r = quarter * 32 + lane;
            const int s1 = tl.rb * TF_RS + r / 2, p1 = r & 1;
            for (int c = tl.c0; c < tl.c1; ++c, ++it) {
                // with partials, chunk c of every unit goes to its own copy
                // of the output (summed by tf32_reduce_kernel)
                float2 *out_u = (p.partial ? p.partial + (size_t)c * p.units * B * 4 : p.out) +
                                (size_t)tl.unit * B * 4;
                const bool add = !p.partial && c > 0;
                const uint32_t b = it & 1;
                // the warp leaves together (the TMEM loads below are warp-wide)
                const bool got =
                    mbar_wait_bounded(&bars->acc_full[b], (it >> 1) & 1, abort_flag, p.err, p.wait_ns);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + b * 256;
                for (int cg = 0; cg < 8; ++cg) {
                    uint32_t re[16], im[16];
                    tmem_ld_32x32b_x16(taddr + cg * 16, re);
                    tmem_ld_32x32b_x16(taddr + 128 + cg * 16, im);
                    tmem_wait_ld();
                    if (cg == 7) {
                        // the accumulator is read out: the next item but one
                        // may start its MMAs in it
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&bars->acc_empty[b]);
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int s2 = tl.cb * TF_RS + cg * 8 + k;
                        if (s1 <= s2 && s2 < p.S) {
                            const long long bl = (long long)s2 * (s2 + 1) / 2 + s1;
                            float4 *dst = reinterpret_cast<float4 *>(out_u + bl * 4 + p1 * 2);
                            float4 v = make_float4(__uint_as_float(re[2 * k]), __uint_as_float(im[2 * k]),
                                                   __uint_as_float(re[2 * k + 1]), __uint_as_float(im[2 * k + 1]));
                            if (add) {
                                const float4 o = *dst;
                                v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
                            }
                            *dst = v;
                        }
                    }
                }
            }
        }
    } else {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            constexpr uint32_t ID = idesc_tf32_f32(128, 128, false);
            constexpr uint32_t IDN = idesc_tf32_f32(128, 128, true);
            long long g = 0;
            uint32_t it = 0;
            bool ok = true;
            for (int i = 0; i < my_tiles && ok; ++i) {
                const TfTile tl = tf_tile(blockIdx.x + (long long)i * gridDim.x, nch, p);
                const bool diag = tl.rb == tl.cb;
                for (int c = tl.c0; c < tl.c1 && ok; ++c, ++it) {
                    const uint32_t b = it & 1;
                    if (it >= 2 && !mbar_wait_bounded(&bars->acc_empty[b], ((it >> 1) - 1) & 1, abort_flag, p.err,
                                                      p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t acc_re = tmem + b * 256, acc_im = acc_re + 128;
                    const int kb0 = c * p.chunk_kb, kb1 = min(KB, kb0 + p.chunk_kb);
                    for (int kb = kb0; kb < kb1; ++kb, ++g) {
                        const int s = (int)(g % TF_STAGES);
                        if (!mbar_wait_bounded(&bars->full[s], (uint32_t)(g / TF_STAGES) & 1, abort_flag, p.err,
                                               p.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t ah = a_hi(s), al = a_lo(s);
                        const uint32_t bh = diag ? ah : b_hi(s), bl = diag ? al : b_lo(s);
                        // the three split products of A[ka] B[kb]^T (32 bytes
                        // of K per step) into d
                        auto prod = [&](uint32_t d, uint32_t ka, uint32_t kbo, uint32_t id, uint32_t acc) {
                            tc_mma_tf32(d, smem_desc_sw128(ah + ka), smem_desc_sw128(bh + kbo), id, acc);
                            tc_mma_tf32(d, smem_desc_sw128(ah + ka), smem_desc_sw128(bl + kbo), id, 1u);
                            tc_mma_tf32(d, smem_desc_sw128(al + ka), smem_desc_sw128(bh + kbo), id, 1u);
                        };
                        const uint32_t first = kb == kb0 ? 0u : 1u;
                        // Re: real parts (steps 0, 1) and imaginary parts (2, 3)
                        prod(acc_re, 0, 0, ID, first);
                        prod(acc_re, 32, 32, ID, 1u);
                        prod(acc_re, 64, 64, ID, 1u);
                        prod(acc_re, 96, 96, ID, 1u);
                        // Im: A imaginary x B real, minus A real x B imaginary
                        prod(acc_im, 64, 0, ID, first);
                        prod(acc_im, 96, 32, ID, 1u);
                        prod(acc_im, 0, 64, IDN, 1u);
                        prod(acc_im, 32, 96, IDN, 1u);
                        tc_commit(&bars->empty[s]);
                    }
                    if (ok) tc_commit(&bars->acc_full[b]);
                }
            }
            // before TMEM is freed every MMA issued must have completed
            // (fixed 2 s bound)
            tc_commit(&bars->done);
            int dummy = 0;
            mbar_wait_bounded(&bars->done, 0, &dummy, p.err, 2000000000ull);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == TF_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, TF_TMEM_COLS);
    }
}

// out[i] = sum over the chunks c of partial[c][i], in the order of c (a
// fixed order: the result does not depend on the launch).
__global__ void __launch_bounds__(256) tf32_reduce_kernel(const float4 *partial, float4 *out, long long n, int nch)
{
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        float4 a = partial[i];
        for (int c = 1; c < nch; ++c) {
            const float4 b = partial[(size_t)c * n + i];
            a = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
        }
        out[i] = a;
    }
}

} // namespace

cudaError_t tf32_correlate_launch(const void *xmap, const TfParams &p, cudaStream_t s)
{
    if (p.T <= 0 || p.units <= 0) return cudaSuccess;
    const size_t smem = tf_smem_bytes();
    cudaError_t e =
        cudaFuncSetAttribute(tf32_correlate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int KB = (p.T + TF_KT - 1) / TF_KT, nch = (KB + p.chunk_kb - 1) / p.chunk_kb;
    const long long n_items = (long long)p.units * (p.nb * (p.nb + 1) / 2) * (p.partial ? nch : 1);
    const unsigned grid = (unsigned)std::min<long long>(n_items, std::max(1, sms));
    tf32_correlate_kernel<<<grid, TF_THREADS, smem, s>>>(*static_cast<const CUtensorMap *>(xmap), p);
    if ((e = cudaGetLastError()) != cudaSuccess || !p.partial) return e;
    // the chunks' partial sums, in chunk order
    const long long n = (long long)p.units * p.S * (p.S + 1) / 2;   // float4 per baseline (2 x 2 complex / 2)
    const long long n4 = n * 2;
    const unsigned rg = (unsigned)std::min<long long>((n4 + 255) / 256, 8LL * std::max(1, sms));
    tf32_reduce_kernel<<<rg, 256, 0, s>>>(reinterpret_cast<const float4 *>(p.partial),
                                          reinterpret_cast<float4 *>(p.out), n4, nch);
    return cudaGetLastError();
}

} // namespace corr
