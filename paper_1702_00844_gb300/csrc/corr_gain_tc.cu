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
// lo = (value - hi), exact in FP32, rounded to tf32 as well, and
//     A'B' ~ A_hi B_hi + A_hi B_lo + A_lo B_hi
// accumulated in FP32 (the dropped A_lo B_lo and lo's rounding are about
// 2^-22 of each product).
//
// One CTA per (channel, 128-row tile of M', 256-time tile of N). Per K-block
// of 32 reduction values (8 stations x 2 pols x re/im):
//   - one thread issues the loads: A_hi and A_lo as 16 KB bulk copies of
//     tiles that the gain-gradient kernel wrote already split and swizzled,
//     and the samples with one TMA box of 4 floats x 8 stations x 256 times,
//     which lands as 256 K-major rows (one time each) of 128 bytes (without
//     a swizzle mode: with one, TMA would give each 16-byte inner row of the
//     box a 128-byte span of its own);
//   - 128 threads split the samples into hi and lo and move each 16-byte
//     chunk j of row t to chunk j ^ (t mod 8), the 128-byte swizzled layout
//     the MMA reads (hi in place, lo in its own tile);
//   - one thread issues 4 K-steps x 3 MMAs (M = 128, N = 256, K = 8).
// The same 128 threads then store the accumulator: TMEM -> registers ->
// a per-warp transpose in shared memory -> 16-byte stores of (XX, YY)
// complex pairs of one station and time.
// Every wait is bounded (mbar_wait_bounded).
#include <cuda.h>

#include "corr_internal.h"
#include "ptx.cuh"

namespace corr {

namespace {

constexpr int IG_THREADS = 192;          // warp 0 loads, warps 1-4 split and store, warp 5 MMAs
constexpr int IG_M = 128, IG_N = 256;    // tile: rows of M' x times
constexpr int IG_STAGES = 2;
constexpr uint32_t IG_A_BYTES = IG_M * 128;      // 16 KB: 128 rows x 32 tf32
constexpr uint32_t IG_B_BYTES = IG_N * 128;      // 32 KB: 256 rows x 32 tf32
constexpr uint32_t IG_STAGE_BYTES = 2 * IG_A_BYTES + 2 * IG_B_BYTES;   // A hi, A lo, B hi, B lo
constexpr uint32_t IG_EPI_BYTES = 4 * 32 * 17 * 4;                       // per-warp transpose
constexpr uint32_t IG_TMEM_COLS = 256;

struct IgBars {
    uint64_t raw[IG_STAGES];     // loads landed (transaction bytes)
    uint64_t full[IG_STAGES];    // samples split (128 arrivals)
    uint64_t empty[IG_STAGES];   // MMAs of the stage done (commit)
    uint64_t acc_full;           // all MMAs done (commit)
    uint32_t tmem_base;
    int abort_flag;
};

constexpr size_t ig_smem_bytes() { return IG_STAGES * IG_STAGE_BYTES + IG_EPI_BYTES + sizeof(IgBars) + 1024; }
static_assert(ig_smem_bytes() <= 227 * 1024, "input-gradient tiles must fit in shared memory");

__global__ void __launch_bounds__(IG_THREADS, 1)
    input_grad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const IgParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t base = smem_u32(smem);
    float *epi = reinterpret_cast<float *>(smem + IG_STAGES * IG_STAGE_BYTES);
    IgBars *bars = reinterpret_cast<IgBars *>(smem + IG_STAGES * IG_STAGE_BYTES + IG_EPI_BYTES);
    volatile int *abort_flag = &bars->abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = blockIdx.x, mt = blockIdx.y, unit = p.unit0 + (int)blockIdx.z;
    const int t0 = nt * IG_N;
    const int KB = p.k_blocks;
    // A' tiles of this (unit, row tile): [k block][hi, lo][128 rows x 128 B]
    const uint8_t *a_tiles =
        reinterpret_cast<const uint8_t *>(p.at) + ((size_t)unit * p.m_tiles + mt) * (size_t)KB * 2 * IG_A_BYTES;

    if (tid == 0) {
        prefetch_tmap(&xmap);
        for (int s = 0; s < IG_STAGES; ++s) {
            mbar_init(&bars->raw[s], 1);
            mbar_init(&bars->full[s], 128);
            mbar_init(&bars->empty[s], 1);
        }
        mbar_init(&bars->acc_full, 1);
        bars->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 5) {
        tmem_alloc(&bars->tmem_base, IG_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    auto a_hi = [&](int s) { return base + (uint32_t)s * IG_STAGE_BYTES; };
    auto a_lo = [&](int s) { return a_hi(s) + IG_A_BYTES; };
    auto b_hi = [&](int s) { return a_hi(s) + 2 * IG_A_BYTES; };
    auto b_lo = [&](int s) { return b_hi(s) + IG_B_BYTES; };

    if (warp == 0) {
        // ----------------------------------------------------------- loads
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % IG_STAGES;
                if (kb >= IG_STAGES &&
                    !mbar_wait_bounded(&bars->empty[s], ((kb / IG_STAGES) - 1) & 1, abort_flag, p.err, p.wait_ns))
                    break;
                mbar_arrive_expect_tx(&bars->raw[s], 2 * IG_A_BYTES + IG_B_BYTES);
                bulk_load_g2s(a_hi(s), a_tiles + (size_t)kb * 2 * IG_A_BYTES, IG_A_BYTES, &bars->raw[s]);
                bulk_load_g2s(a_lo(s), a_tiles + (size_t)kb * 2 * IG_A_BYTES + IG_A_BYTES, IG_A_BYTES, &bars->raw[s]);
                // the 8 stations of this K block, 256 times from t0 (zero outside)
                tma_load_4d(smem + (size_t)s * IG_STAGE_BYTES + 2 * IG_A_BYTES, &xmap, &bars->raw[s], 0, kb * 8, t0,
                            unit);
                ++issued;
            }
            // on a give-up, let the copies in flight land before the CTA (and
            // its shared memory) goes away; fixed 2 s bound per stage
            if (*abort_flag) {
                int dummy = 0;
                for (int kb = issued > IG_STAGES ? issued - IG_STAGES : 0; kb < issued; ++kb)
                    mbar_wait_bounded(&bars->raw[kb % IG_STAGES], (kb / IG_STAGES) & 1, &dummy, p.err,
                                      2000000000ull);
            }
        }
        __syncwarp();
    } else if (warp <= 4) {
        // ---------------------------------------- split, then the epilogue
        const int pt = tid - 32;   // 0 .. 127
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            const int s = kb % IG_STAGES;
            if (!mbar_wait_bounded(&bars->raw[s], (kb / IG_STAGES) & 1, abort_flag, p.err, p.wait_ns)) {
                ok = false;
                break;
            }
            // 8 lanes per row: each reads one 16-byte chunk of the linear
            // row, the warp waits until all its rows are read, then each lane
            // writes hi and lo to the chunk's swizzled position (a row stays
            // within one warp, so no other warp touches it)
            const int wp = pt >> 5, j = lane & 7;
#pragma unroll 4
            for (int q = 0; q < IG_N / 16; ++q) {
                const int t = q * 16 + wp * 4 + (lane >> 3);
                const uint4 v = lds128(b_hi(s) + (uint32_t)(t * 128 + j * 16));
                __syncwarp();
                const float4 f = make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                             __uint_as_float(v.w));
                const float4 hf = make_float4(tf32_round(f.x), tf32_round(f.y), tf32_round(f.z), tf32_round(f.w));
                const uint4 h = make_uint4(__float_as_uint(hf.x), __float_as_uint(hf.y), __float_as_uint(hf.z),
                                           __float_as_uint(hf.w));
                const uint4 l = make_uint4(__float_as_uint(tf32_round(f.x - hf.x)), __float_as_uint(tf32_round(f.y - hf.y)),
                                           __float_as_uint(tf32_round(f.z - hf.z)), __float_as_uint(tf32_round(f.w - hf.w)));
                const uint32_t sw = (uint32_t)(t * 128 + ((j ^ (t & 7)) * 16));
                sts128(b_hi(s) + sw, h);
                sts128(b_lo(s) + sw, l);
            }
            fence_proxy_async_smem();
            mbar_arrive(&bars->full[s]);
        }
        if (ok && mbar_wait_bounded(&bars->acc_full, 0, abort_flag, p.err, p.wait_ns)) {
            tc_fence_after();
            // TMEM lanes of this warp: 32 * (warp % 4) ..; lane r of the tile
            // is row m = 128 mt + r of M': c = m / 2 = (station, pol), and
            // re (r even) or im. A quad of lanes holds (X re, X im, Y re, Y im)
            // of one station.
            const int quarter = warp & 3;
            const int r = quarter * 32 + lane;
            const int station = (IG_M * mt + quarter * 32) / 4 + (lane >> 2);
            float *w = epi + (size_t)quarter * 32 * 17;
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
            const int k = lane & 3, quad = lane & ~3;
            (void)r;
            for (int cg = 0; cg < IG_N / 16; ++cg) {
                uint32_t v[16];
                tmem_ld_32x32b_x16(taddr + cg * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int m = 0; m < 16; ++m) w[lane * 17 + m] = __uint_as_float(v[m]);
                __syncwarp();
                // lane k of the quad stores times m = k, k + 4, k + 8, k + 12
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int m = k + 4 * i;
                    const int t = t0 + cg * 16 + m;
                    const float4 o = make_float4(w[(quad + 0) * 17 + m], w[(quad + 1) * 17 + m],
                                                 w[(quad + 2) * 17 + m], w[(quad + 3) * 17 + m]);
                    if (station < p.S && t < p.T)
                        *reinterpret_cast<float4 *>(p.gx + (((size_t)unit * p.S + station) * p.T + t) * 2) = o;
                }
                __syncwarp();
            }
        }
    } else {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            constexpr uint32_t ID = idesc_tf32_f32(IG_M, IG_N);
            bool ok = true;
            for (int kb = 0; kb < KB && ok; ++kb) {
                const int s = kb % IG_STAGES;
                if (!mbar_wait_bounded(&bars->full[s], (kb / IG_STAGES) & 1, abort_flag, p.err, p.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t o = 32u * ks;   // 8 tf32 of K per step
                    tc_mma_tf32(tmem, smem_desc_sw128(a_hi(s) + o), smem_desc_sw128(b_hi(s) + o), ID,
                                (kb | ks) ? 1u : 0u);
                    tc_mma_tf32(tmem, smem_desc_sw128(a_hi(s) + o), smem_desc_sw128(b_lo(s) + o), ID, 1u);
                    tc_mma_tf32(tmem, smem_desc_sw128(a_lo(s) + o), smem_desc_sw128(b_hi(s) + o), ID, 1u);
                }
                tc_commit(&bars->empty[s]);
            }
            // the epilogue starts once every MMA has completed; on a give-up
            // the same commit tells when TMEM may be freed (fixed 2 s bound)
            tc_commit(&bars->acc_full);
            int dummy = 0;
            mbar_wait_bounded(&bars->acc_full, 0, &dummy, p.err, 2000000000ull);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tmem, IG_TMEM_COLS);
    }
}

} // namespace

cudaError_t input_grad_tc_launch(const void *xmap, const IgParams &p, cudaStream_t s)
{
    if (p.T <= 0) return cudaSuccess;
    const size_t smem = ig_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(input_grad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // at most 65535 units per launch (the grid's z dimension)
    for (int u0 = 0; u0 < p.units; u0 += 65535) {
        IgParams q = p;
        q.unit0 = u0;
        dim3 grid((unsigned)((p.T + IG_N - 1) / IG_N), (unsigned)p.m_tiles, (unsigned)std::min(65535, p.units - u0));
        input_grad_tc_kernel<<<grid, IG_THREADS, smem, s>>>(*static_cast<const CUtensorMap *>(xmap), q);
        if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

} // namespace corr
