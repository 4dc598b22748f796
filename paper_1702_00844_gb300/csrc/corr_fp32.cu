// FP32 CUDA-core correlator.
//
// Section 2's register tiling of the correlation triangle: each thread owns
// a 4x4-station tile (16 baselines x 4 polarisation pairs = 128 FP32
// accumulators kept in registers for the whole integration) and performs
// the conjugate multiply-add with four FMAs,
//     acc_r += a_r b_r + a_i b_i,   acc_i += a_i b_r - a_r b_i,
// issued as two packed FP32x2 FMAs on the (acc_r, acc_i) pair,
// reusing each loaded sample against 4 partner stations (Table 1, 4x4 tile:
// 512 flops per 128 bytes loaded). Tiles in the same row of the triangle are
// assigned to neighbouring threads so they consume the same samples at the
// same time (Section 2's inter-tile reuse through co-scheduling).
//
// Registers are capped at 168 per thread and CTAs at 192 threads so that two
// CTAs share an SM (at most 3 warps per SM sub-partition). Up to 64 stations
// the sub-tiles are 4 x 2 stations instead (64 accumulators, 96 registers,
// CTAs of up to 288 compute threads plus one warp that only issues the TMA
// loads): the same FMAs per accumulator in the same order, on more threads.
//
// One polarisation (NPOL = 1): stations 2m and 2m+1 act as the two pols of
// pseudo-station m. A box of 16 stations x tc samples of 8-byte complex
// values, stored time-major, is byte for byte a box of 8 pseudo-stations of
// 16-byte two-pol samples, so the arithmetic is unchanged. Those boxes are
// staged with 8-byte asynchronous copies by all threads (a TMA box needs an
// innermost extent of 16 bytes), and only the output mapping differs.
//
// Samples are staged by TMA: each stage holds `tc` samples of every station
// the CTA needs, as boxes of 8 stations stored time-major
// ([box][t][8 stations][2 pols x complex]). Thread j reads its four column
// stations in the rotated order 4j + ((k + j/2) mod 4) so that the 8
// threads of a quarter-warp read 8 distinct 16-byte bank groups; the rotation
// is undone when the result is stored.
#include <cuda.h>

#include <algorithm>

#include "corr_internal.h"
#include "ptx.cuh"

namespace corr {

namespace {

__device__ __forceinline__ uint64_t pack2(float lo, float hi)
{
    uint64_t v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(lo), "f"(hi));
    return v;
}

// (lo, hi) += (a.lo * b.lo, a.hi * b.hi): two fused multiply-adds, each
// rounded to nearest, in one packed instruction.
__device__ __forceinline__ void fma2(float &lo, float &hi, uint64_t a, uint64_t b)
{
    asm("{\n\t.reg .b64 q;\n\t"
        "mov.b64 q, {%0, %1};\n\t"
        "fma.rn.f32x2 q, %2, %3, q;\n\t"
        "mov.b64 {%0, %1}, q;\n\t}"
        : "+f"(lo), "+f"(hi)
        : "l"(a), "l"(b));
}

// Sub-tile k of the row-major upper triangle of 4 x TW-station sub-tiles:
// row i (stations 4i .. 4i+3) holds column groups j = 4i/TW .. ncq-1 (stations
// TW j .. TW j + TW - 1).
template <int TW> __device__ __forceinline__ void decode_subtile(int ncq, int k, int &i, int &j)
{
    int row = 0, off = 0;
    while (k >= off + (ncq - 4 * row / TW)) {
        off += ncq - 4 * row / TW;
        ++row;
    }
    i = row;
    j = 4 * row / TW + (k - off);
}

// Column station of sub-tile column j, lane b, rotated so that the 8 threads
// of a quarter-warp (consecutive j) read 8 distinct 16-byte bank groups.
template <int TW> __device__ __forceinline__ int col_station(int j, int b)
{
    return TW * j + (TW == 4 ? ((b + (j >> 1)) & 3) : ((b + (j >> 2)) & 1));
}

// Waits for the TMA loads of chunks kc .. kc + STAGES - 1 (those issued by
// the time chunk kc is consumed) to land; fixed 2 s bound per stage. Called
// only when the kernel gives up, before the CTA exits.
__device__ __noinline__ void drain_issued(uint64_t *full, int kc, int nchunks, int *err)
{
    int dummy = 0;
    for (int c = kc; c < min(nchunks, kc + FP32_STAGES); ++c)
        mbar_wait_bounded(&full[c % FP32_STAGES], (c / FP32_STAGES) & 1, &dummy, err, 2000000000ull);
}

// One polarisation: copies chunk kc (tc samples) of stations 2*s_lo ..
// 2*s_lo + 16*nbox - 1 into the stage at shared address `base`, laid out
// [box][t][16 stations][8 bytes]; this thread takes elements tid, tid +
// nthreads, ... (time fastest); zero fill outside the array. Ends one
// commit group (empty past the last chunk). Kept out of line so that its
// registers do not compete with the accumulators.
__device__ __noinline__ void stage_single_pol(uint32_t base, const float2 *in1u, const float2 *any,
                                              int S1, int T, int tc, int s_lo, int nbox, int kc,
                                              int nchunks, int tid, int nthreads)
{
    if (kc < nchunks) {
        const int n = nbox * 16 * tc;
        for (int e = tid; e < n; e += nthreads) {
            const int tl = e % tc, sl16 = e / tc; // station offset from 2 * s_lo
            const int s = 2 * s_lo + sl16, t = kc * tc + tl;
            const uint32_t dst = base + (uint32_t)(((sl16 >> 4) * tc + tl) * 16 + (sl16 & 15)) * 8u;
            const bool in = s < S1 && t < T;
            cp_async_small<8>(dst, in ? in1u + (size_t)s * T + t : any, in ? 8u : 0u);
        }
    }
    cp_async_commit();
}

// TW = 4: 4 x 4-station sub-tiles (128 accumulators, 168 registers, CTAs of
// at most 192 threads); TW = 2: 4 x 2 (64 accumulators, 96 registers, CTAs of
// at most 288 threads). A warp's registers come from one SM sub-partition's
// 64 KB file: 168 registers allow 3 warps per sub-partition (two 5-warp
// CTAs), 96 allow 5 (two 9-warp CTAs).
template <int NPOL, int TW>
__global__ void __maxnreg__(TW == 4 ? 168 : 96) fp32_correlate_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                       const Fp32Params p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ uint64_t full[FP32_STAGES];
    __shared__ uint64_t empty[FP32_STAGES];
    __shared__ int abort_flag;

    // With TMA staging and p.load_warp: one extra warp (the last) issues the
    // loads, and each compute warp releases a stage on its own (one arrival
    // per warp on the stage's "empty" barrier), so warps meet no block
    // barrier per stage and can drift apart by up to FP32_STAGES - 1 stages.
    const bool PW = NPOL == 2 && TW == 2 && p.load_warp;
    const int ncomp = PW ? (int)blockDim.x - 32 : (int)blockDim.x;
    const int tid = threadIdx.x;
    const int grp = blockIdx.x % p.groups;
    const int unit = (blockIdx.x / p.groups) % p.n_units;
    const int kpart = blockIdx.x / (p.groups * p.n_units);   // range of the sample axis
    const int k_first = grp * p.group_size;
    const int k = k_first + tid;
    const bool active = tid < p.group_size && k < p.nsub;

    int i, j, i_first, j_first;
    decode_subtile<TW>(p.ncq, active ? k : k_first, i, j);
    decode_subtile<TW>(p.ncq, k_first, i_first, j_first);
    const int s_lo = (4 * i_first) & ~7;
    const int nbox = (p.S - s_lo + 7) / 8;
    const int box_f4 = p.tc * 8;                 // float4 per box
    const int stage_f4 = nbox * box_f4;
    const uint32_t stage_bytes = (uint32_t)stage_f4 * 16u;
    // this CTA's chunks: kc0 .. kc0 + nchunks - 1 of the whole sample axis
    const int kc0 = kpart * p.kchunks;
    const int nchunks = min(p.kchunks, (p.T + p.tc - 1) / p.tc - kc0);

    if (tid == 0) {
        if (NPOL == 2) prefetch_tmap(&tmap);
        for (int s = 0; s < FP32_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (uint32_t)(ncomp / 32));
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int kc) {
        const int st = kc % FP32_STAGES;
        mbar_arrive_expect_tx(&full[st], stage_bytes);
        for (int b = 0; b < nbox; ++b)
            tma_load_4d(smem + (size_t)st * stage_bytes + (size_t)b * box_f4 * 16, &tmap, &full[st],
                        0, s_lo + 8 * b, (kc0 + kc) * p.tc, unit);
    };
    // NPOL = 1: every thread copies its share of the stage's (station, time)
    // values (time fastest, so a warp reads contiguous samples of a station);
    // one commit group per stage, zero fill outside the array.
    auto issue1 = [&](int kc) {
        stage_single_pol(smem_u32(smem) + (uint32_t)(kc % FP32_STAGES) * stage_bytes,
                         p.in1 + (size_t)unit * p.S1 * p.T, p.in1, p.S1, p.T, p.tc, s_lo, nbox, kc0 + kc,
                         kc0 + nchunks, tid, (int)blockDim.x);
    };
    if (NPOL == 1) {
        for (int kc = 0; kc < FP32_STAGES; ++kc) issue1(kc);
    } else if (!PW && tid == 0) {
        for (int kc = 0; kc < FP32_STAGES && kc < nchunks; ++kc) issue(kc);
    }
    if (PW && tid >= ncomp) {
        // the load warp: refills stage kc % FP32_STAGES once every compute
        // warp has released its previous use
        if (tid == ncomp) {
            int issued = 0;
            for (int kc = 0; kc < nchunks; ++kc) {
                const int st = kc % FP32_STAGES;
                if (kc >= FP32_STAGES &&
                    !mbar_wait_bounded(&empty[st], ((kc / FP32_STAGES) - 1) & 1, &abort_flag, p.err, p.wait_ns))
                    break;
                issue(kc);
                ++issued;
            }
            // on a give-up, let the loads in flight land before the CTA (and
            // its shared memory) goes away; fixed 2 s bound per stage
            if (abort_flag) drain_issued(full, max(0, issued - FP32_STAGES), issued, p.err);
        }
        return;
    }

    int row_off[4], col_off[TW];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = 4 * i + a - s_lo;
        row_off[a] = (r >> 3) * box_f4 + (r & 7);
    }
#pragma unroll
    for (int b = 0; b < TW; ++b) {
        const int c = col_station<TW>(j, b) - s_lo;
        col_off[b] = (c >> 3) * box_f4 + (c & 7);
    }

    float acc[4][TW][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < TW; ++b)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[a][b][q] = 0.f;

    const float4 *sm4 = reinterpret_cast<const float4 *>(smem);
    for (int kc = 0; kc < nchunks; ++kc) {
        const int st = kc % FP32_STAGES;
        bool ok = true;
        if (NPOL == 1) {
            cp_async_wait<FP32_STAGES - 1>(); // this thread's copies of chunk kc
            __syncthreads();                  // everyone's
        } else {
            ok = mbar_wait_bounded(&full[st], (kc / FP32_STAGES) & 1, &abort_flag, p.err, p.wait_ns);
        }
        if (ok) {
            const float4 *base = sm4 + (size_t)st * stage_f4;
            const int tn = min(p.tc, p.T - (kc0 + kc) * p.tc);
#pragma unroll 1
            for (int t = 0; t < tn; ++t) {
                float4 r[4], c[TW];
#pragma unroll
                for (int a = 0; a < 4; ++a) r[a] = base[row_off[a] + t * 8];
#pragma unroll
                for (int b = 0; b < TW; ++b) c[b] = base[col_off[b] + t * 8];
                // The four FMAs of each complex multiply-add as two packed
                // FMAs on the (re, im) accumulator pair of pol pair (p1, p2):
                //   (re, im) += (r_re, r_im) * (c_re, c_re)
                //   (re, im) += (r_im, -r_re) * (c_im, c_im)
                // the same fused operations in the same order as
                //   re += r_re c_re + r_im c_im,   im += r_im c_re - r_re c_im.
                uint64_t R1[4][2], R2[4][2], C1[TW][2], C2[TW][2];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    R1[a][0] = pack2(r[a].x, r[a].y);
                    R2[a][0] = pack2(r[a].y, -r[a].x);
                    R1[a][1] = pack2(r[a].z, r[a].w);
                    R2[a][1] = pack2(r[a].w, -r[a].z);
                }
#pragma unroll
                for (int b = 0; b < TW; ++b) {
                    C1[b][0] = pack2(c[b].x, c[b].x);
                    C2[b][0] = pack2(c[b].y, c[b].y);
                    C1[b][1] = pack2(c[b].z, c[b].z);
                    C2[b][1] = pack2(c[b].w, c[b].w);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < TW; ++b)
#pragma unroll
                        for (int pp = 0; pp < 4; ++pp) { // (p1, p2) = (pp >> 1, pp & 1)
                            fma2(acc[a][b][2 * pp], acc[a][b][2 * pp + 1], R1[a][pp >> 1], C1[b][pp & 1]);
                            fma2(acc[a][b][2 * pp], acc[a][b][2 * pp + 1], R2[a][pp >> 1], C2[b][pp & 1]);
                        }
            }
        }
        if (PW) {
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[st]);
            if (!ok || abort_flag) break;
            continue;
        }
        __syncthreads();
        if (NPOL == 1) {
            issue1(kc + FP32_STAGES);
            continue;
        }
        if (abort_flag) {
            // Let every issued TMA load land before the CTA (and its shared
            // memory) goes away; fixed 2 s bound per stage.
            if (tid == 0) drain_issued(full, kc, nchunks, p.err);
            break;
        }
        if (tid == 0 && kc + FP32_STAGES < nchunks) issue(kc + FP32_STAGES);
    }
    if (NPOL == 1) cp_async_wait<0>();

    if (!active || abort_flag) return;
    if (NPOL == 1) {
        // pseudo rows 4i+a (stations 2(4i+a)+p1) x pseudo columns (stations
        // 2 col + p2); one complex per baseline
        const long long B1 = (long long)p.S1 * (p.S1 + 1) / 2;
        float2 *out = (p.partial ? p.partial + (long long)kpart * p.n_units * B1 : p.out) + (long long)unit * B1;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < TW; ++b) {
                const int m1 = 4 * i + a, m2 = col_station<TW>(j, b);
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    const int s1 = 2 * m1 + (pp >> 1), s2 = 2 * m2 + (pp & 1);
                    if (s1 <= s2 && s2 < p.S1)
                        out[(long long)s2 * (s2 + 1) / 2 + s1] =
                            make_float2(acc[a][b][2 * pp], acc[a][b][2 * pp + 1]);
                }
            }
        return;
    }
    const long long B = (long long)p.S * (p.S + 1) / 2;
    float2 *out = (p.partial ? p.partial + (long long)kpart * p.n_units * B * 4 : p.out) +
                  (long long)unit * B * 4;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int s1 = 4 * i + a;
#pragma unroll
        for (int b = 0; b < TW; ++b) {
            const int s2 = col_station<TW>(j, b);
            if (s1 <= s2 && s2 < p.S) {
                float4 *dst = reinterpret_cast<float4 *>(out + ((long long)s2 * (s2 + 1) / 2 + s1) * 4);
                dst[0] = make_float4(acc[a][b][0], acc[a][b][1], acc[a][b][2], acc[a][b][3]);
                dst[1] = make_float4(acc[a][b][4], acc[a][b][5], acc[a][b][6], acc[a][b][7]);
            }
        }
    }
}

} // namespace

// out[i] = sum over k of partial[k][i], k in order (deterministic).
__global__ void __launch_bounds__(256) fp32_reduce_kernel(const float2 *__restrict__ partial,
                                                          float2 *__restrict__ out, long long n, int ksplit)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float2 a = __ldg(partial + i);
        for (int k = 1; k < ksplit; ++k) {
            const float2 b = __ldg(partial + (long long)k * n + i);
            a.x += b.x;
            a.y += b.y;
        }
        out[i] = a;
    }
}

// Sums the ksplit partial results of a launch: units x baselines x pol
// pairs complex values each.
cudaError_t fp32_reduce(const Fp32Params &p, int npol, cudaStream_t s)
{
    const long long B = (long long)p.S1 * (p.S1 + 1) / 2;
    const long long n = (long long)p.n_units * B * npol * npol;
    const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
    fp32_reduce_kernel<<<(unsigned)std::max(1LL, blocks), 256, 0, s>>>(p.partial, p.out, n, p.ksplit);
    return cudaGetLastError();
}

namespace {

template <int NPOL, int TW>
cudaError_t launch_tw(const void *tmap, const Fp32Params &p, int threads, size_t smem, cudaStream_t s)
{
    const unsigned grid = (unsigned)(p.n_units * p.groups * p.ksplit);
    cudaError_t e = cudaFuncSetAttribute(fp32_correlate_kernel<NPOL, TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // all of the unified L1/shared array as shared memory, so that two CTAs'
    // stages fit an SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fp32_correlate_kernel<NPOL, TW>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (NPOL == 1) {
        CUtensorMap unused{};
        fp32_correlate_kernel<NPOL, TW><<<grid, threads, smem, s>>>(unused, p);
    } else {
        fp32_correlate_kernel<NPOL, TW><<<grid, threads, smem, s>>>(*static_cast<const CUtensorMap *>(tmap), p);
    }
    e = cudaGetLastError();
    return (e == cudaSuccess && p.partial) ? fp32_reduce(p, NPOL, s) : e;
}

} // namespace

cudaError_t fp32_launch(const void *tmap, const Fp32Params &p, int npol, int threads, size_t smem,
                        cudaStream_t s)
{
    if (npol == 1)
        return p.tw == 2 ? launch_tw<1, 2>(tmap, p, threads, smem, s) : launch_tw<1, 4>(tmap, p, threads, smem, s);
    return p.tw == 2 ? launch_tw<2, 2>(tmap, p, threads, smem, s) : launch_tw<2, 4>(tmap, p, threads, smem, s);
}

} // namespace corr
