// Tensor-core correlator (tcgen05, kind::f16, FP32 accumulation in TMEM).
//
// Per channel the X-step of Section 2 is the Hermitian product V = X X^H of
// the (station, pol) x time sample matrix. With a = x_{s1,p1}(t) and
// b = x_{s2,p2}(t),
//     Re V_ab = sum_t (a_r b_r + a_i b_i),   Im V_ab = sum_t (a_i b_r - a_r b_i),
// i.e. the four FMAs of Section 2 expressed as real matrix products. Each
// operand row (station, pol) holds, per block of 32 samples, the 32 real
// parts followed by the 32 imaginary parts (64 f16 = one 128-byte swizzle
// row). With K-steps k0,k1 = real parts and k2,k3 = imaginary parts:
//     Re += A[k0]B[k0] + A[k1]B[k1] + A[k2]B[k2] + A[k3]B[k3]
//     Im += A[k2]B[k0] + A[k3]B[k1] - A[k0]B[k2] - A[k1]B[k3]   (negate-A bit)
// so no rotated copy of either operand is needed.
//
// Work is a triangular schedule of tiles over the correlation triangle
// (Section 2's tiling; blocks of stations as for large station counts in
// Section 4.5): the row block is 64 stations (M = 128 rows), the column range
// one block of 64 stations (N = 128, "narrow") or up to two (N = 256,
// "wide"), starting at or after the row block. A persistent CTA per SM walks
// its share of the (problem, channel, tile) list.
//
// "pair": a cluster of two CTAs on two SMs works on one 128 x 128-station
// tile with CTA-pair MMAs (M = 256, N = 256): each CTA stages its own row
// block (rb + rank) and one of the two column blocks (cb0 + rank), so per SM
// the tensor core reads half as much B per MMA as in "wide" and the
// producers stage two blocks per K-block instead of three. Each CTA's TMEM
// holds its row block against both column blocks; each CTA stores its own
// rows. Work items are taken per cluster.
//
// Warp roles (416 threads):
//   warps 0-7  : stage raw samples with 16-byte asynchronous copies into a
//                per-thread ring in shared memory (each thread later converts
//                exactly the bytes it copied, so the ring needs no barrier;
//                int8 pair tiles load into a ring of registers instead),
//                widen int8 to f16 exactly, split polarisations and
//                real/imaginary parts, and store the operand tiles in the
//                128-byte swizzled K-major layout of a ring of operand stages.
//   warps 8-11 : epilogue: TMEM -> registers, mask s1 <= s2, store
//                [channel][baseline][p1][p2] once (int8: fold each 512-sample
//                chunk into INT32 exactly);
//   warp 12    : allocates TMEM (narrow: 2 accumulator buffers x (Re 128 +
//                Im 128) columns; wide and pair: 1 buffer x (Re 256 + Im 256))
//                and issues the MMAs (one thread; in a pair, of the even CTA).
// Every wait is bounded (see mbar_wait_bounded).
#include "corr_tc_internal.h"
#include "ptx.cuh"

namespace corr {

namespace {

constexpr int TILE_BYTES = 128 * 128; // one operand block: 128 rows x 128 B

// 13 warps: 8 producers, 4 epilogue (one per TMEM lane quarter), 1 MMA.
constexpr int N_PROD_WARPS = 8;
constexpr int N_PRODUCERS = N_PROD_WARPS * 32; // 256
constexpr int N_EPILOGUE = 128;
constexpr int WARP_MMA = 12;
static_assert(TC_THREADS == 13 * 32, "warp roles");
constexpr uint32_t TMEM_COLS = 512;

// Bytes of one unit of raw samples (8 times of one station, both pols).
template <int DT> struct RawBytes { static constexpr int value = DT == 1 ? 64 : 32; };

// Per input type and tile width: operand stages, raw stages, operand blocks
// of B per tile and TMEM accumulator buffers.
#ifndef CORR_TC_OPS_F16
#define CORR_TC_OPS_F16 3
#endif
#ifndef CORR_TC_RAW_F16
#define CORR_TC_RAW_F16 3
#endif
#ifndef CORR_TC_OPS_I8
#define CORR_TC_OPS_I8 4
#endif
#ifndef CORR_TC_RAW_I8
#define CORR_TC_RAW_I8 5
#endif
#ifndef CORR_TC_OPS_PAIR_F16
#define CORR_TC_OPS_PAIR_F16 5
#endif
#ifndef CORR_TC_RAW_PAIR_F16
#define CORR_TC_RAW_PAIR_F16 2
#endif
#ifndef CORR_TC_OPS_PAIR_I8
#define CORR_TC_OPS_PAIR_I8 4
#endif
#ifndef CORR_TC_RAW_PAIR_I8
#define CORR_TC_RAW_PAIR_I8 5
#endif
// int8 pair producers load samples straight into a ring of registers (PF
// K-blocks ahead) instead of staging them in shared memory (RAW = 0 selects
// it). The freed shared memory deepens the operand ring. On the 256-station
// workload this measured 1-2% faster for pair tiles and slower for narrow and
// wide tiles, which keep the asynchronous-copy ring.
#ifndef CORR_TC_REGPF
#define CORR_TC_REGPF 1
#endif
#ifndef CORR_TC_PF
#define CORR_TC_PF 4
#endif
#ifndef CORR_TC_OPS_REG_PAIR_I8
#define CORR_TC_OPS_REG_PAIR_I8 6
#endif
constexpr int MAX_OPS = 6; // size of the stage barrier arrays
template <int DT, int V> struct Cfg;
template <> struct Cfg<1, TC_NARROW> {
    static constexpr int OPS = CORR_TC_OPS_F16, RAW = CORR_TC_RAW_F16, MAXB = 1, NBUF = 2;
};
template <> struct Cfg<1, TC_WIDE> { static constexpr int OPS = 2, RAW = 2, MAXB = 2, NBUF = 1; };
template <> struct Cfg<1, TC_PAIR> {
    static constexpr int OPS = CORR_TC_OPS_PAIR_F16, RAW = CORR_TC_RAW_PAIR_F16, MAXB = 1, NBUF = 1;
};
template <> struct Cfg<2, TC_NARROW> {
    static constexpr int OPS = CORR_TC_OPS_I8, RAW = CORR_TC_RAW_I8, MAXB = 1, NBUF = 2;
};
template <> struct Cfg<2, TC_WIDE> { static constexpr int OPS = 3, RAW = 3, MAXB = 2, NBUF = 1; };
#if CORR_TC_REGPF
template <> struct Cfg<2, TC_PAIR> {
    static constexpr int OPS = CORR_TC_OPS_REG_PAIR_I8, RAW = 0, MAXB = 1, NBUF = 1;
};
#else
template <> struct Cfg<2, TC_PAIR> {
    static constexpr int OPS = CORR_TC_OPS_PAIR_I8, RAW = CORR_TC_RAW_PAIR_I8, MAXB = 1, NBUF = 1;
};
#endif

// int8 pair tiles stage the epilogue's last column groups in shared memory:
// STG groups of 8 column (pseudo-)stations (4 KB per epilogue warp), copied
// there raw from TMEM so that the accumulator is released sooner; their
// conversion and global stores follow while the next tile's MMAs run. The
// operand ring is one stage shorter to make room. Measured on 256 stations:
// 4 operand stages + 6 staged groups 1-1.5% faster than 6 stages without
// staging (3 + 8: equal; f16 pair tiles: slower, so STG = 0 there); one pol
// (512 stations), 4% faster.
#ifndef CORR_TC_OPS_STG_I8
#define CORR_TC_OPS_STG_I8 4
#endif
#ifndef CORR_TC_STG_I8
#define CORR_TC_STG_I8 6
#endif
constexpr int STG_GROUP_BYTES = 8 * 512;  // per warp: 8 column stations x 32 rows x 16 B

// Stage counts per (input type, tile variant, pols, layout): OPS operand
// stages, RAW raw-sample stages, STG staged epilogue groups per epilogue
// warp. Layout LY = 1 (int8 pair tiles of two pols only, a second
// instantiation the autotuner can choose) keeps the six-stage operand ring
// and stores every epilogue group directly.
template <int DT, int V, int NPOL, int LY = 0> struct Lay {
    static constexpr bool STAGED = V == TC_PAIR && DT == 2 && LY == 0 && CORR_TC_STG_I8 > 0;
    static constexpr int STG = STAGED ? CORR_TC_STG_I8 : 0;
    static constexpr int OPS = STAGED ? CORR_TC_OPS_STG_I8 : Cfg<DT, V>::OPS;
    static constexpr int RAW = Cfg<DT, V>::RAW;
};

template <int DT, int V> __host__ __device__ constexpr int stage_bytes()
{
    return (1 + Cfg<DT, V>::MAXB) * TILE_BYTES;
}
template <int DT, int V> __host__ __device__ constexpr int raw_stage_bytes()
{
    return (1 + Cfg<DT, V>::MAXB) * RawBytes<DT>::value * N_PRODUCERS;
}
template <int DT, int V, int NPOL, int LY = 0> __host__ __device__ constexpr int smem_bytes()
{
    using L = Lay<DT, V, NPOL, LY>;
    return L::OPS * stage_bytes<DT, V>() + L::RAW * raw_stage_bytes<DT, V>() +
           L::STG * 4 * STG_GROUP_BYTES;
}

struct Bars {
    uint64_t full[MAX_OPS];
    uint64_t empty[MAX_OPS];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t fin;
    uint32_t tmem_base;
    int abort_flag;
};

template <int DT, int V, int NPOL, int LY = 0> constexpr bool cfg_ok()
{
    using L = Lay<DT, V, NPOL, LY>;
    return L::OPS >= 2 && L::OPS <= MAX_OPS && (L::RAW >= 2 || (L::RAW == 0 && DT == 2)) &&
           L::STG >= 0 && L::STG <= 16 &&
           smem_bytes<DT, V, NPOL, LY>() + (int)sizeof(Bars) + 1024 <= 227 * 1024;
}
template <int DT> constexpr bool cfg_ok_dt()
{
    return cfg_ok<DT, TC_NARROW, 1>() && cfg_ok<DT, TC_NARROW, 2>() && cfg_ok<DT, TC_WIDE, 1>() &&
           cfg_ok<DT, TC_WIDE, 2>() && cfg_ok<DT, TC_PAIR, 1>() && cfg_ok<DT, TC_PAIR, 2>();
}
static_assert(cfg_ok_dt<1>() && cfg_ok_dt<2>() && cfg_ok<2, TC_PAIR, 2, 1>(),
              "stage counts must fit the barrier arrays and shared memory");

template <int DT> struct Raw;          // raw samples of 8 times of one station
template <> struct Raw<1> { uint4 v[4]; }; // complex f16 x 2 pols: 64 bytes
template <> struct Raw<2> { uint4 v[2]; }; // complex int8 x 2 pols: 32 bytes

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Issues the asynchronous copies of one unit: station s, chunks g, g+4, ...
// (16 bytes each) of the K-block starting at sample t0, into the unit's slot
// (chunk q at dst + q*chunk_stride). The four threads of a station thus read
// 64 contiguous bytes per copy instruction. The unit holds 8 samples that are
// not consecutive in time; A and B use the same assignment, so the products
// pair the same samples. Samples outside [0,S) x [0,T) are zero-filled. With
// vec (rows of whole 16-byte chunks) 16-byte copies are used, otherwise one
// copy per sample.
template <int DT, int NPOL>
__device__ __forceinline__ void issue_raw(const uint8_t *unit_in, int S, int T, bool vec, int s,
                                          int t0, int g, uint32_t dst, uint32_t chunk_stride)
{
    if constexpr (NPOL == 1) {
        // Single polarisation: s is a pseudo-station, stations 2s and 2s+1
        // play its two pols. Chunk q = (station parity p, half h): samples
        // t0 + 8g + 4h*(DT == 1) .. of station 2s + p, 16 bytes each.
        constexpr int BPS = DT == 1 ? 4 : 2;  // bytes per sample of one station
        constexpr int HALVES = DT == 1 ? 2 : 1;
        constexpr int TPC = 16 / BPS;         // samples per chunk
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int st = 2 * s + p;
            const bool srow = st < S;
            const uint8_t *row = unit_in + (srow ? (size_t)st * T * BPS : 0);
#pragma unroll
            for (int h = 0; h < HALVES; ++h) {
                const uint32_t d = dst + (p * HALVES + h) * chunk_stride;
                const int tq = t0 + 8 * g + h * TPC;
                if (vec) {
                    int nb = srow ? (T - tq) * BPS : 0;
                    nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
                    cp_async16(d, nb ? row + (size_t)tq * BPS : unit_in, (uint32_t)nb);
                } else if (BPS == 4) {
#pragma unroll
                    for (int i = 0; i < TPC; ++i) {
                        const uint32_t nb = (srow && tq + i < T) ? 4u : 0u;
                        cp_async_small<4>(d + i * 4, nb ? row + (size_t)(tq + i) * 4 : unit_in, nb);
                    }
                } else {
                    // 2-byte samples have no asynchronous copy: plain loads
                    // and shared stores, read back by this thread only
#pragma unroll
                    for (int i = 0; i < TPC; ++i) {
                        const unsigned short v = (srow && tq + i < T)
                            ? *reinterpret_cast<const unsigned short *>(row + (size_t)(tq + i) * 2)
                            : (unsigned short)0;
                        asm volatile("st.shared.u16 [%0], %1;" ::"r"(d + i * 2), "h"(v) : "memory");
                    }
                }
            }
        }
        return;
    }
    constexpr int BPT = DT == 1 ? 8 : 4;     // bytes per time sample (2 pols, re+im)
    constexpr int NQ = RawBytes<DT>::value / 16;
    constexpr int TPQ = 16 / BPT;            // samples per 16-byte chunk
    const bool srow = s < S;
    const uint8_t *row = unit_in + (srow ? (size_t)s * T * BPT : 0);
    if (vec && srow && t0 + TC_KB_T <= T) {  // whole K-block in range
        const uint8_t *src = row + (size_t)t0 * BPT + g * 16;
#pragma unroll
        for (int q = 0; q < NQ; ++q) cp_async16(dst + q * chunk_stride, src + q * 64, 16u);
    } else if (vec) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int tq = t0 + (g + 4 * q) * TPQ;
            int nb = srow ? (T - tq) * BPT : 0;
            nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
            cp_async16(dst + q * chunk_stride, nb ? row + (size_t)tq * BPT : unit_in, (uint32_t)nb);
        }
    } else {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int i = 0; i < TPQ; ++i) {
                const int tt = t0 + (g + 4 * q) * TPQ + i;
                const uint32_t nb = (srow && tt < T) ? BPT : 0;
                cp_async_small<BPT>(dst + q * chunk_stride + i * BPT,
                                    nb ? row + (size_t)tt * BPT : unit_in, nb);
            }
    }
}

template <int DT>
__device__ __forceinline__ void read_raw(uint32_t src, uint32_t chunk_stride, Raw<DT> &r)
{
#pragma unroll
    for (int q = 0; q < RawBytes<DT>::value / 16; ++q) r.v[q] = lds128(src + q * chunk_stride);
}

// Loads into registers the bytes that issue_raw<2, NPOL> copies for one unit
// (int8 samples; the same chunk order and the same zero fill outside
// [0,S) x [0,T)). Rows of whole 16-byte chunks take 16-byte loads where the
// chunk is in range, other samples plain loads of their own size.
template <int NPOL>
__device__ __forceinline__ void load_raw_i8(const uint8_t *unit_in, int S, int T, bool vec, int s, int t0,
                                            int g, Raw<2> &r)
{
    if constexpr (NPOL == 1) {
        // chunk p: samples t0 + 8g .. +7 of station 2s + p, 2 bytes each
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int st = 2 * s + p;
            const bool srow = st < S;
            const uint8_t *row = unit_in + (srow ? (size_t)st * T * 2 : 0);
            const int tq = t0 + 8 * g;
            if (vec && srow && tq + 8 <= T) {
                r.v[p] = __ldg(reinterpret_cast<const uint4 *>(row + (size_t)tq * 2));
            } else {
                uint32_t w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int ta = tq + 2 * i;
                    const uint32_t lo = (srow && ta < T)
                        ? __ldg(reinterpret_cast<const unsigned short *>(row + (size_t)ta * 2)) : 0u;
                    const uint32_t hi = (srow && ta + 1 < T)
                        ? __ldg(reinterpret_cast<const unsigned short *>(row + (size_t)(ta + 1) * 2)) : 0u;
                    w[i] = lo | (hi << 16);
                }
                r.v[p] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        return;
    }
    const bool srow = s < S;
    const uint8_t *row = unit_in + (srow ? (size_t)s * T * 4 : 0);
    if (vec && srow && t0 + TC_KB_T <= T) {  // whole K-block in range
        const uint4 *src = reinterpret_cast<const uint4 *>(row + (size_t)t0 * 4 + g * 16);
        r.v[0] = __ldg(src);
        r.v[1] = __ldg(src + 4);
    } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int tq = t0 + (g + 4 * q) * 4;   // 4 samples of 4 bytes per chunk
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                w[i] = (srow && tq + i < T) ? __ldg(reinterpret_cast<const unsigned int *>(row + (size_t)(tq + i) * 4))
                                            : 0u;
            r.v[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Two int8 (as the low bytes of the two halves of u) -> two exact f16:
// half bits 0x6400 | (v ^ 0x80) encode 1024 + (v + 128); subtracting 1152
// leaves v exactly (all integers of magnitude <= 2048 are f16 values).
__device__ __forceinline__ uint32_t i8pair_to_h2(uint32_t u)
{
    uint32_t b = (u & 0x00FF00FFu) ^ 0x64806480u;
    __half2 h = *reinterpret_cast<__half2 *>(&b);
    const __half2 off = __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));
    __half2 d = __hsub2(h, off);
    return *reinterpret_cast<uint32_t *>(&d);
}

// Splits 8 samples of one station into 4 chunks of 8 f16 each:
// re[p] = real parts of pol p, im[p] = imaginary parts of pol p.
template <int DT, int NPOL>
__device__ __forceinline__ void split(const Raw<DT> &r, uint4 (&re)[2], uint4 (&im)[2])
{
    uint32_t o_re[2][4], o_im[2][4];
    if (NPOL == 1 && DT == 1) {
        // chunk 2p+h = 4 samples of station 2s+p, word = (re, im) f16
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 &c = r.v[2 * p + (q >> 1)];
                const uint32_t w0 = word_of(c, 2 * (q & 1)), w1 = word_of(c, 2 * (q & 1) + 1);
                o_re[p][q] = __byte_perm(w0, w1, 0x5410);
                o_im[p][q] = __byte_perm(w0, w1, 0x7632);
            }
    } else if (NPOL == 1) {
        // chunk p = 8 samples of station 2s+p, word = bytes (re, im, re, im)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t w = word_of(r.v[p], q);
                o_re[p][q] = i8pair_to_h2(w);
                o_im[p][q] = i8pair_to_h2(w >> 8);
            }
    } else if (DT == 1) {
        // word 2t+p = (re, im) of pol p at the unit's t-th sample (low half = re)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i0 = 2 * (2 * q) + p, i1 = 2 * (2 * q + 1) + p;
                const uint32_t w0 = word_of(r.v[i0 >> 2], i0 & 3);
                const uint32_t w1 = word_of(r.v[i1 >> 2], i1 & 3);
                o_re[p][q] = __byte_perm(w0, w1, 0x5410);
                o_im[p][q] = __byte_perm(w0, w1, 0x7632);
            }
    } else {
        // word t = bytes (p0 re, p0 im, p1 re, p1 im) of the unit's t-th sample
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t w0 = word_of(r.v[(2 * q) >> 2], (2 * q) & 3);
                const uint32_t w1 = word_of(r.v[(2 * q + 1) >> 2], (2 * q + 1) & 3);
                const uint32_t sre = (uint32_t)(2 * p) | ((uint32_t)(4 + 2 * p) << 8);
                const uint32_t sim = (uint32_t)(2 * p + 1) | ((uint32_t)(5 + 2 * p) << 8);
                o_re[p][q] = i8pair_to_h2(__byte_perm(w0, w1, sre));
                o_im[p][q] = i8pair_to_h2(__byte_perm(w0, w1, sim));
            }
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        re[p] = make_uint4(o_re[p][0], o_re[p][1], o_re[p][2], o_re[p][3]);
        im[p] = make_uint4(o_im[p][0], o_im[p][1], o_im[p][2], o_im[p][3]);
    }
}

// Stores the 4 chunks of station-local sl, time group g into a 128-row tile
// (row = 2*sl + pol; chunk g = real parts, chunk 4+g = imaginary parts) in the
// 128-byte swizzled layout. The order of the four stores alternates with the
// station parity so that each quarter-warp hits 8 distinct 16-byte bank groups.
template <int DT, int NPOL>
__device__ __forceinline__ void store_tile(uint32_t tile, int sl, int g, const Raw<DT> &r)
{
    uint4 re[2], im[2];
    split<DT, NPOL>(r, re, im);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = k >> 1;
        const int part = (k ^ sl) & 1;
        const int row = 2 * sl + p;
        const int chunk = g + 4 * part;
        sts128(tile + row * 128 + ((chunk ^ (row & 7)) << 4), part ? im[p] : re[p]);
    }
}

// A work item: channel `unit` of problem `prob`, row block rb, column blocks
// cb0 .. cb0 + ncb - 1 (64 stations each), packed as {prob, unit, rb, cb0 | ncb << 16}.
struct Item {
    int prob, unit, rb, cb0, ncb;
};

__device__ __forceinline__ Item get_item(const TcParams &p, int i)
{
    const int4 v = __ldg(p.items + i);
    return Item{v.x, v.y, v.z, v.w & 0xFFFF, v.w >> 16};
}

// Redo launch: counts this CTA as finished; the last CTA of the grid (every
// CTA has read the redo count by then) clears the marks of the listed items
// and zeroes the count and itself, ready for the next call.
__device__ __forceinline__ void redo_finish(const TcParams &p)
{
    if (!p.redo_done || threadIdx.x != 0) return;
    __threadfence();
    if (atomicAdd(p.redo_done, 1) != (int)gridDim.x - 1) return;
    __threadfence();
    volatile int *count = p.redo_count;
    const int n = *count;
    for (int i = 0; i < n; ++i) p.redo_mark[p.redo_index[i]] = 0;
    *count = 0;
    *reinterpret_cast<volatile int *>(p.redo_done) = 0;
    __threadfence();
}

__device__ __forceinline__ TcProblem get_prob(const TcParams &p, int k)
{
    return p.probs ? p.probs[k] : p.prob0;
}

// MMA rows of column block cb that hold stations (2 per station with two
// pols, 1 per station with one), rounded up to a multiple of 16: a partial
// last block (S not a multiple of the block) is not multiplied in full by
// narrow and wide tiles.
template <int NPOL> __device__ __forceinline__ int narrow_n(int S, int cb)
{
    const int rows = NPOL == 2 ? 2 * min(TC_RS, S - cb * TC_RS) : min(2 * TC_RS, S - cb * 2 * TC_RS);
    return (rows + 15) & ~15;
}

__device__ __forceinline__ int n_chunks(int nkb, int chunk_kb)
{
    return chunk_kb > 0 ? (nkb + chunk_kb - 1) / chunk_kb : 1;
}

// Stores the visibilities of one TMEM column group: row (s1, p1) of this
// thread against column stations s2_0 .. s2_0+7 (both p2), masked to
// s1 <= s2 < S. int8: converts the exact FP32 chunk sums to INT32 and adds
// the earlier chunks' partial sums (fold). PLAIN: the common case, one chunk
// (no fold, streaming stores), with the branches of the others compiled out:
// the epilogue issues these stores while the accumulator is held, one warp
// per scheduler, so every instruction counts.
template <int DT, int NPOL, bool PLAIN>
__device__ __forceinline__ void store_group_impl(const TcProblem &P, long long unit_off, int s1, int s2_0,
                                                 bool fold_arg, bool last_arg, const uint32_t (&vre)[16],
                                                 const uint32_t (&vim)[16])
{
    const bool fold = !PLAIN && fold_arg;
    const bool last = PLAIN || last_arg;
    if constexpr (NPOL == 1) {
        // s1: this row's station; column k = 2j + p2 is station s2b + k with
        // s2b = 2 s2_0; one complex per baseline. Twice the stores of the
        // two-pol case, so their indices come from the group's first one,
        // tri(s2b) + s1 with tri(s) = s(s+1)/2, as + k*s2b + k(k+1)/2: one
        // independent multiply-add per store.
        const int s2b = 2 * s2_0;
        const long long base = unit_off + (long long)s2b * (s2b + 1) / 2 + s1;
        const int lo = s1 - s2b, hi = P.S - s2b;   // valid columns: lo <= k < hi
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < lo || k >= hi) continue;
            const long long e = base + (long long)(k * s2b + k * (k + 1) / 2);
            if (DT == 1) {
                float2 *dst = static_cast<float2 *>(P.out) + e;
                __stcs(dst, make_float2(__uint_as_float(vre[k]), __uint_as_float(vim[k])));
            } else {
                int2 *dst = static_cast<int2 *>(P.out) + e;
                int2 v = make_int2(__float2int_rn(__uint_as_float(vre[k])),
                                   __float2int_rn(__uint_as_float(vim[k])));
                if (fold) {
                    const int2 o = __ldcg(dst);
                    v.x += o.x;
                    v.y += o.y;
                }
                if (last)
                    __stcs(dst, v);
                else
                    __stcg(dst, v);
            }
        }
        return;
    }
    // Two pols: baseline tri(s2_0 + j) + s1 = tri(s2_0) + s1 + j*s2_0 +
    // j(j+1)/2, 4 complex values each; one multiply-add per store from the
    // group's first index.
    const long long base = unit_off + ((long long)s2_0 * (s2_0 + 1) / 2 + s1) * 4;
    const int lo = s1 - s2_0, hi = P.S - s2_0;   // valid columns: lo <= j < hi
    if (DT == 1) {
        float2 *out = static_cast<float2 *>(P.out) + base;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < lo || j >= hi) continue;
            const float4 v = make_float4(__uint_as_float(vre[2 * j]), __uint_as_float(vim[2 * j]),
                                         __uint_as_float(vre[2 * j + 1]), __uint_as_float(vim[2 * j + 1]));
            st_global_cs(out + (j * s2_0 + j * (j + 1) / 2) * 4, v);
        }
    } else if (PLAIN) {
        int2 *out = static_cast<int2 *>(P.out) + base;
        const bool all = lo <= 0 && hi >= 8;   // the whole group lies in the triangle
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!all && (j < lo || j >= hi)) continue;
            const int4 v = make_int4(__float2int_rn(__uint_as_float(vre[2 * j])),
                                     __float2int_rn(__uint_as_float(vim[2 * j])),
                                     __float2int_rn(__uint_as_float(vre[2 * j + 1])),
                                     __float2int_rn(__uint_as_float(vim[2 * j + 1])));
            st_global_cs(out + (j * s2_0 + j * (j + 1) / 2) * 4, v);
        }
    } else {
        int2 *out = static_cast<int2 *>(P.out) + unit_off;
        int4 old[8];
        if (fold) {
            // read every earlier partial first so the loads overlap
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int s2 = s2_0 + j;
                old[j] = (s1 <= s2 && s2 < P.S) ? ld_global_cg(out + ((long long)s2 * (s2 + 1) / 2 + s1) * 4)
                                                : make_int4(0, 0, 0, 0);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) old[j] = make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int s2 = s2_0 + j;
            if (s1 <= s2 && s2 < P.S) {
                const int4 v = make_int4(__float2int_rn(__uint_as_float(vre[2 * j])) + old[j].x,
                                         __float2int_rn(__uint_as_float(vim[2 * j])) + old[j].y,
                                         __float2int_rn(__uint_as_float(vre[2 * j + 1])) + old[j].z,
                                         __float2int_rn(__uint_as_float(vim[2 * j + 1])) + old[j].w);
                int2 *dst = out + ((long long)s2 * (s2 + 1) / 2 + s1) * 4;
                if (last)
                    st_global_cs(dst, v);
                else
                    st_global_cg(dst, v);
            }
        }
    }
}

template <int DT, int NPOL>
__device__ __forceinline__ void store_group(const TcProblem &P, long long unit_off, int s1, int s2_0,
                                            bool fold, bool last, const uint32_t (&vre)[16],
                                            const uint32_t (&vim)[16])
{
    if (DT == 1 || (!fold && last))
        store_group_impl<DT, NPOL, true>(P, unit_off, s1, s2_0, false, true, vre, vim);
    else
        store_group_impl<DT, NPOL, false>(P, unit_off, s1, s2_0, fold, last, vre, vim);
}

// NPOL = 2: rows are (station, pol). NPOL = 1: rows are stations; stations
// 2m and 2m+1 take the places of the two pols of "pseudo-station" m, so the
// tiles, the schedule (over pseudo-stations) and the MMAs are those of the
// two-pol case and only the sample copies and the output mapping differ.
template <int DT, int V, int NPOL, int LY = 0> __device__ __forceinline__ void tc_correlate_body(const TcParams &p)
{
    using C = Cfg<DT, V>;
    using L = Lay<DT, V, NPOL, LY>;
    constexpr bool PAIR = V == TC_PAIR;
    constexpr bool N256 = V != TC_NARROW;          // tiles of two column blocks
    constexpr int OPS = L::OPS;
    constexpr int RAW = L::RAW;
    constexpr int STG = L::STG;
    constexpr int NBUF = C::NBUF;
    constexpr uint32_t STAGE = stage_bytes<DT, V>();
    constexpr uint32_t IMOFF = N256 ? 256 : 128;   // TMEM column of Im relative to Re
    constexpr uint32_t BUFCOLS = N256 ? 0 : 256;   // TMEM columns between buffers

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t tiles_u32 = smem_u32(smem);
    const uint32_t raw_base = tiles_u32 + OPS * STAGE;
    Bars *bars = reinterpret_cast<Bars *>(smem + smem_bytes<DT, V, NPOL, LY>());
    volatile int *abort_flag = &bars->abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    // The redo launch reads the count that the launch before it wrote: wait
    // for that launch's end. A launch lets its own dependent be scheduled
    // once it has waited for its own predecessor (a main launch: after its
    // set-up, below), so that a dependent which does not wait (a tail list)
    // never starts before what preceded the call on the stream has ended.
    if (p.n_items_dev) griddep_wait();
    if (!p.dep_wait) griddep_launch_dependents();
    const int n_items = p.n_items_dev ? *p.n_items_dev : p.n_items;
    // A pair (cluster of 2 CTAs) shares each work item; rank 0 issues the MMAs.
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    const int item0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int item_step = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    // No work (e.g. an empty redo list): leave before any barrier, TMEM or
    // cluster step. Both CTAs of a pair see the same item0 and leave together.
    if (item0 >= n_items) {
        redo_finish(p);
        return;
    }

    // In a pair, the even CTA's full barriers also count one arrival of the
    // odd CTA's relay thread (see the relay below), and its acc_empty
    // barriers one arrival of each of the odd CTA's four epilogue warps.
    const uint32_t relay = PAIR && leader ? 1u : 0u;
    if (tid == 0) {
        for (int s = 0; s < OPS; ++s) {
            mbar_init(&bars->full[s], N_PRODUCERS + relay);
            mbar_init(&bars->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars->acc_full[b], 1);
            mbar_init(&bars->acc_empty[b], N_EPILOGUE + 4 * relay);
        }
        mbar_init(&bars->fin, 1);
        bars->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == WARP_MMA) {
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
    if constexpr (PAIR) cluster_sync(); // both CTAs' barriers are initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem_base = bars->tmem_base;
    // A main launch scheduled early (programmatic dependent): the set-up
    // above overlapped the previous kernel's end; its samples and outputs
    // may be that kernel's, so wait for it here.
    if (p.dep_wait) {
        griddep_wait();
        griddep_launch_dependents();
    }

    if (warp < N_PROD_WARPS) {
        // ------------------------------------------------------ producers
        // Units per K-block: (operand block, station-local sl, group g of 8
        // samples); thread pt owns unit pt of A and unit pt of each B block.
        // Operand block slots per stage: 0 = A, 1.. = the B blocks that are
        // not A itself (a diagonal tile reuses A as its first B block).
        const int pt = tid;
        const int sl = pt >> 2;
        const int g = pt & 3;
        constexpr uint32_t CHUNK = 16 * N_PRODUCERS;                  // stride between chunks
        constexpr uint32_t SLOT = (RawBytes<DT>::value / 16) * CHUNK; // one unit slot
        constexpr int NSLOT = 1 + C::MAXB;
        int stage = 0;
        uint32_t phase = 0;
        for (int it = item0; it < n_items; it += item_step) {
            const Item item = get_item(p, it);
            const TcProblem P = get_prob(p, item.prob);
            const bool diag = item.cb0 == item.rb;
            // B blocks to stage and the first of them; a pair CTA stages
            // column block cb0 + rank (none on the diagonal: it is its A).
            const int nB = PAIR ? (diag ? 0 : 1) : item.ncb - (diag ? 1 : 0);
            const int b_first = PAIR ? item.cb0 + (int)rank : (diag ? item.cb0 + 1 : item.cb0);
            const uint8_t *unit_in = static_cast<const uint8_t *>(P.in) +
                                     (size_t)item.unit * (size_t)P.in_unit_bytes;
            const int nkb = (P.T + TC_KB_T - 1) / TC_KB_T;
            const bool vec = P.vec != 0;
            const bool check = DT == 2 && p.check_power != 0;
            int power[NSLOT];   // this thread's share of sum_t |x|^2 per staged station
#pragma unroll
            for (int j = 0; j < NSLOT; ++j) power[j] = 0;
            int st_of[NSLOT];
            st_of[0] = (item.rb + (int)rank) * TC_RS + sl;
#pragma unroll
            for (int j = 1; j < NSLOT; ++j) st_of[j] = (b_first + j - 1) * TC_RS + sl;
            auto slot_addr = [&](int k, int j) {
                return raw_base + (uint32_t)((k % (RAW > 0 ? RAW : 1)) * NSLOT + j) * SLOT + (uint32_t)pt * 16u;
            };
            auto issue_kb = [&](int k) {
                if (k < nkb) {
#pragma unroll
                    for (int j = 0; j < NSLOT; ++j)
                        if (j <= nB)
                            issue_raw<DT, NPOL>(unit_in, P.S, P.T, vec, st_of[j], k * TC_KB_T, g,
                                          slot_addr(k, j), CHUNK);
                }
                cp_async_commit(); // one group per K-block (empty past the end)
            };
            bool ok = true;
            // Converts K-block data r into operand stage `stage`, adds its
            // power and publishes the stage to the MMA thread.
            auto produce = [&](const Raw<DT> (&r)[NSLOT]) {
                const uint32_t st = tiles_u32 + stage * STAGE;
#pragma unroll
                for (int j = 0; j < NSLOT; ++j)
                    if (j <= nB) store_tile<DT, NPOL>(st + j * TILE_BYTES, sl, g, r[j]);
                if (check) {
#pragma unroll
                    for (int j = 0; j < NSLOT; ++j)
                        if (j <= nB)
#pragma unroll
                            for (int q = 0; q < (int)(sizeof(Raw<DT>) / 16); ++q) {
                                // 4 int8 (re, im of both pols) per word: sum of squares
                                power[j] = __dp4a((int)r[j].v[q].x, (int)r[j].v[q].x, power[j]);
                                power[j] = __dp4a((int)r[j].v[q].y, (int)r[j].v[q].y, power[j]);
                                power[j] = __dp4a((int)r[j].v[q].z, (int)r[j].v[q].z, power[j]);
                                power[j] = __dp4a((int)r[j].v[q].w, (int)r[j].v[q].w, power[j]);
                            }
                }
            };
            auto publish = [&]() {
                fence_proxy_async_smem();
                mbar_arrive(&bars->full[stage]);
                if (++stage == OPS) {
                    stage = 0;
                    phase ^= 1;
                }
            };
            if constexpr (RAW == 0) {
                // int8: a ring of PF K-blocks in registers. The loads of
                // K-block k + PF are issued once K-block k is converted, so
                // each has PF K-block periods to arrive; a stage barrier
                // arrival does not wait for them.
                constexpr int PF = CORR_TC_PF;
                Raw<DT> ring[PF][NSLOT];
                auto load_kb = [&](int k, Raw<DT> (&dst)[NSLOT]) {
                    if (k < nkb) {
#pragma unroll
                        for (int j = 0; j < NSLOT; ++j)
                            if (j <= nB) load_raw_i8<NPOL>(unit_in, P.S, P.T, vec, st_of[j], k * TC_KB_T, g, dst[j]);
                    }
                };
#pragma unroll
                for (int d = 0; d < PF; ++d) load_kb(d, ring[d]);
#pragma unroll 1
                for (int k0 = 0; k0 < nkb && ok; k0 += PF) {
#pragma unroll
                    for (int d = 0; d < PF; ++d) {
                        if (k0 + d < nkb && ok) {
                            if (!mbar_wait_bounded(&bars->empty[stage], phase ^ 1, abort_flag, p.err,
                                                   p.wait_ns)) {
                                ok = false;
                            } else {
                                produce(ring[d]);
                                load_kb(k0 + d + PF, ring[d]);
                                publish();
                            }
                        }
                    }
                }
                if (!ok) break;
            } else {
#pragma unroll 1
                for (int q = 0; q < RAW - 1; ++q) issue_kb(q);
#pragma unroll 1
                for (int k = 0; k < nkb; ++k) {
                    issue_kb(k + RAW - 1);
                    cp_async_wait<RAW - 1>(); // this thread's copies of K-block k have landed
                    Raw<DT> r[NSLOT];
#pragma unroll
                    for (int j = 0; j < NSLOT; ++j)
                        if (j <= nB) read_raw<DT>(slot_addr(k, j), CHUNK, r[j]);
                    if (!mbar_wait_bounded(&bars->empty[stage], phase ^ 1, abort_flag, p.err,
                                           p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    produce(r);
                    publish();
                }
                cp_async_wait<0>();
                if (!ok) break;
            }
            if (check) {
                // station power = sum over the 4 threads of the station (both
                // pols together, which bounds each pol); any station above
                // 2^24 makes the unchunked FP32 sums of this tile unproven.
                bool unsafe = false;
#pragma unroll
                for (int j = 0; j < NSLOT; ++j) {
                    int v = min(power[j], 1 << 25); // clamp: keeps the test, avoids overflow
                    v += __shfl_xor_sync(0xffffffffu, v, 1);
                    v += __shfl_xor_sync(0xffffffffu, v, 2);
                    unsafe |= j <= nB && v > (1 << 24);
                }
                if (__any_sync(0xffffffffu, unsafe) && lane == 0) {
                    if (atomicExch(p.redo_mark + it, 1) == 0) {
                        const int slot = atomicAdd(p.redo_count, 1);
                        p.redo_items[slot] = __ldg(p.items + it);
                        p.redo_index[slot] = it;
                    }
                }
            }
        }
    } else if (warp < WARP_MMA) {
        // ------------------------------------------------------- epilogue
        const int eq = warp & 3;            // TMEM lane quarter of this warp
        const int row = eq * 32 + lane;     // A row = 2*station + pol
        const int sl = row >> 1;
        const int p1 = row & 1;
        // this warp's ring of STG staged groups: group slot k at k * 4 KB,
        // column station j of it at j * 512 B, one thread's row at lane * 16 B
        const uint32_t stg_base = raw_base + RAW * raw_stage_bytes<DT, V>() + eq * STG * STG_GROUP_BYTES;
        uint32_t acc_it = 0;
        bool ok = true;
        for (int it = item0; it < n_items && ok; it += item_step) {
            const Item item = get_item(p, it);
            const TcProblem P = get_prob(p, item.prob);
            const int nkb = (P.T + TC_KB_T - 1) / TC_KB_T;
            const int nch = n_chunks(nkb, p.chunk_kb);
            // NPOL = 1: the row's station; NPOL = 2: its station (pol p1)
            const int s1 = NPOL == 1 ? (item.rb + (int)rank) * 2 * TC_RS + row
                                     : (item.rb + (int)rank) * TC_RS + sl;
            // groups of 8 column (pseudo-)stations; narrow and wide tiles
            // read the columns their MMAs wrote (narrow_n)
            const int ngroups = PAIR ? 8 * item.ncb
                                     : ((item.ncb - 1) * 128 + narrow_n<NPOL>(P.S, item.cb0 + item.ncb - 1)) / 16;
            const long long unit_off = (long long)item.unit * P.out_unit_elems + (NPOL == 1 ? 0 : p1 * 2);
            for (int c = 0; c < nch; ++c, ++acc_it) {
                const uint32_t buf = acc_it % NBUF, ap = (acc_it / NBUF) & 1;
                // the warp takes the wait's outcome together: its TMEM loads
                // and its release below are warp-wide
                const bool got = mbar_wait_bounded(&bars->acc_full[buf], ap, abort_flag, p.err, p.wait_ns);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + buf * BUFCOLS + ((uint32_t)(eq * 32) << 16);
                // Every column of this chunk has been read: the next chunk's
                // MMAs may overwrite the accumulator. In a pair the odd CTA's
                // warps arrive on the even CTA's barrier, where the MMAs are
                // issued, one cluster-scope arrival per warp.
                auto release_acc = [&]() {
                    tc_fence_before();
                    if (PAIR && !leader) {
                        __syncwarp();
                        if (lane == 0) mbar_arrive_cluster(mapa_shared(smem_u32(&bars->acc_empty[buf]), 0));
                    } else {
                        mbar_arrive(&bars->acc_empty[buf]);
                    }
                };
                const bool last = c == nch - 1;
                // Column groups of 16 TMEM columns (8 column stations x 2 pols),
                // Re and Im. The first ndirect groups are stored to global
                // memory from registers; the load of the next group overlaps
                // the stores of the current one (two register sets). The last
                // nst groups (int8 pair tiles, one chunk) are
                // staged in this warp's shared-memory ring, so that the
                // accumulator is released once they are there; their global
                // writes then overlap the next tile's MMAs.
                const int nst = (STG > 0 && nch == 1) ? min(STG, ngroups) : 0;
                const int ndirect = ngroups - nst;
                uint32_t ra[16], ia[16], rb2[16], ib2[16];
                bool released = false;
                if (ndirect > 0) {
                    tmem_ld_32x32b_x16(taddr, ra);
                    tmem_ld_32x32b_x16(taddr + IMOFF, ia);
                    tmem_wait_ld();
                }
#pragma unroll 1
                for (int cc = 0; cc < ndirect; cc += 2) {
                    const bool has1 = cc + 1 < ndirect;
                    if (has1) {
                        tmem_ld_32x32b_x16(taddr + (cc + 1) * 16, rb2);
                        tmem_ld_32x32b_x16(taddr + IMOFF + (cc + 1) * 16, ib2);
                    }
                    store_group<DT, NPOL>(P, unit_off, s1, item.cb0 * TC_RS + cc * 8, c > 0, last, ra, ia);
                    tmem_wait_ld();
                    if (nst == 0 && cc + 2 >= ndirect) {  // every column of this chunk has been read
                        release_acc();
                        released = true;
                    }
                    if (has1) {
                        if (cc + 2 < ndirect) {
                            tmem_ld_32x32b_x16(taddr + (cc + 2) * 16, ra);
                            tmem_ld_32x32b_x16(taddr + IMOFF + (cc + 2) * 16, ia);
                        }
                        store_group<DT, NPOL>(P, unit_off, s1, item.cb0 * TC_RS + (cc + 1) * 8, c > 0, last,
                                              rb2, ib2);
                        if (cc + 2 < ndirect) tmem_wait_ld();
                    }
                }
                if constexpr (STG > 0) {
                    if (nst > 0) {
                        // Staged groups: each thread copies its row's raw
                        // accumulator values to its own 16-byte slots of this
                        // warp's ring (conflict-free: a warp writes 512
                        // contiguous bytes per column station), the
                        // accumulator is released, and the same thread then
                        // converts and stores them to global memory while
                        // the MMAs of the next tile run. Each thread reads
                        // back only what it wrote, so no barrier or fence is
                        // needed, and a slot is rewritten only by its own
                        // thread after it has been read back.
                        auto stage = [&](int k, const uint32_t(&vr)[16], const uint32_t(&vi)[16]) {
                            const uint32_t slot = stg_base + (uint32_t)k * STG_GROUP_BYTES + lane * 16u;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                sts128(slot + j * 512, make_uint4(vr[2 * j], vi[2 * j], vr[2 * j + 1], vi[2 * j + 1]));
                        };
                        auto release = [&]() {  // every column of this chunk has been read
                            release_acc();
                            released = true;
                        };
                        tmem_ld_32x32b_x16(taddr + ndirect * 16, ra);
                        tmem_ld_32x32b_x16(taddr + IMOFF + ndirect * 16, ia);
                        tmem_wait_ld();
                        if (nst == 1) release();
#pragma unroll 1
                        for (int k = 0; k < nst; k += 2) {
                            const bool has1 = k + 1 < nst;
                            const bool has2 = k + 2 < nst;
                            if (has1) {
                                tmem_ld_32x32b_x16(taddr + (ndirect + k + 1) * 16, rb2);
                                tmem_ld_32x32b_x16(taddr + IMOFF + (ndirect + k + 1) * 16, ib2);
                            }
                            stage(k, ra, ia);
                            if (has1) {
                                tmem_wait_ld();
                                if (k + 1 == nst - 1) release();
                                if (has2) {
                                    tmem_ld_32x32b_x16(taddr + (ndirect + k + 2) * 16, ra);
                                    tmem_ld_32x32b_x16(taddr + IMOFF + (ndirect + k + 2) * 16, ia);
                                }
                                stage(k + 1, rb2, ib2);
                                if (has2) {
                                    tmem_wait_ld();
                                    if (k + 2 == nst - 1) release();
                                }
                            }
                        }
                        // drain: the staged groups to global memory
#pragma unroll 1
                        for (int k = 0; k < nst; ++k) {
                            const uint32_t slot = stg_base + (uint32_t)k * STG_GROUP_BYTES + lane * 16u;
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const uint4 v = lds128(slot + j * 512);
                                ra[2 * j] = v.x;
                                ia[2 * j] = v.y;
                                ra[2 * j + 1] = v.z;
                                ia[2 * j + 1] = v.w;
                            }
                            store_group<DT, NPOL>(P, unit_off, s1, item.cb0 * TC_RS + (ndirect + k) * 8, false,
                                                  true, ra, ia);
                        }
                    }
                }
                if (!released) release_acc();
            }
        }
    } else if (leader) {
        // ------------------------------------------------------------ MMA
        // M = 256 for a pair (128 rows from each CTA), else 128.
        constexpr int M = PAIR ? 256 : 128;
        constexpr uint32_t ID128 = idesc_f16_f32(M, 128, false);
        constexpr uint32_t ID128N = idesc_f16_f32(M, 128, true);
        constexpr uint32_t ID256 = idesc_f16_f32(M, 256, false);
        constexpr uint32_t ID256N = idesc_f16_f32(M, 256, true);
        int stage = 0;
        uint32_t phase = 0;
        uint32_t acc_it = 0;
        bool ok = true;
        auto mma = [&](uint32_t d, uint32_t a, uint32_t b, uint32_t id, uint32_t acc) {
            if constexpr (PAIR)
                tc_mma_f16_pair(d, smem_desc_sw128(a), smem_desc_sw128(b), id, acc);
            else
                tc_mma_f16(d, smem_desc_sw128(a), smem_desc_sw128(b), id, acc);
        };
        auto commit = [&](uint64_t *bar) {
            if constexpr (PAIR)
                tc_commit_pair(bar, 3);   // the barrier at this offset in both CTAs
            else
                tc_commit(bar);
        };
        for (int it = item0; it < n_items && ok; it += item_step) {
            const Item item = get_item(p, it);
            const TcProblem P = get_prob(p, item.prob);
            const bool diag = item.cb0 == item.rb;
            const bool n256 = N256 && item.ncb == 2;
            uint32_t idesc = n256 ? ID256 : ID128;
            uint32_t idesc_neg = n256 ? ID256N : ID128N;
            if constexpr (!PAIR) {
                // full column blocks, then the last one's rows with stations:
                // 16 .. 256, a multiple of 16
                const int n = (item.ncb - 1) * 128 + narrow_n<NPOL>(P.S, item.cb0 + item.ncb - 1);
                idesc = idesc_f16_f32(M, n, false);
                idesc_neg = idesc_f16_f32(M, n, true);
            }
            const int nkb = (P.T + TC_KB_T - 1) / TC_KB_T;
            const int nch = n_chunks(nkb, p.chunk_kb);
            const int ckb = p.chunk_kb > 0 ? p.chunk_kb : nkb;
            for (int c = 0; c < nch && ok; ++c, ++acc_it) {
                const uint32_t buf = acc_it % NBUF, ap = (acc_it / NBUF) & 1;
                if (!mbar_wait_bounded<PAIR>(&bars->acc_empty[buf], ap ^ 1, abort_flag, p.err,
                                             p.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_re = tmem_base + buf * BUFCOLS;
                const uint32_t d_im = d_re + IMOFF;
                const int kb_lo = c * ckb;
                const int kb_hi = min(nkb, kb_lo + ckb);
                for (int kb = kb_lo; kb < kb_hi; ++kb) {
                    if (!mbar_wait_bounded<PAIR>(&bars->full[stage], phase, abort_flag, p.err,
                                                 p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (lane == 0) {
                        const uint32_t a = tiles_u32 + stage * STAGE;
                        const uint32_t b = diag ? a : a + TILE_BYTES;
                        const uint32_t first = kb == kb_lo ? 1u : 0u;
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)
                            mma(d_re, a + 32 * ks, b + 32 * ks, idesc, (first && ks == 0) ? 0u : 1u);
                        mma(d_im, a + 64, b + 0, idesc, first ? 0u : 1u);
                        mma(d_im, a + 96, b + 32, idesc, 1u);
                        mma(d_im, a + 0, b + 64, idesc_neg, 1u);
                        mma(d_im, a + 32, b + 96, idesc_neg, 1u);
                        commit(&bars->empty[stage]);
                    }
                    __syncwarp();
                    if (++stage == OPS) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                if (lane == 0) commit(&bars->acc_full[buf]);
                __syncwarp();
            }
        }
        // Wait for every MMA this thread issued before TMEM is freed (and, in
        // a pair, before the odd CTA's shared memory can go away). This wait
        // keeps a fixed 2 s bound whatever p.wait_ns is, so that an aborted
        // kernel never frees TMEM under a running MMA.
        if (lane == 0) commit(&bars->fin);
        __syncwarp();
        int dummy_abort = 0;
        mbar_wait_bounded(&bars->fin, 0, &dummy_abort, p.err, 2000000000ull);
    } else if constexpr (PAIR) {
        // ------------------------------------------ relay (odd CTA of a pair)
        // This CTA's producers arrive on its own "full" barriers (CTA scope,
        // as in a single CTA: a cluster-scope release in every producer
        // thread would also wait for its asynchronous copies in flight). One
        // thread forwards each completed phase, in the MMA thread's order of
        // K-blocks, to the even CTA with one cluster-scope arrival. It never
        // waits for the accumulator (the epilogue warps release it
        // themselves), so the next tile's first K-blocks reach the even CTA
        // while this tile's accumulator is still being read.
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int it = item0; it < n_items && ok; it += item_step) {
                const Item item = get_item(p, it);
                const TcProblem P = get_prob(p, item.prob);
                const int nkb = (P.T + TC_KB_T - 1) / TC_KB_T;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait_bounded(&bars->full[stage], phase, abort_flag, p.err, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(smem_u32(&bars->full[stage]), 0));
                    if (++stage == OPS) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    // A pair leaves together: the even CTA has seen its MMAs complete, and the
    // odd CTA's remote arrivals have all been made.
    if constexpr (PAIR) cluster_sync();
    if (warp == WARP_MMA) {
        tc_fence_after();
        if constexpr (PAIR)
            tmem_dealloc_pair(tmem_base, TMEM_COLS);
        else
            tmem_dealloc(tmem_base, TMEM_COLS);
    }
    redo_finish(p);
}

template <int DT, int V, int NPOL>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_correlate_kernel(const __grid_constant__ TcParams p)
{
    tc_correlate_body<DT, V, NPOL>(p);
}

template <int DT, int NPOL, int LY>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
    tc_pair_kernel(const __grid_constant__ TcParams p)
{
    tc_correlate_body<DT, TC_PAIR, NPOL, LY>(p);
}

template <int DT, int V, int NPOL, int LY> const void *kernel_ptr()
{
    if constexpr (V == TC_PAIR)
        return reinterpret_cast<const void *>(&tc_pair_kernel<DT, NPOL, LY>);
    else
        return reinterpret_cast<const void *>(&tc_correlate_kernel<DT, V, NPOL>);
}

template <int DT, int V, int NPOL, int LY> size_t smem_total()
{
    return (size_t)smem_bytes<DT, V, NPOL, LY>() + sizeof(Bars) + 1024;
}

template <int DT, int V, int NPOL, int LY>
cudaError_t launch_one(const TcParams &p, int grid, cudaStream_t s, bool pdl)
{
    const size_t smem = smem_total<DT, V, NPOL, LY>();
    cudaError_t e = cudaFuncSetAttribute(kernel_ptr<DT, V, NPOL, LY>(),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid, 1, 1);
        cfg.blockDim = dim3(TC_THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if constexpr (V == TC_PAIR)
            return cudaLaunchKernelEx(&cfg, tc_pair_kernel<DT, NPOL, LY>, p);
        else
            return cudaLaunchKernelEx(&cfg, tc_correlate_kernel<DT, V, NPOL>, p);
    }
    if constexpr (V == TC_PAIR)
        tc_pair_kernel<DT, NPOL, LY><<<grid, TC_THREADS, smem, s>>>(p);
    else
        tc_correlate_kernel<DT, V, NPOL><<<grid, TC_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

template <int DT, int NPOL>
cudaError_t launch_dt(int variant, const TcParams &p, int grid, cudaStream_t s, bool pdl, int layout)
{
    if (variant == TC_PAIR) {
        if constexpr (DT == 2 && NPOL == 2)
            if (layout == 1) return launch_one<DT, TC_PAIR, NPOL, 1>(p, grid, s, pdl);
        return launch_one<DT, TC_PAIR, NPOL, 0>(p, grid, s, pdl);
    }
    if (variant == TC_WIDE) return launch_one<DT, TC_WIDE, NPOL, 0>(p, grid, s, pdl);
    return launch_one<DT, TC_NARROW, NPOL, 0>(p, grid, s, pdl);
}

template <int DT> cudaError_t pair_clusters_dt(int *n)
{
    const size_t smem = smem_total<DT, TC_PAIR, 2, 0>();
    cudaError_t e = cudaFuncSetAttribute(tc_pair_kernel<DT, 2, 0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    return cudaOccupancyMaxActiveClusters(n, tc_pair_kernel<DT, 2, 0>, &cfg);
}

} // namespace

cudaError_t tc_launch(int dtype, int variant, int npol, const TcParams &p, int grid, cudaStream_t s, bool pdl,
                      int layout)
{
    if (variant == TC_PAIR && (grid < 2 || grid % 2 != 0)) return cudaErrorInvalidValue;
    if (npol == 1)
        return dtype == 1 ? launch_dt<1, 1>(variant, p, grid, s, pdl, layout)
                          : launch_dt<2, 1>(variant, p, grid, s, pdl, layout);
    return dtype == 1 ? launch_dt<1, 2>(variant, p, grid, s, pdl, layout)
                      : launch_dt<2, 2>(variant, p, grid, s, pdl, layout);
}

cudaError_t tc_pair_max_clusters(int dtype, int *n)
{
    *n = 0;
    return dtype == 1 ? pair_clusters_dt<1>(n) : pair_clusters_dt<2>(n);
}

} // namespace corr
