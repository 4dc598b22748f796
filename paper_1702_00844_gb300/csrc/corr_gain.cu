// Gain-calibration loss and its hand-written adjoint (FP32).
//
// The correlator output feeds calibration (Section 2 keeps autocorrelations
// for it). With per-station, per-polarisation complex gains g and samples x,
// y = g x, the visibilities of y are V_ab = g_a conj(g_b) R_ab with R the
// correlation of x. For a model M the loss is L = sum |V_ab - M_ab|^2 over
// baselines s1 <= s2 and all polarisation pairs. Gradients follow PyTorch's
// convention for a real function of complex inputs, grad = 2 dL/d conj(z):
//   dL/d conj(g_c)   = sum_{(c,b)} E_cb g_b conj(R_cb) + sum_{(a,c)} conj(E_ac) g_a R_ac
//   dL/d conj(x_c(t)) = conj(g_c) sum_b W_cb g_b x_b(t),
//   W_cb = [s_c <= s_b] E_cb + [s_b <= s_c] conj(E_bc),   E = V - M.
// The input gradient is a complex GEMM per channel: W' = 2 conj(g) W g is
// formed once, then grad_x[c][t] = sum_b W'[c][b] x[b][t].
#include "corr_internal.h"
#include "ptx.cuh"

namespace corr {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ long long bl(int s1, int s2) { return (long long)s2 * (s2 + 1) / 2 + s1; }

// E_ab for a = (s1,p1), b = (s2,p2), s1 <= s2.
__device__ __forceinline__ float2 residual(const float2 *R, const float2 *g, const float2 *M,
                                           int s1, int p1, int s2, int p2)
{
    const long long k = bl(s1, s2) * 4 + p1 * 2 + p2;
    const float2 w = cmul(g[s1 * 2 + p1], cconj(g[s2 * 2 + p2]));
    const float2 v = cmul(w, R[k]);
    return make_float2(v.x - M[k].x, v.y - M[k].y);
}

__global__ void gain_loss_kernel(const float2 *R, const float2 *g, const float2 *M, float2 *V,
                                 float *partial, int S)
{
    const int unit = blockIdx.x;
    const long long B4 = (long long)S * (S + 1) / 2 * 4;
    const float2 *Ru = R + unit * B4;
    const float2 *Mu = M + unit * B4;
    const float2 *gu = g + (long long)unit * S * 2;
    float sum = 0.f;
    for (long long k = threadIdx.x; k < B4; k += blockDim.x) {
        const long long b = k >> 2;
        const int p1 = (k >> 1) & 1, p2 = k & 1;
        // invert b = s2(s2+1)/2 + s1 (single-precision estimate, then
        // corrected exactly in integers)
        int s2 = (int)((sqrtf(8.f * (float)b + 1.f) - 1.f) * 0.5f);
        while ((long long)s2 * (s2 + 1) / 2 > b) --s2;
        while ((long long)(s2 + 1) * (s2 + 2) / 2 <= b) ++s2;
        const int s1 = (int)(b - (long long)s2 * (s2 + 1) / 2);
        const float2 w = cmul(gu[s1 * 2 + p1], cconj(gu[s2 * 2 + p2]));
        const float2 v = cmul(w, Ru[k]);
        if (V) V[unit * B4 + k] = v;
        const float er = v.x - Mu[k].x, ei = v.y - Mu[k].y;
        sum = fmaf(er, er, fmaf(ei, ei, sum));
    }
    __shared__ float red[256];
    red[threadIdx.x] = sum;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[unit] = red[0];
}

__global__ void sum_partials_kernel(const float *partial, int n, float *loss)
{
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0];
}

// Writes W'cb = v into the tensor-core input gradient's A' tiles: rows 2c
// (re) and 2c+1 (im) of M', columns 2b (x re) and 2b+1 (x im) of K', in the
// 128-byte swizzled K-major layout (row r at r x 128 B, 16-byte chunk q at
// (q ^ (r % 8)) x 16 B). With CORR_IG_A_FP32 the values are stored as they
// are (the kernel splits them in shared memory); otherwise as hi = the value
// rounded to tf32 and lo = (value - hi) rounded to tf32, in two tiles.
__device__ __forceinline__ void store_w_tiles(float *at, int unit, int S, int c, int b, float2 v)
{
    constexpr int PARTS = CORR_IG_A_FP32 ? 1 : 2;
    constexpr int KV = CORR_IG_KV;   // floats per tile row
    const int mt = (2 * c) / 128, r = (2 * c) % 128, kb = (2 * b) / KV, kk = (2 * b) % KV;
    const size_t tile = (((size_t)unit * ig_m_alloc(S) + mt) * ig_k_blocks(S) + kb) * PARTS;
    const int q = kk >> 2;   // 16-byte chunk of the row
    const float vals[2][2] = {{v.x, -v.y}, {v.y, v.x}};   // rows r (re) and r + 1 (im)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int rr = r + h;
        // chunk q of row rr at 16-byte position q ^ (rr mod 8) (128-byte
        // swizzle) or q ^ ((rr / 2) mod 4) (64-byte swizzle)
        const int pos = KV == 32 ? (q ^ (rr & 7)) : (q ^ ((rr >> 1) & 3));
        const size_t off = (size_t)rr * KV + (size_t)(pos << 2) + (kk & 3);
        const float a0 = vals[h][0], a1 = vals[h][1];
        constexpr size_t TF = 128 * KV;   // floats per tile
        if (PARTS == 1) {
            *reinterpret_cast<float2 *>(at + tile * TF + off) = make_float2(a0, a1);
        } else {
            const float h0 = tf32_round(a0), h1 = tf32_round(a1);
            *reinterpret_cast<float2 *>(at + tile * TF + off) = make_float2(h0, h1);
            *reinterpret_cast<float2 *>(at + (tile + 1) * TF + off) =
                make_float2(tf32_round(a0 - h0), tf32_round(a1 - h1));
        }
    }
}

// One CTA per (unit, row c = (s, p)), its threads over b: the residuals of
// row c give both sums of dL/d conj(g_c) (reduced over b in a fixed order)
// and, when W is given, the row W'[unit][c][:] = 2 scale conj(g_c) W_cb g_b of
// the input gradient (TILES: written as the tensor-core path's A' tiles).
template <bool TILES>
__global__ void __launch_bounds__(256) gain_grad_w_kernel(const float2 *R, const float2 *g, const float2 *M,
                                                          const float *scale, float2 *grad, void *Wv, int S)
{
    float2 *W = TILES ? nullptr : static_cast<float2 *>(Wv);
    const int N = 2 * S;
    const int c = (int)(blockIdx.x % (unsigned)N), unit = (int)(blockIdx.x / (unsigned)N);
    const int sc = c >> 1, pc = c & 1;
    const long long B4 = (long long)S * (S + 1) / 2 * 4;
    const float2 *Ru = R + unit * B4;
    const float2 *Mu = M + unit * B4;
    const float2 *gu = g + (long long)unit * N;
    const float s = 2.f * (scale ? *scale : 1.f);
    const float2 gc = cconj(gu[c]);
    float2 acc = make_float2(0.f, 0.f);
    for (int b = threadIdx.x; b < N; b += blockDim.x) {
        const int sb = b >> 1, pb = b & 1;
        const float2 gb = gu[b];
        float2 w = make_float2(0.f, 0.f);
        if (sc <= sb) { // (c, b) in the triangle: E_cb g_b conj(R_cb)
            const long long k = bl(sc, sb) * 4 + pc * 2 + pb;
            const float2 e = residual(Ru, gu, Mu, sc, pc, sb, pb);
            const float2 t = cmul(cmul(e, gb), cconj(Ru[k]));
            acc.x += t.x;
            acc.y += t.y;
            w.x += e.x;
            w.y += e.y;
        }
        if (sb <= sc) { // (b, c) in the triangle: conj(E_bc) g_b R_bc
            const long long k = bl(sb, sc) * 4 + pb * 2 + pc;
            const float2 e = residual(Ru, gu, Mu, sb, pb, sc, pc);
            const float2 t = cmul(cmul(cconj(e), gb), Ru[k]);
            acc.x += t.x;
            acc.y += t.y;
            w.x += e.x;
            w.y -= e.y;
        }
        if (TILES) {
            const float2 v = cmul(cmul(gc, w), gb);
            store_w_tiles(static_cast<float *>(Wv), unit, S, c, b, make_float2(s * v.x, s * v.y));
        } else if (W) {
            const float2 v = cmul(cmul(gc, w), gb);
            W[((long long)unit * N + c) * N + b] = make_float2(s * v.x, s * v.y);
        }
    }
    __shared__ float2 red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[threadIdx.x].x += red[threadIdx.x + h].x;
            red[threadIdx.x].y += red[threadIdx.x + h].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[(long long)unit * N + c] = make_float2(s * red[0].x, s * red[0].y);
}

// grad_x[unit][s][t][p] = sum_b W'[unit][(s,p)][b] x[unit][b][t], b = (s', p').
// CTA tile: 16 TM rows (c) x 64 times; thread tile TM rows x 4 times. The b
// axis goes through shared memory 16 at a time in two stages: the
// asynchronous copies of step k + 1 are in flight while step k is computed.
// W' is staged k-major, so that a thread's TM rows at one k are contiguous.
#ifndef CORR_IG_TM
#define CORR_IG_TM 8
#endif
template <int TM>
__global__ void __launch_bounds__(256) input_grad_gemm_kernel(const float2 *W, const float2 *x,
                                                              float2 *gx, int S, int T)
{
    constexpr int BM = 16 * TM;
    constexpr int WLD = BM + 2;   // padded row: the staging writes of one k spread over banks
    const int N = 2 * S;
    const int unit = blockIdx.z;
    const int c0 = blockIdx.y * BM;
    const int t0 = blockIdx.x * 64;
    const float2 *Wu = W + (long long)unit * N * N;
    const float2 *xu = x + (long long)unit * S * T * 2;
    float2 *gu = gx + (long long)unit * S * T * 2;
    extern __shared__ __align__(16) float2 ig_smem[];
    float2 (*Ws)[16][WLD] = reinterpret_cast<float2 (*)[16][WLD]>(ig_smem);          // [2][16][WLD]
    float2 (*Xs)[16][64] = reinterpret_cast<float2 (*)[16][64]>(ig_smem + 2 * 16 * WLD); // [2][16][64]
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    float2 acc[TM][4];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[a][q] = make_float2(0.f, 0.f);

    // Stage the W' and x tiles of columns b0 .. b0+15 (zero outside the
    // matrix: a copy with no source bytes fills zeros and reads nothing).
    auto stage = [&](int st, int b0) {
#pragma unroll
        for (int e = tid; e < BM * 16; e += 256) {
            const int r = e >> 4, k = e & 15;
            const int c = c0 + r, b = b0 + k;
            const bool in = c < N && b < N;
            cp_async_small<8>(smem_u32(&Ws[st][k][r]), in ? Wu + (long long)c * N + b : Wu, in ? 8u : 0u);
        }
#pragma unroll
        for (int e = tid; e < 16 * 64; e += 256) {
            // e -> (station-local, t, pol) in memory order of x
            const int sl = e >> 7, rem = e & 127, tt = rem >> 1, pp = rem & 1;
            const int s = (b0 >> 1) + sl, t = t0 + tt;
            const bool in = s < S && t < T;
            cp_async_small<8>(smem_u32(&Xs[st][2 * sl + pp][tt]),
                              in ? xu + ((long long)s * T + t) * 2 + pp : xu, in ? 8u : 0u);
        }
        cp_async_commit();
    };
    stage(0, 0);
    for (int b0 = 0, st = 0; b0 < N; b0 += 16, st ^= 1) {
        if (b0 + 16 < N) {
            stage(st ^ 1, b0 + 16);   // that buffer was released by the barrier closing the last step
            cp_async_wait<1>();       // this thread's copies of step b0 have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();              // ... and everyone else's
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float2 wv[TM], xv[4];
#pragma unroll
            for (int a = 0; a < TM; a += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(&Ws[st][k][ty * TM + a]);
                wv[a] = make_float2(v.x, v.y);
                wv[a + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int q = 0; q < 4; q += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(&Xs[st][k][tx * 4 + q]);
                xv[q] = make_float2(v.x, v.y);
                xv[q + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[a][q].x = fmaf(wv[a].x, xv[q].x, fmaf(-wv[a].y, xv[q].y, acc[a][q].x));
                    acc[a][q].y = fmaf(wv[a].x, xv[q].y, fmaf(wv[a].y, xv[q].x, acc[a][q].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const int c = c0 + ty * TM + a;
        if (c >= N) continue;
        const int s = c >> 1, pp = c & 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = t0 + tx * 4 + q;
            if (t < T) gu[((long long)s * T + t) * 2 + pp] = acc[a][q];
        }
    }
}

} // namespace

cudaError_t gain_loss_launch(const float2 *R, const float2 *g, const float2 *M, float2 *V,
                             float *partial, float *loss, int S, int units, cudaStream_t s)
{
    gain_loss_kernel<<<units, 256, 0, s>>>(R, g, M, V, partial, S);
    if (loss) sum_partials_kernel<<<1, 256, 0, s>>>(partial, units, loss);
    return cudaGetLastError();
}

cudaError_t gain_grad_launch(const float2 *R, const float2 *g, const float2 *M,
                             const float *scale, float2 *grad_g, void *W, int S, int units,
                             cudaStream_t s, int tiles)
{
    const int N = 2 * S;
    // threads: a power of two (the reduction halves), up to 256, about N
    int threads = 32;
    while (threads < N && threads < 256) threads <<= 1;
    if (tiles && W)
        gain_grad_w_kernel<true><<<(unsigned)((long long)N * units), threads, 0, s>>>(R, g, M, scale, grad_g, W, S);
    else
        gain_grad_w_kernel<false><<<(unsigned)((long long)N * units), threads, 0, s>>>(R, g, M, scale, grad_g, W, S);
    return cudaGetLastError();
}

cudaError_t input_grad_launch(const float2 *x, const float2 *W, float2 *grad_x, int S, int T, int units,
                              cudaStream_t s)
{
    const long long N = 2LL * S;
    if (T > 0) {
        constexpr int BM = 16 * CORR_IG_TM;
        constexpr size_t smem = (size_t)(2 * 16 * (BM + 2) + 2 * 16 * 64) * sizeof(float2);
        cudaError_t e = cudaFuncSetAttribute(input_grad_gemm_kernel<CORR_IG_TM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // at most 65535 units per launch (the grid's z dimension)
        for (long long u0 = 0; u0 < units; u0 += 65535) {
            const unsigned n = (unsigned)std::min<long long>(65535, units - u0);
            dim3 grid((T + 63) / 64, (unsigned)((N + BM - 1) / BM), n);
            input_grad_gemm_kernel<CORR_IG_TM><<<grid, 256, smem, s>>>(W + u0 * N * N, x + u0 * S * T * 2,
                                                                        grad_x + u0 * S * T * 2, S, T);
        }
    }
    return cudaGetLastError();
}

} // namespace corr
