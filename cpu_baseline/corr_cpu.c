/* Multithreaded FP32 CPU correlator: the design the paper reports as the
 * fastest on a general-purpose multi-core CPU (Section 4.1 and its results
 * in Section 5): 2x2 station tiles, the integration-time loop vectorised
 * (consecutive time samples in the lanes of a vector), and threads over the
 * work. It is a comparison baseline for the GPU path, not the product path
 * and not the oracle.
 *
 * Input  x[unit][station][time][pol] complex float32 (re, im interleaved).
 * Output V[unit][baseline][p1][p2] complex float32,
 *        V_{s1 s2}[p1][p2] = sum_t x_{s1,p1}(t) conj(x_{s2,p2}(t)), s1 <= s2,
 *        baseline(s1, s2) = s2 (s2 + 1) / 2 + s1 (Section 2, Fig. 2).
 *
 * Each thread takes one (unit, tile row) at a time. A 2x2 tile keeps its 32
 * partial sums (2 x 2 stations x 4 pol pairs x re/im) as VL lanes each: lane
 * v accumulates the time samples t = v (mod VL), so the lane loops below
 * vectorise without reassociating any sum; the lanes are added in a fixed
 * order at the end. Plain C (no intrinsics): the compiler's vectoriser
 * targets whatever vector unit the host has. */
#include <stddef.h>
#include <omp.h>

#define VL 8

static void tile(const float *restrict x, size_t T, int S, int i, int j, float *restrict out_unit)
{
    /* stations of the tile: rows a0, a1 = 2i, 2i+1; columns b0, b1 = 2j, 2j+1 */
    const int a[2] = {2 * i, 2 * i + 1};
    const int b[2] = {2 * j, 2 * j + 1};
    const float *ra[2], *rb[2];
    int ok_a[2], ok_b[2];
    for (int k = 0; k < 2; ++k) {
        ok_a[k] = a[k] < S;
        ok_b[k] = b[k] < S;
        ra[k] = x + (size_t)(ok_a[k] ? a[k] : a[0]) * T * 4;
        rb[k] = x + (size_t)(ok_b[k] ? b[k] : b[0]) * T * 4;
    }
    /* acc[m][n][p][q][c][v]: row station m, column station n, pols p, q,
     * c = 0 real / 1 imaginary part, lane v */
    float acc[2][2][2][2][2][VL];
    for (int m = 0; m < 2; ++m)
        for (int n = 0; n < 2; ++n)
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q)
                    for (int c = 0; c < 2; ++c)
                        for (int v = 0; v < VL; ++v) acc[m][n][p][q][c][v] = 0.f;
    const size_t Tv = T / VL * VL;
    for (size_t t0 = 0; t0 < Tv; t0 += VL) {
        /* samples of the 4 stations, 2 pols, re/im, VL times: deinterleaved */
        float sa[2][2][2][VL], sb[2][2][2][VL];
        for (int k = 0; k < 2; ++k)
            for (int v = 0; v < VL; ++v) {
                const float *pa = ra[k] + (t0 + v) * 4, *pb = rb[k] + (t0 + v) * 4;
                sa[k][0][0][v] = pa[0];
                sa[k][0][1][v] = pa[1];
                sa[k][1][0][v] = pa[2];
                sa[k][1][1][v] = pa[3];
                sb[k][0][0][v] = pb[0];
                sb[k][0][1][v] = pb[1];
                sb[k][1][0][v] = pb[2];
                sb[k][1][1][v] = pb[3];
            }
        for (int m = 0; m < 2; ++m)
            for (int n = 0; n < 2; ++n)
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q)
                        for (int v = 0; v < VL; ++v) {
                            const float ar = sa[m][p][0][v], ai = sa[m][p][1][v];
                            const float br = sb[n][q][0][v], bi = sb[n][q][1][v];
                            /* a conj(b): the four multiply-adds of Section 2 */
                            acc[m][n][p][q][0][v] += ar * br + ai * bi;
                            acc[m][n][p][q][1][v] += ai * br - ar * bi;
                        }
    }
    for (size_t t = Tv; t < T; ++t) /* the time samples left over, in lane 0 */
        for (int m = 0; m < 2; ++m)
            for (int n = 0; n < 2; ++n)
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) {
                        const float ar = ra[m][t * 4 + 2 * p], ai = ra[m][t * 4 + 2 * p + 1];
                        const float br = rb[n][t * 4 + 2 * q], bi = rb[n][t * 4 + 2 * q + 1];
                        acc[m][n][p][q][0][0] += ar * br + ai * bi;
                        acc[m][n][p][q][1][0] += ai * br - ar * bi;
                    }
    for (int m = 0; m < 2; ++m)
        for (int n = 0; n < 2; ++n) {
            const int s1 = a[m], s2 = b[n];
            if (!ok_a[m] || !ok_b[n] || s1 > s2) continue;
            float *o = out_unit + ((size_t)s2 * (s2 + 1) / 2 + s1) * 8;
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q)
                    for (int c = 0; c < 2; ++c) {
                        float s = 0.f;
                        for (int v = 0; v < VL; ++v) s += acc[m][n][p][q][c][v];
                        o[(p * 2 + q) * 2 + c] = s;
                    }
        }
}

/* Correlates `units` channels of S stations and T samples (two pols). */
void cpu_correlate(const float *x, long units, int S, long T, float *out, int threads)
{
    const int nt = (S + 1) / 2; /* tiles per side */
    const size_t B = (size_t)S * (S + 1) / 2;
    const long work = units * nt;
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
    for (long w = 0; w < work; ++w) {
        const long u = w / nt;
        const int i = (int)(w % nt);
        const float *xu = x + (size_t)u * S * T * 4;
        float *ou = out + (size_t)u * B * 8;
        for (int j = i; j < nt; ++j) tile(xu, (size_t)T, S, i, j, ou);
    }
}

int cpu_threads(void) { return omp_get_max_threads(); }
