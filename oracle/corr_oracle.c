/*
 * FP64 CPU oracle of the correlator X-step and of the gain-calibration loss
 * and its gradients.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this file: it is used by the tests, by the package's smoke check and by the
 * benchmark's CPU-baseline leg. It shares no code, header or table with the
 * CUDA path.
 *
 * Plain loops in the order the definitions are written, in double precision.
 * The only parallelism is OpenMP over independent channels (Section 2: the
 * channels are independent), which does not change any arithmetic.
 *
 * Complex numbers are stored as interleaved (re, im) doubles.
 *   samples   z : [unit][station][time][pol][2]     (unit = integration*channel)
 *   visibility  : [unit][baseline][pol1][pol2][2],  baseline = s2*(s2+1)/2 + s1
 *   gains     g : [unit][station][pol][2]
 */
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static long baseline_of(long s1, long s2) { return s2 * (s2 + 1) / 2 + s1; }

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Correlation (Section 2, the formula for C_{s1, s2>=s1, p1, p2} and the loop
 * nest of Fig. 2): for every channel, every station2, every station1 <= station2
 * and every polarisation pair, sum over time of
 *     samples[ch][station1][time][pol1] * conj(samples[ch][station2][time][pol2]).
 * The conjugate is on station2. Baselines are numbered s2*(s2+1)/2 + s1, the
 * order in which the loop nest visits them; the output axes are
 * [channel][baseline][pol1][pol2].
 */
void oracle_correlate(const double *z, long n_units, int S, int T, int P,
                      double *out)
{
    const long B = (long)S * (S + 1) / 2;
    long ch;
#pragma omp parallel for schedule(dynamic, 1)
    for (ch = 0; ch < n_units; ch++) {
        const double *zc = z + (size_t)ch * S * T * P * 2;
        double *oc = out + (size_t)ch * B * P * P * 2;
        for (long s2 = 0; s2 < S; s2++)
            for (long s1 = 0; s1 <= s2; s1++)
                for (int p1 = 0; p1 < P; p1++)
                    for (int p2 = 0; p2 < P; p2++) {
                        double sr = 0.0, si = 0.0;
                        for (long t = 0; t < T; t++) {
                            const double *a = zc + ((s1 * T + t) * P + p1) * 2;
                            const double *b = zc + ((s2 * T + t) * P + p2) * 2;
                            /* a * conj(b) = (ar*br + ai*bi) + i(ai*br - ar*bi) */
                            sr += a[0] * b[0] + a[1] * b[1];
                            si += a[1] * b[0] - a[0] * b[1];
                        }
                        double *o = oc + ((baseline_of(s1, s2) * P + p1) * P + p2) * 2;
                        o[0] = sr;
                        o[1] = si;
                    }
    }
}

/*
 * Gain-corrupted visibilities and calibration loss.
 *   y_{s,p}(t) = g_{s,p} x_{s,p}(t)  =>  V_ab = g_a conj(g_b) R_ab, R = corr(x)
 *   E_ab = V_ab - M_ab,  L = sum over units, baselines and pol pairs of |E_ab|^2.
 * V_out may be NULL. The loss is written to *loss.
 */
void oracle_gain_loss(const double *R, const double *g, const double *M,
                      long n_units, int S, int P, double *V_out, double *loss)
{
    const long B = (long)S * (S + 1) / 2;
    double total = 0.0;
    long ch;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (ch = 0; ch < n_units; ch++) {
        const double *gc = g + (size_t)ch * S * P * 2;
        for (long s2 = 0; s2 < S; s2++)
            for (long s1 = 0; s1 <= s2; s1++)
                for (int p1 = 0; p1 < P; p1++)
                    for (int p2 = 0; p2 < P; p2++) {
                        size_t k = (((size_t)ch * B + baseline_of(s1, s2)) * P + p1) * P + p2;
                        const double *ga = gc + (s1 * P + p1) * 2;
                        const double *gb = gc + (s2 * P + p2) * 2;
                        /* w = g_a * conj(g_b) */
                        double wr = ga[0] * gb[0] + ga[1] * gb[1];
                        double wi = ga[1] * gb[0] - ga[0] * gb[1];
                        double vr = wr * R[2 * k] - wi * R[2 * k + 1];
                        double vi = wr * R[2 * k + 1] + wi * R[2 * k];
                        if (V_out) { V_out[2 * k] = vr; V_out[2 * k + 1] = vi; }
                        double er = vr - M[2 * k], ei = vi - M[2 * k + 1];
                        total += er * er + ei * ei;
                    }
    }
    *loss = total;
}

/*
 * Gradient of the loss with respect to the gains, in the convention of
 * PyTorch for a real loss of complex inputs: grad = dL/dRe g + i dL/dIm g
 * = 2 dL/d(conj g). With E on the baseline set (a,b), a=(s1,p1), b=(s2,p2),
 * s1 <= s2:
 *   dL/d(conj g_c) = sum_{(c,b)} E_cb g_b conj(R_cb) + sum_{(a,c)} conj(E_ac) g_a R_ac
 * where an entry with a = b = c contributes to both sums.
 */
void oracle_gain_grad(const double *R, const double *g, const double *M,
                      long n_units, int S, int P, double *grad_g)
{
    const long B = (long)S * (S + 1) / 2;
    long ch;
#pragma omp parallel for schedule(static)
    for (ch = 0; ch < n_units; ch++) {
        const double *gc = g + (size_t)ch * S * P * 2;
        double *dc = grad_g + (size_t)ch * S * P * 2;
        for (long i = 0; i < (long)S * P * 2; i++) dc[i] = 0.0;
        for (long s2 = 0; s2 < S; s2++)
            for (long s1 = 0; s1 <= s2; s1++)
                for (int p1 = 0; p1 < P; p1++)
                    for (int p2 = 0; p2 < P; p2++) {
                        size_t k = (((size_t)ch * B + baseline_of(s1, s2)) * P + p1) * P + p2;
                        const double *ga = gc + (s1 * P + p1) * 2;
                        const double *gb = gc + (s2 * P + p2) * 2;
                        double rr = R[2 * k], ri = R[2 * k + 1];
                        double wr = ga[0] * gb[0] + ga[1] * gb[1];
                        double wi = ga[1] * gb[0] - ga[0] * gb[1];
                        double er = wr * rr - wi * ri - M[2 * k];
                        double ei = wr * ri + wi * rr - M[2 * k + 1];
                        /* term for c = a: E_ab * g_b * conj(R_ab) */
                        double tr = er * gb[0] - ei * gb[1];
                        double ti = er * gb[1] + ei * gb[0];
                        double *da = dc + (s1 * P + p1) * 2;
                        da[0] += 2.0 * (tr * rr + ti * ri);
                        da[1] += 2.0 * (ti * rr - tr * ri);
                        /* term for c = b: conj(E_ab) * g_a * R_ab */
                        double ur = er * ga[0] + ei * ga[1];
                        double ui = er * ga[1] - ei * ga[0];
                        double *db = dc + (s2 * P + p2) * 2;
                        db[0] += 2.0 * (ur * rr - ui * ri);
                        db[1] += 2.0 * (ur * ri + ui * rr);
                    }
    }
}

/*
 * Gradient of the loss with respect to the samples x (PyTorch convention,
 * 2 dL/d(conj x)). With y = g x and E as above,
 *   dL/d(conj y_c(t)) = sum_b W_cb y_b(t),
 *   W_cb = [s_c <= s_b] E_cb + [s_b <= s_c] conj(E_bc),
 * and dL/d(conj x_c) = conj(g_c) dL/d(conj y_c).
 */
void oracle_input_grad(const double *x, const double *R, const double *g,
                       const double *M, long n_units, int S, int T, int P,
                       double *grad_x)
{
    const long B = (long)S * (S + 1) / 2;
    const long N = (long)S * P;
    long ch;
#pragma omp parallel for schedule(dynamic, 1)
    for (ch = 0; ch < n_units; ch++) {
        const double *gc = g + (size_t)ch * N * 2;
        const double *xc = x + (size_t)ch * N * T * 2;
        double *oc = grad_x + (size_t)ch * N * T * 2;
        for (long sc = 0; sc < S; sc++)
            for (int pc = 0; pc < P; pc++) {
                const double *gcc = gc + (sc * P + pc) * 2;
                for (long t = 0; t < T; t++) {
                    double accr = 0.0, acci = 0.0;
                    for (long sb = 0; sb < S; sb++)
                        for (int pb = 0; pb < P; pb++) {
                            double wr = 0.0, wi = 0.0;
                            const double *gbb = gc + (sb * P + pb) * 2;
                            if (sc <= sb) { /* E_cb, baseline (s1=sc, s2=sb) */
                                size_t k = (((size_t)ch * B + baseline_of(sc, sb)) * P + pc) * P + pb;
                                double vr0 = gcc[0] * gbb[0] + gcc[1] * gbb[1];
                                double vi0 = gcc[1] * gbb[0] - gcc[0] * gbb[1];
                                wr += vr0 * R[2 * k] - vi0 * R[2 * k + 1] - M[2 * k];
                                wi += vr0 * R[2 * k + 1] + vi0 * R[2 * k] - M[2 * k + 1];
                            }
                            if (sb <= sc) { /* conj(E_bc), baseline (s1=sb, s2=sc) */
                                size_t k = (((size_t)ch * B + baseline_of(sb, sc)) * P + pb) * P + pc;
                                double vr0 = gbb[0] * gcc[0] + gbb[1] * gcc[1];
                                double vi0 = gbb[1] * gcc[0] - gbb[0] * gcc[1];
                                wr += vr0 * R[2 * k] - vi0 * R[2 * k + 1] - M[2 * k];
                                wi -= vr0 * R[2 * k + 1] + vi0 * R[2 * k] - M[2 * k + 1];
                            }
                            /* y_b(t) = g_b x_b(t) */
                            const double *xb = xc + ((sb * T + t) * P + pb) * 2;
                            double yr = gbb[0] * xb[0] - gbb[1] * xb[1];
                            double yi = gbb[0] * xb[1] + gbb[1] * xb[0];
                            accr += wr * yr - wi * yi;
                            acci += wr * yi + wi * yr;
                        }
                    /* 2 * conj(g_c) * acc */
                    double *o = oc + ((sc * T + t) * P + pc) * 2;
                    o[0] = 2.0 * (gcc[0] * accr + gcc[1] * acci);
                    o[1] = 2.0 * (gcc[0] * acci - gcc[1] * accr);
                }
            }
    }
}
