/*
 * nsfrb_oracle.c -- plain, slow FP64 CPU statement of the image-plane
 * single-pulse search of the DSA-110 NSFRB paper (arXiv 2510.18136).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle: it is built and
 * called by the test-suite, by the smoke check and by the timed CPU baseline
 * of the benchmark, never by the library.  It shares no code, header, table
 * or constant with the CUDA implementation.
 *
 * Everything is written in the order of the paper's description of the
 * search (Sec. 2.2, "cerberus Search Pipeline"):
 *   median subtraction per pixel (optional robust normalisation)
 *   -> integer-delay de-dispersion with pre-computed shifts
 *   -> boxcar filtering over a set of widths
 *   -> normalisation by the noise level to S/N
 *   -> maximum S/N and its time of arrival over time.
 * The boxcar sums use FP64 prefix sums (exact to ~1e-16 relative); a direct
 * double-loop summation mode is provided for tiny cubes so that the prefix
 * form can itself be checked by brute force.
 *
 * Every float result is computed in double precision from the caller's
 * input values (float32, or bf16/fp16 values widened exactly to float32).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * Cold-plasma dispersion delay table (Sec. 2.2: shift indices per frequency
 * channel are pre-computed; the delay law is the standard
 * dt = K * DM * (f_lo^-2 - f_hi^-2) with K = 4.149 ms GHz^2 and f in GHz).
 *
 * shifts[d*n_sub + k] = floor(K*DM_d*(1/f_k^2 - 1/f_top^2)/t_samp + 0.5)
 * with f_top the highest subband centre (the frame the TOA refers to).
 * The expression order is fixed: delay_ms first, then the rounding.
 * Returns 0, or -1 on invalid arguments.
 */
int orc_delay_table(int n_sub, const double *freq_mhz, int n_dm,
                    const double *dm, double k_dm_ms, double t_samp_ms,
                    int32_t *shifts)
{
    if (n_sub <= 0 || n_dm <= 0 || t_samp_ms <= 0.0) return -1;
    double f_top = freq_mhz[0];
    for (int k = 1; k < n_sub; ++k)
        if (freq_mhz[k] > f_top) f_top = freq_mhz[k];
    double f_top_ghz = f_top / 1000.0;
    for (int d = 0; d < n_dm; ++d) {
        for (int k = 0; k < n_sub; ++k) {
            double f_ghz = freq_mhz[k] / 1000.0;
            double delay_ms = k_dm_ms * dm[d] *
                (1.0 / (f_ghz * f_ghz) - 1.0 / (f_top_ghz * f_top_ghz));
            shifts[(int64_t)d * n_sub + k] =
                (int32_t)floor(delay_ms / t_samp_ms + 0.5);
        }
    }
    return 0;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Median of v[0..n) by sorting a copy; even n -> mean of the two middle
 * order statistics. */
static double median_of(const double *v, int n, double *work)
{
    memcpy(work, v, sizeof(double) * (size_t)n);
    qsort(work, (size_t)n, sizeof(double), cmp_double);
    if (n & 1) return work[n / 2];
    return 0.5 * (work[n / 2 - 1] + work[n / 2]);
}

/*
 * Robust per-(pixel, subband) normalisation over the time window (Sec. 2.2
 * removes each pixel's median and scales by a running noise estimate; the
 * robust reading takes the median absolute deviation as that estimate):
 *   m   = median_t x[t]
 *   MAD = median_t |x[t] - m|
 *   y[t] = (x[t] - m) / (1.4826 * MAD)
 * x and y are [n_rows][n_t] (a row = one pixel and one subband).
 * Returns the number of rows whose MAD is zero (those rows are left zero).
 */
int64_t orc_mad_normalise(int64_t n_rows, int n_t, const double *x, double *y)
{
    int64_t n_bad = 0;
#pragma omp parallel reduction(+ : n_bad)
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)n_t);
        double *dev = (double *)malloc(sizeof(double) * (size_t)n_t);
#pragma omp for schedule(static)
        for (int64_t r = 0; r < n_rows; ++r) {
            const double *xr = x + r * n_t;
            double *yr = y + r * n_t;
            double m = median_of(xr, n_t, work);
            for (int t = 0; t < n_t; ++t) dev[t] = fabs(xr[t] - m);
            double mad = median_of(dev, n_t, work);
            if (mad == 0.0) {
                ++n_bad;
                for (int t = 0; t < n_t; ++t) yr[t] = 0.0;
                continue;
            }
            for (int t = 0; t < n_t; ++t) yr[t] = (xr[t] - m) / (1.4826 * mad);
        }
        free(work);
        free(dev);
    }
    return n_bad;
}

/*
 * The search itself (Sec. 2.2), for n pixels given as a dense
 * x[n][n_sub][n_t] array, in double precision:
 *
 *   smax_d   = max_k shifts[d][k];  L_d = n_t - smax_d
 *   D_d[t]   = sum_k x[k][t + shifts[d][k]]            t in [0, L_d)
 *   B_dw[t]  = sum_{u=t}^{t+w-1} D_d[u]                t in [0, L_d - w]
 *   S/N      = B_dw[t] / (sigma * sqrt(w))
 *   snr[d][w] = max_t S/N,  tidx[d][w] = smallest argmax t,
 *   snr2[d][w] = max over t != tidx of S/N (near-tie margin), -inf if none.
 * A (d, w) pair with w > L_d has no trials: snr = -inf, tidx = -1.
 *
 * t_lo (optional, [n_dm][n_w] or NULL) restricts trials to t >= t_lo[d][w];
 * the serving loop searches only the trials that end in the newest block.
 *
 * direct == 0: boxcar sums as differences of FP64 prefix sums
 *              P[0] = 0, P[t+1] = P[t] + D[t], B = P[t+w] - P[t].
 * direct != 0: boxcar sums as the explicit double loop over u and k
 *              (brute force, tiny cubes only).
 */
void orc_search(int64_t n, int n_sub, int n_t, const double *x,
                const double *sigma, int n_dm, const int32_t *shifts,
                int n_w, const int32_t *widths, const int32_t *t_lo,
                int direct, double *snr, int32_t *tidx, double *snr2)
{
#pragma omp parallel
    {
        double *D = (double *)malloc(sizeof(double) * (size_t)(n_t + 1));
        double *P = (double *)malloc(sizeof(double) * (size_t)(n_t + 1));
#pragma omp for schedule(dynamic, 4)
        for (int64_t p = 0; p < n; ++p) {
            const double *xp = x + p * (int64_t)n_sub * n_t;
            for (int d = 0; d < n_dm; ++d) {
                const int32_t *s = shifts + (int64_t)d * n_sub;
                int smax = 0;
                for (int k = 0; k < n_sub; ++k)
                    if (s[k] > smax) smax = s[k];
                int L = n_t - smax;
                if (!direct && L > 0) {
                    for (int t = 0; t < L; ++t) {
                        double acc = 0.0;
                        for (int k = 0; k < n_sub; ++k)
                            acc += xp[(int64_t)k * n_t + t + s[k]];
                        D[t] = acc;
                    }
                    P[0] = 0.0;
                    for (int t = 0; t < L; ++t) P[t + 1] = P[t] + D[t];
                }
                for (int wi = 0; wi < n_w; ++wi) {
                    int w = widths[wi];
                    int64_t o = (p * n_dm + d) * n_w + wi;
                    double best = -INFINITY, second = -INFINITY;
                    int bt = -1;
                    int t0 = 0;
                    if (t_lo) {
                        t0 = t_lo[d * n_w + wi];
                        if (t0 < 0) t0 = 0;
                    }
                    double norm = sigma[p] * sqrt((double)w);
                    for (int t = t0; t + w <= L; ++t) {
                        double b;
                        if (direct) {
                            b = 0.0;
                            for (int u = t; u < t + w; ++u)
                                for (int k = 0; k < n_sub; ++k)
                                    b += xp[(int64_t)k * n_t + u + s[k]];
                        } else {
                            b = P[t + w] - P[t];
                        }
                        double v = b / norm;
                        if (v > best) {
                            second = best;
                            best = v;
                            bt = t;
                        } else if (v > second) {
                            second = v;
                        }
                    }
                    snr[o] = best;
                    tidx[o] = bt;
                    if (snr2) snr2[o] = second;
                }
            }
        }
        free(D);
        free(P);
    }
}
