/*
 * FP64 CPU oracle for the FDAS frequency-domain convolution power plane.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg call this code; the library's product path never
 * links or loads it, and it shares no code, header or table with the CUDA path.
 *
 * Complex values are interleaved (re, im) doubles.  Template banks are row-major
 * [m][k], outputs row-major [m][n].  Every output element is produced by one
 * thread in a fixed summation order, so results do not depend on the number of
 * OpenMP threads.
 *
 *   oracle_direct_conv / oracle_direct_power / oracle_direct_points
 *       Eq. (1): y[i] = sum_{k<K} x[i-k] h[k], i = 0..N-1, x[j] = 0 for j < 0,
 *       followed by the spectral power |y|^2 (Sec. 4.3: power, no square root).
 *   oracle_fft
 *       unnormalised radix-2 DFT, X[k] = sum_j v[j] exp(sign 2 pi i jk / L).
 *   oracle_ols_power
 *       Algorithm 2 (overlap-save): FFT of the zero-padded coefficients once,
 *       then per input sub-array (successive sub-arrays overlap by K-1, the first
 *       is preceded by K-1 zeros): FFT, element-wise product, inverse FFT,
 *       discard the first K-1 points, concatenate; then |y|^2.
 *
 *   oracle_harmonic_sums / oracle_harmonic_candidates
 *       the harmonic-summing stage that receives the power plane (Sec. 3 names
 *       it without defining it; read as the incoherent harmonic sum): for the
 *       fundamental at frequency bin r >= 1 and drift z, the powers at bin k r,
 *       drift k z, k = 1..h, added for h = 1, 2, 4, .., max_harm.
 *
 * Parity: pinned by tests against brute force (numpy.convolve), a delta
 * template, linearity, Parseval, numpy's FFT and the direct form; the harmonic
 * sums against closed forms (planes linear in row and column, constant planes,
 * single cells, injected harmonic trains).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

void oracle_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. (1) for one output point of one template: complex result in (*yr, *yi). */
static void direct_point(const double *x, int64_t n, const double *h, int k_len,
                         int64_t i, double *yr, double *yi)
{
    double sr = 0.0, si = 0.0;
    (void)n;
    for (int k = 0; k < k_len; ++k) {
        int64_t j = i - k;
        if (j < 0) break;                       /* x[j] = 0 for j < 0 */
        double xr = x[2 * j], xi = x[2 * j + 1];
        double hr = h[2 * k], hi = h[2 * k + 1];
        sr += xr * hr - xi * hi;
        si += xr * hi + xi * hr;
    }
    *yr = sr;
    *yi = si;
}

void oracle_direct_conv(const double *x, int64_t n, const double *h, int m, int k_len, double *y)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < m; ++z)
        for (int64_t i = 0; i < n; ++i)
            direct_point(x, n, h + (int64_t)2 * k_len * z, k_len, i,
                         &y[2 * ((int64_t)z * n + i)], &y[2 * ((int64_t)z * n + i) + 1]);
}

void oracle_power(const double *y, int64_t count, double *p)
{
    for (int64_t i = 0; i < count; ++i)
        p[i] = y[2 * i] * y[2 * i] + y[2 * i + 1] * y[2 * i + 1];
}

void oracle_direct_power(const double *x, int64_t n, const double *h, int m, int k_len, double *p)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < m; ++z)
        for (int64_t i = 0; i < n; ++i) {
            double yr, yi;
            direct_point(x, n, h + (int64_t)2 * k_len * z, k_len, i, &yr, &yi);
            p[(int64_t)z * n + i] = yr * yr + yi * yi;
        }
}

/* Power at a list of (template, index) points; p[j] for (zi[j], ii[j]). */
void oracle_direct_points(const double *x, int64_t n, const double *h, int m, int k_len,
                          const int32_t *zi, const int64_t *ii, int64_t npts, double *p)
{
    (void)m;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < npts; ++j) {
        double yr, yi;
        direct_point(x, n, h + (int64_t)2 * k_len * zi[j], k_len, ii[j], &yr, &yi);
        p[j] = yr * yr + yi * yi;
    }
}

/* Unnormalised radix-2 DFT in place; L must be a power of two.  Returns 0 or -1. */
int oracle_fft(double *v, int L, int sign)
{
    if (L < 1 || (L & (L - 1))) return -1;
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < L; ++i) {
        int bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = v[2 * i], ti = v[2 * i + 1];
            v[2 * i] = v[2 * j];         v[2 * i + 1] = v[2 * j + 1];
            v[2 * j] = tr;               v[2 * j + 1] = ti;
        }
    }
    /* butterflies; each twiddle is evaluated directly, not by recurrence */
    for (int len = 2; len <= L; len <<= 1) {
        int half = len >> 1;
        for (int q = 0; q < half; ++q) {
            double ang = sign * 2.0 * ORACLE_PI * (double)q / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int b = 0; b < L; b += len) {
                double *u = v + 2 * (b + q), *t = v + 2 * (b + q + half);
                double tr = t[0] * wr - t[1] * wi;
                double ti = t[0] * wi + t[1] * wr;
                t[0] = u[0] - tr;  t[1] = u[1] - ti;
                u[0] += tr;        u[1] += ti;
            }
        }
    }
    return 0;
}

/*
 * Algorithm 2 with segment FFT length L and segment step S (1 <= S <= L-K+1;
 * the algorithm's own choice is S = L-K+1, any smaller step gives the same
 * result in exact arithmetic).  Writes p[z*n + i].  Returns 0 or -1.
 */
int oracle_ols_power(const double *x, int64_t n, const double *h, int m, int k_len,
                     int L, int S, double *p)
{
    if (L < 2 || (L & (L - 1)) || k_len < 1 || k_len > L || S < 1 || S > L - k_len + 1 || n < 1)
        return -1;
    /* F{h}: zero-padded coefficients, transformed once */
    double *H = (double *)calloc((size_t)2 * L * m, sizeof(double));
    if (!H) return -1;
    for (int z = 0; z < m; ++z) {
        memcpy(H + (size_t)2 * L * z, h + (size_t)2 * k_len * z, sizeof(double) * 2 * k_len);
        oracle_fft(H + (size_t)2 * L * z, L, -1);
    }
    int64_t nseg = (n + S - 1) / S;
    int fail = 0;
    #pragma omp parallel
    {
        double *X = (double *)malloc(sizeof(double) * 2 * L);
        double *Y = (double *)malloc(sizeof(double) * 2 * L);
        if (!X || !Y) {
            #pragma omp atomic write
            fail = 1;
        } else {
            #pragma omp for schedule(dynamic, 4)
            for (int64_t s = 0; s < nseg; ++s) {
                /* sub-array x_s[t] = x[s*S - (K-1) + t], zero outside [0, n) */
                int64_t start = s * (int64_t)S - (k_len - 1);
                for (int t = 0; t < L; ++t) {
                    int64_t j = start + t;
                    X[2 * t] = (j >= 0 && j < n) ? x[2 * j] : 0.0;
                    X[2 * t + 1] = (j >= 0 && j < n) ? x[2 * j + 1] : 0.0;
                }
                oracle_fft(X, L, -1);
                int64_t valid = n - s * (int64_t)S;
                if (valid > S) valid = S;
                for (int z = 0; z < m; ++z) {
                    const double *Hz = H + (size_t)2 * L * z;
                    for (int f = 0; f < L; ++f) {           /* element-wise product */
                        Y[2 * f] = X[2 * f] * Hz[2 * f] - X[2 * f + 1] * Hz[2 * f + 1];
                        Y[2 * f + 1] = X[2 * f] * Hz[2 * f + 1] + X[2 * f + 1] * Hz[2 * f];
                    }
                    oracle_fft(Y, L, +1);                  /* inverse, scaled below */
                    for (int64_t t = 0; t < valid; ++t) {  /* discard the first K-1 */
                        double yr = Y[2 * (t + k_len - 1)] / L;
                        double yi = Y[2 * (t + k_len - 1) + 1] / L;
                        p[(int64_t)z * n + s * (int64_t)S + t] = yr * yr + yi * yi;
                    }
                }
            }
        }
        free(X);
        free(Y);
    }
    free(H);
    return fail ? -1 : 0;
}

/*
 * Harmonic sums of a power plane P [m][n] (float32, as stored), m odd, rows
 * ordered by drift z = y - c with c = (m-1)/2, column bin0 holding frequency
 * bin 0.  For the fundamental (r, z), r >= 1:
 *     S_h(r, z) = sum_{k=1..h} P[c + k z][bin0 + k r]        (added for k = 1, 2, ..)
 * defined where |h z| <= c and bin0 + h r <= n - 1, for the levels
 * h = 2^j <= max_harm.  S is [nlev][m][n] in FP64, cell (j, c + z, bin0 + r);
 * NaN where S_h is undefined.  Returns 0, or -1 on invalid arguments.
 */
static int harmonic_args_ok(int m, int64_t n, int64_t bin0, int max_harm)
{
    if (m < 1 || (m & 1) == 0 || n < 1 || bin0 < 0 || bin0 >= n) return 0;
    if (max_harm < 1 || max_harm > 32 || (max_harm & (max_harm - 1))) return 0;
    return 1;
}

static int harmonic_levels(int max_harm)
{
    int nlev = 0;
    while ((1 << nlev) <= max_harm) ++nlev;
    return nlev;
}

int oracle_harmonic_sums(const float *P, int m, int64_t n, int64_t bin0, int max_harm, double *S)
{
    if (!harmonic_args_ok(m, n, bin0, max_harm)) return -1;
    const int c = (m - 1) / 2, nlev = harmonic_levels(max_harm);
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < m; ++y) {
        const int z = y - c;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t r = i - bin0;
            double acc = 0.0;
            int k = 1;
            for (int j = 0; j < nlev; ++j) {
                const int h = 1 << j;
                int defined = r >= 1 && (int64_t)h * (z < 0 ? -z : z) <= c && bin0 + (int64_t)h * r <= n - 1;
                if (defined) {
                    for (; k <= h; ++k) acc += (double)P[(int64_t)(c + k * z) * n + bin0 + k * r];
                }
                S[((int64_t)j * m + y) * n + i] = defined ? acc : NAN;
            }
        }
    }
    return 0;
}

/*
 * The crossings S_h(r, z) > thr[j] (h = 2^j) of the same sums, in the order
 * (j, y, i) ascending: level j, row y = c + z, column i = bin0 + r and the sum.
 * Stores at most cap of them; returns their total count, or -1 on invalid
 * arguments or allocation failure.
 */
int64_t oracle_harmonic_candidates(const float *P, int m, int64_t n, int64_t bin0, int max_harm,
                                   const double *thr, int32_t *lev_out, int32_t *row_out,
                                   int64_t *bin_out, double *val_out, int64_t cap)
{
    if (!harmonic_args_ok(m, n, bin0, max_harm)) return -1;
    const int c = (m - 1) / 2, nlev = harmonic_levels(max_harm);
    int64_t *cnt = (int64_t *)calloc((size_t)nlev * m + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int pass = 0; pass < 2; ++pass) {
        /* pass 0 counts the crossings of each (level, row); pass 1 stores them */
        #pragma omp parallel for schedule(dynamic, 1)
        for (int y = 0; y < m; ++y) {
            const int z = y - c;
            int64_t next[32];
            for (int j = 0; j < nlev; ++j) next[j] = pass ? cnt[(int64_t)j * m + y] : 0;
            for (int64_t i = bin0 + 1; i < n; ++i) {
                const int64_t r = i - bin0;
                double acc = 0.0;
                int k = 1;
                for (int j = 0; j < nlev; ++j) {
                    const int h = 1 << j;
                    if ((int64_t)h * (z < 0 ? -z : z) > c || bin0 + (int64_t)h * r > n - 1) break;
                    for (; k <= h; ++k) acc += (double)P[(int64_t)(c + k * z) * n + bin0 + k * r];
                    if (acc > thr[j]) {
                        const int64_t at = next[j]++;
                        if (pass && at < cap) {
                            lev_out[at] = j;
                            row_out[at] = y;
                            bin_out[at] = i;
                            val_out[at] = acc;
                        }
                    }
                }
            }
            if (!pass)
                for (int j = 0; j < nlev; ++j) cnt[(int64_t)j * m + y] = next[j];
        }
        if (!pass) {   /* exclusive prefix over (level, row) */
            int64_t run = 0;
            for (int64_t q = 0; q < (int64_t)nlev * m; ++q) {
                const int64_t v = cnt[q];
                cnt[q] = run;
                run += v;
            }
            cnt[(int64_t)nlev * m] = run;
        }
    }
    const int64_t total = cnt[(int64_t)nlev * m];
    free(cnt);
    return total;
}
