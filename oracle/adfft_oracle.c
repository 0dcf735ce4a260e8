/*
 * FP64 direct-summation oracle for the alpha-densified DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * What it computes (Sec. 2, Eq. 7, with the scale factor of Eq. 2):
 *
 *     X_m = S * sum_{n=0}^{N-1} x_n * exp(-2*pi*i * m*n / M),   m = 0 .. M-1,
 *
 * where M = alpha*N is the number of output bins (Eq. 6: nu -> m/(alpha T),
 * m = 0 .. alpha N - 1) and S = T/N (Eq. 2; S = 1 reproduces Eq. 7 as
 * printed).  The sign convention is W_M^{mn} = exp(-2 pi i m n / M) (Sec. 3).
 *
 * The adjoint (conjugate transpose of the same N x M matrix, the operator in
 * the second line of Eq. 7 up to the factor 1/(alpha N)) is
 *
 *     xb_n = S * sum_{m=0}^{M-1} exp(+2*pi*i * m*n / M) * g_m.
 *
 * Implementation: the definition written out.  The phase index (m*n) mod M is
 * carried as an exact 64-bit integer (incremented by m at every step of n, so
 * no large product is ever rounded), mapped to the symmetric range
 * (-M/2, M/2] and only then turned into an angle; each term's cos/sin comes
 * from libm in double precision.  The sum over n is Neumaier-compensated.
 * OpenMP parallelises over (signal, bin) pairs; there is no FFT and no
 * reordering of the sum beyond the compensation.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* Neumaier-compensated accumulator (sum + running correction). */
typedef struct { double s, c; } acc_t;

static inline void acc_add(acc_t *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else                       a->c += (v - t) + a->s;
    a->s = t;
}
static inline double acc_get(const acc_t *a) { return a->s + a->c; }

/* exp(sign * 2 pi i * j / M) for an exact integer index 0 <= j < M. */
static inline void unit_root(int64_t j, int64_t M, int sign, double *c, double *s) {
    int64_t k = (2 * j > M) ? j - M : j;          /* symmetric range (-M/2, M/2] */
    double ang = (ORACLE_TWO_PI * (double)k) / (double)M;
    *c = cos(ang);
    *s = (double)sign * sin(ang);
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Forward transform, Eq. 7 with scale S.
 *   x_re, x_im : [batch][N]; x_im == NULL means a real input signal.
 *   bins       : nbins bin indices m (each 0 <= m < M); NULL means all M bins
 *                in natural order (then nbins must equal M).
 *   X_re, X_im : [batch][nbins] outputs.
 * Returns 0, or -1 on invalid sizes.
 */
int oracle_alpha_dft(int64_t batch, int64_t N, int64_t M, double S,
                     const double *x_re, const double *x_im,
                     const int64_t *bins, int64_t nbins,
                     double *X_re, double *X_im, int nthreads) {
    if (batch < 0 || N < 1 || M < 1 || nbins < 0) return -1;
    if (bins == NULL && nbins != M) return -1;
    int64_t total = batch * nbins;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < total; ++t) {
        int64_t b = t / nbins, q = t % nbins;
        int64_t m = bins ? bins[q] : q;
        const double *xr = x_re + b * N;
        const double *xi = x_im ? x_im + b * N : NULL;
        acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
        int64_t j = 0;                          /* (m*n) mod M, exact */
        int64_t step = m % M;
        for (int64_t n = 0; n < N; ++n) {
            double c, s;
            unit_root(j, M, -1, &c, &s);        /* W_M^{mn} */
            double a = xr[n], bi = xi ? xi[n] : 0.0;
            acc_add(&re, a * c - bi * s);
            acc_add(&im, a * s + bi * c);
            j += step;
            if (j >= M) j -= M;
        }
        X_re[t] = S * acc_get(&re);
        X_im[t] = S * acc_get(&im);
    }
    return 0;
}

/* One output sample of the adjoint: S * sum_m conj(W_M^{mn}) g_m for signal row gr, gi. */
static void adjoint_sample(int64_t N, int64_t M, double S, const double *gr, const double *gi,
                           int64_t n, double *out_re, double *out_im) {
    (void)N;
    acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
    int64_t j = 0;                          /* (m*n) mod M, exact */
    int64_t step = n % M;
    for (int64_t m = 0; m < M; ++m) {
        double c, s;
        unit_root(j, M, +1, &c, &s);        /* conj(W_M^{mn}) */
        acc_add(&re, gr[m] * c - gi[m] * s);
        acc_add(&im, gr[m] * s + gi[m] * c);
        j += step;
        if (j >= M) j -= M;
    }
    *out_re = S * acc_get(&re);
    *out_im = S * acc_get(&im);
}

/*
 * Adjoint transform (conjugate transpose of the Eq. 7 matrix, times S).
 *   g_re, g_im : [batch][M] (all M bins in natural order).
 *   xb_re, xb_im : [batch][N] outputs.
 */
int oracle_alpha_dft_adjoint(int64_t batch, int64_t N, int64_t M, double S,
                             const double *g_re, const double *g_im,
                             double *xb_re, double *xb_im, int nthreads) {
    if (batch < 0 || N < 1 || M < 1) return -1;
    int64_t total = batch * N;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < total; ++t) {
        int64_t b = t / N, n = t % N;
        adjoint_sample(N, M, S, g_re + b * M, g_im + b * M, n, &xb_re[t], &xb_im[t]);
    }
    return 0;
}

/*
 * The same adjoint at chosen output samples only (for transforms whose full
 * adjoint would take too long): xb[b][q] = sample samples[q] (0 <= samples[q] < N)
 * of signal b.  Same arithmetic per sample as oracle_alpha_dft_adjoint.
 *   xb_re, xb_im : [batch][nsamples] outputs.
 */
int oracle_alpha_dft_adjoint_samples(int64_t batch, int64_t N, int64_t M, double S,
                                     const double *g_re, const double *g_im,
                                     const int64_t *samples, int64_t nsamples,
                                     double *xb_re, double *xb_im, int nthreads) {
    if (batch < 0 || N < 1 || M < 1 || nsamples < 0 || (nsamples > 0 && samples == NULL)) return -1;
    for (int64_t q = 0; q < nsamples; ++q)
        if (samples[q] < 0 || samples[q] >= N) return -1;
    int64_t total = batch * nsamples;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < total; ++t) {
        int64_t b = t / nsamples, q = t % nsamples;
        adjoint_sample(N, M, S, g_re + b * M, g_im + b * M, samples[q], &xb_re[t], &xb_im[t]);
    }
    return 0;
}
