/*
 * FP64 CPU oracle for the polyphase filter bank (PPF) of Adamek, Novotny and
 * Armour, "The Implementation of a Real-Time Polyphase Filter" (arXiv 1411.3656).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes (plain definitions, no blocking, fusion or reordering):
 *
 *   FIR stage (Section 2, Eq. 1; loop order of Algorithm 1: spectra, then
 *   channels, then taps).  For N channels and T taps the filter of channel c
 *   runs along the samples of that channel, i.e. along every N-th input
 *   sample.  With the index convention fixed for this library,
 *
 *       y[s][c] = sum_{t=0}^{T-1} h[t*N + c] * x[(s+t)*N + c],
 *
 *   x complex, h real.  This is Eq. 1 with b_i = h[(T-1-i)*N + c] for
 *   channel c and output sample n = (s+T-1)*N + c: h[c] weights the oldest
 *   of the T samples, h[(T-1)*N + c] the newest.
 *
 *   DFT stage (Section 2: the N channels are the DFT bins; Section 3 uses a
 *   standard forward FFT from a library): for every spectrum s,
 *
 *       Y[s][k] = sum_{c=0}^{N-1} y[s][c] * exp(-2*pi*i * ((k*c) mod N) / N),
 *
 *   forward sign, no normalisation, natural bin order.  The angle is reduced
 *   exactly in integers and cos/sin are evaluated once per m = 0..N-1.
 *
 * Memory layout: complex values interleaved (re, im) as double.  A "window"
 * is the T*N consecutive input samples that one spectrum reads; window w
 * starts at x + w*window_stride (complex samples).  For a contiguous input
 * stream window_stride = N (consecutive spectra overlap by T-1 rows); for
 * gathered, non-overlapping windows window_stride = T*N.
 *
 * All functions return 0 on success and -1 on an invalid argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int bad_args(const void* x, const double* h, int N, int T, int64_t n,
                    const void* out, int64_t stride)
{
    if (!x || !h || !out) return 1;
    if (N < 1 || T < 1 || n < 0 || stride < 0) return 1;
    return 0;
}

/* FIR stage only (Eq. 1 / Algorithm 1): y[w][c] for n windows. */
int ppf_oracle_fir(const double* x, int64_t window_stride, const double* h,
                   int N, int T, int64_t n, double* y)
{
    if (bad_args(x, h, N, T, n, y, window_stride)) return -1;
    int64_t w;
#pragma omp parallel for schedule(static)
    for (w = 0; w < n; ++w) {                       /* spectra */
        const double* xw = x + 2 * (w * window_stride);
        double* yw = y + 2 * (w * (int64_t)N);
        for (int c = 0; c < N; ++c) {               /* channels */
            double re = 0.0, im = 0.0;
            for (int t = 0; t < T; ++t) {           /* taps */
                const double coeff = h[(int64_t)t * N + c];
                const double* xs = xw + 2 * ((int64_t)t * N + c);
                re = coeff * xs[0] + re;
                im = coeff * xs[1] + im;
            }
            yw[2 * c] = re;
            yw[2 * c + 1] = im;
        }
    }
    return 0;
}

/* DFT stage only: naive O(N^2) forward DFT of n rows of N complex values. */
int ppf_oracle_dft(const double* y, int N, int64_t n, double* Y)
{
    if (!y || !Y || N < 1 || n < 0) return -1;
    double* cs = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!cs) return -1;
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < N; ++m) {
        const double a = two_pi * (double)m / (double)N;
        cs[2 * m] = cos(a);
        cs[2 * m + 1] = sin(a);
    }
    int64_t w;
#pragma omp parallel for schedule(static)
    for (w = 0; w < n; ++w) {
        const double* yw = y + 2 * (w * (int64_t)N);
        double* Yw = Y + 2 * (w * (int64_t)N);
        for (int k = 0; k < N; ++k) {
            double re = 0.0, im = 0.0;
            for (int c = 0; c < N; ++c) {
                const int m = (int)(((int64_t)k * c) % N);
                const double cr = cs[2 * m], si = cs[2 * m + 1];
                /* y * exp(-i a) = (yr + i yi)(cos a - i sin a) */
                re += yw[2 * c] * cr + yw[2 * c + 1] * si;
                im += yw[2 * c + 1] * cr - yw[2 * c] * si;
            }
            Yw[2 * k] = re;
            Yw[2 * k + 1] = im;
        }
    }
    free(cs);
    return 0;
}

/* Whole PPF: FIR then DFT, for n windows. */
int ppf_oracle_ppf(const double* x, int64_t window_stride, const double* h,
                   int N, int T, int64_t n, double* Y)
{
    if (bad_args(x, h, N, T, n, Y, window_stride)) return -1;
    if (n == 0) return 0;
    double* y = (double*)malloc(sizeof(double) * 2 * (size_t)N * (size_t)n);
    if (!y) return -1;
    int rc = ppf_oracle_fir(x, window_stride, h, N, T, n, y);
    if (rc == 0) rc = ppf_oracle_dft(y, N, n, Y);
    free(y);
    return rc;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int ppf_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
