/*
 * Second FP64 CPU path for the polyphase filter bank of Adamek, Novotny and
 * Armour, "The Implementation of a Real-Time Polyphase Filter"
 * (arXiv 1411.3656): the same FIR stage followed by an iterative radix-2 FFT
 * instead of the naive O(N^2) DFT.
 *
 * TEST INFRASTRUCTURE ONLY, like ppf_oracle.c, and independent of it (no
 * shared code, header or table; compiled into its own library).  It serves
 * two roles:
 *   - a pin: an O(N log N) transform that must agree with the naive DFT to
 *     FP64 rounding (about 1e-13 relative), and that must pass every pin the
 *     naive oracle passes;
 *   - a CPU baseline: the paper's CPU implementation filters with its own
 *     code and takes the FFT from a library (Section 3, the CPU subsection
 *     and the paragraph on FFT libraries); this stands in for that pairing
 *     with a plain FFT of our own, in FP64, OpenMP over spectra.
 *
 * FIR stage (Section 2, Eq. 1), index convention of this library:
 *     y[s][c] = sum_{t=0}^{T-1} h[t*N + c] * x[(s+t)*N + c].
 * FFT stage (Section 2: the channels are the DFT bins; Section 3: a standard
 * forward FFT): for every spectrum,
 *     Y[k] = sum_{c=0}^{N-1} y[c] * exp(-2*pi*i*k*c/N),
 * forward sign, unnormalised, natural bin order; N a power of two.
 * Radix-2 decimation in time: the input is put in bit-reversed order, then
 * log2(N) stages of butterflies of growing span L = 2, 4, ..., N combine
 * pairs (u, v) at distance L/2 into (u + w*v, u - w*v) with w = W_L^j,
 * W_L = exp(-2*pi*i/L), j the position inside the span.  W_L^j = W_N^(j*N/L),
 * taken from one table of W_N^m, m < N/2, evaluated in FP64.
 *
 * Layout as in ppf_oracle.c: complex values interleaved (re, im) as double;
 * window w of the FIR starts at x + w*window_stride (complex samples).
 * Functions return 0 on success, -1 on an invalid argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

/* FIR stage (Eq. 1) of one window into y (N complex values). */
static void fir_window(const double* xw, const double* h, int N, int T, double* y)
{
    for (int c = 0; c < N; ++c) {
        double re = 0.0, im = 0.0;
        for (int t = 0; t < T; ++t) {
            const double coeff = h[(int64_t)t * N + c];
            const double* xs = xw + 2 * ((int64_t)t * N + c);
            re = coeff * xs[0] + re;
            im = coeff * xs[1] + im;
        }
        y[2 * c] = re;
        y[2 * c + 1] = im;
    }
}

/* In-place iterative radix-2 FFT of a[0..N) (N a power of two), forward,
 * unnormalised.  tw holds W_N^m = (cos, -sin)(2*pi*m/N) for m < N/2. */
static void fft_radix2_inplace(double* a, int N, const double* tw)
{
    /* bit-reversed reordering */
    for (int i = 1, j = 0; i < N; ++i) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j |= bit;
        if (i < j) {
            double tr = a[2 * i], ti = a[2 * i + 1];
            a[2 * i] = a[2 * j];
            a[2 * i + 1] = a[2 * j + 1];
            a[2 * j] = tr;
            a[2 * j + 1] = ti;
        }
    }
    /* butterfly stages */
    for (int L = 2; L <= N; L <<= 1) {
        const int half = L / 2, step = N / L;
        for (int i = 0; i < N; i += L) {
            for (int j = 0; j < half; ++j) {
                const double wr = tw[2 * (j * step)], wi = tw[2 * (j * step) + 1];
                double* u = a + 2 * (i + j);
                double* v = a + 2 * (i + j + half);
                const double vr = v[0] * wr - v[1] * wi;
                const double vi = v[0] * wi + v[1] * wr;
                v[0] = u[0] - vr;
                v[1] = u[1] - vi;
                u[0] = u[0] + vr;
                u[1] = u[1] + vi;
            }
        }
    }
}

static double* twiddles(int N)
{
    const int half = N / 2 > 0 ? N / 2 : 1;
    double* tw = (double*)malloc(sizeof(double) * 2 * (size_t)half);
    if (!tw) return NULL;
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < half; ++m) {
        const double ang = two_pi * (double)m / (double)N;
        tw[2 * m] = cos(ang);
        tw[2 * m + 1] = -sin(ang);
    }
    return tw;
}

/* FFT stage only: n rows of N complex values. */
int ppf_cpu2_fft(const double* y, int N, int64_t n, double* Y)
{
    if (!y || !Y || !is_pow2(N) || n < 0) return -1;
    double* tw = twiddles(N);
    if (!tw) return -1;
    int64_t w;
#pragma omp parallel for schedule(static)
    for (w = 0; w < n; ++w) {
        double* Yw = Y + 2 * (w * (int64_t)N);
        memmove(Yw, y + 2 * (w * (int64_t)N), sizeof(double) * 2 * (size_t)N);
        fft_radix2_inplace(Yw, N, tw);
    }
    free(tw);
    return 0;
}

/* FIR stage only, n windows. */
int ppf_cpu2_fir(const double* x, int64_t window_stride, const double* h, int N, int T, int64_t n, double* y)
{
    if (!x || !h || !y || N < 1 || T < 1 || n < 0 || window_stride < 0) return -1;
    int64_t w;
#pragma omp parallel for schedule(static)
    for (w = 0; w < n; ++w) fir_window(x + 2 * (w * window_stride), h, N, T, y + 2 * (w * (int64_t)N));
    return 0;
}

/* Whole PPF: FIR then radix-2 FFT, window by window. */
int ppf_cpu2_ppf(const double* x, int64_t window_stride, const double* h, int N, int T, int64_t n, double* Y)
{
    if (!x || !h || !Y || !is_pow2(N) || T < 1 || n < 0 || window_stride < 0) return -1;
    double* tw = twiddles(N);
    if (!tw) return -1;
    int64_t w;
#pragma omp parallel for schedule(static)
    for (w = 0; w < n; ++w) {
        double* Yw = Y + 2 * (w * (int64_t)N);
        fir_window(x + 2 * (w * window_stride), h, N, T, Yw);
        fft_radix2_inplace(Yw, N, tw);
    }
    free(tw);
    return 0;
}

int ppf_cpu2_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
