// Two-pass PPF through an L2-resident chunk buffer, for large N*T.
//
// When N*T is large the fused kernels must hold, on every SM at once, the
// coefficients of the channels it filters (registers), a T-row input window
// and the FFT's working rows (shared memory), and they alternate FIR and FFT
// phases behind CTA barriers.  Here the two steps run as separate kernels that
// each have the whole SM to themselves, and the filtered rows go through a
// chunk buffer small enough to stay in L2 (tens of MB against the 129 MB L2)
// instead of through HBM:
//
//   for each chunk of K spectra:
//     ppf_fir_kernel      x (HBM, read once) -> y chunk (L2)       Section 2, Eq. 1
//     ppf_fftrows_kernel  y chunk (L2)       -> Y (HBM, streaming) Section 2, DFT of each row
//
// HBM traffic stays at the fused kernels' 2 bytes per input byte plus the
// chunks' T-1 halo rows; the chunk round trip costs L2 bandwidth only.
#pragma once

#include "ppf_device.cuh"
#include "ppf_generic.cuh"

namespace ppf {

// ------------------------------------------------------------------ FIR pass
// CTA = 32*CW consecutive channels (one per thread) x RBT*STEPS consecutive
// spectra.  A thread keeps its channel's T coefficients as (h, h) pairs and
// walks its rows in steps of RBT spectra, one packed f32x2 FMA per tap:
// step [r, r+RBT) reads input rows r .. r+RBT+T-2.  The T-1 oldest of those
// were read by the thread's earlier steps (L1 hits); the RBT newest were
// loaded into registers during the previous step, so each step's HBM/L2
// latency overlaps the step before it.
template <int T, class In, int RBT, int CW, int STEPS>
__global__ void __launch_bounds__(32 * CW)
ppf_fir_kernel(const typename In::raw* __restrict__ x, const typename Coef<In>::type* __restrict__ h,
               float2* __restrict__ y, int N, int64_t S)
{
    const int c = blockIdx.x * (32 * CW) + threadIdx.x;
    float2 hh[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const float v = coef_f(h[t * N + c]);
        hh[t] = make_float2(v, v);
    }
    const int64_t in_rows = S + T - 1;
    const typename In::raw* xc = x + c;
    auto row = [&](int64_t r) {
        return r < in_rows ? decode(__ldg(xc + r * N)) : make_float2(0.f, 0.f);
    };
    int64_t r = (int64_t)blockIdx.y * (RBT * STEPS);
    float2 pf[RBT];
#pragma unroll
    for (int q = 0; q < RBT; ++q) pf[q] = row(r + T - 1 + q);
    for (int st = 0; st < STEPS && r < S; ++st, r += RBT) {
        float2 cur[RBT];
#pragma unroll
        for (int q = 0; q < RBT; ++q) cur[q] = pf[q];
        if (st + 1 < STEPS) {
#pragma unroll
            for (int q = 0; q < RBT; ++q) pf[q] = row(r + RBT + T - 1 + q);
        }
        float2 a[RBT];
#pragma unroll
        for (int i = 0; i < RBT; ++i) a[i] = make_float2(0.f, 0.f);
        // rows r .. r+T-2
#pragma unroll
        for (int u = 0; u < T - 1; ++u) {
            const float2 v = row(r + u);
#pragma unroll
            for (int i = 0; i < RBT; ++i) {
                const int t = u - i;
                if (t >= 0 && t < T) a[i] = __ffma2_rn(hh[t], v, a[i]);
            }
        }
        // rows r+T-1 .. r+T+RBT-2 (prefetched)
#pragma unroll
        for (int q = 0; q < RBT; ++q) {
            const int u = T - 1 + q;
#pragma unroll
            for (int i = 0; i < RBT; ++i) {
                const int t = u - i;
                if (t >= 0 && t < T) a[i] = __ffma2_rn(hh[t], cur[q], a[i]);
            }
        }
        float2* yp = y + r * N + c;
#pragma unroll
        for (int i = 0; i < RBT; ++i)
            if (r + i < S) yp[(int64_t)i * N] = a[i];
    }
}

// ------------------------------------------------------------------ FFT pass
// N-point forward DFTs of rows of y (Section 2): the first Stockham pass reads
// its butterfly inputs straight from global memory (L2-resident chunk,
// coalesced across threads), the remaining passes run in shared memory and
// the last one stores the spectra with streaming stores.
constexpr int kFftRowsThreads = 256;

template <int N>
__global__ void __launch_bounds__(kFftRowsThreads)
ppf_fftrows_kernel(const float2* __restrict__ y, const float2* __restrict__ tw, float2* __restrict__ Y, int64_t S)
{
    constexpr int NT = kFftRowsThreads;
    constexpr int RB = generic_rows(N);
    constexpr int R = fft_radix(N, 0);
    constexpr int BPR = N / R;
    constexpr int NB = RB * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
    static_assert(fft_npass(N) >= 2, "rows of at least 32 points");
    extern __shared__ float4 smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);

    for (int64_t blk = blockIdx.x; blk * RB < S; blk += gridDim.x) {
        const int64_t s0 = blk * RB;
        const int rows = (int)(S - s0 < RB ? S - s0 : RB);
        // pass 0: global -> registers -> shared (NS = 1, padded store)
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int b = threadIdx.x + k * NT;
            if (NB % NT != 0 && b >= NB) continue;
            const int row = b / BPR, j = b % BPR;
            float2 v[R];
            const float2* src = y + (s0 + row) * N + j;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = row < rows ? __ldcg(src + r * BPR) : make_float2(0.f, 0.f);
            dft<R>(v);
            pass_store<N, R, 1>(buf, row, j, v);
        }
        __syncthreads();
        // passes 1.. in shared memory; the last stores Y (its loads are fenced
        // by the pass's own barrier before the next block's pass 0 stores)
        fft_block<N, RB, NT, 1>(buf, tw, Y + s0 * N, rows);
    }
}

}  // namespace ppf
