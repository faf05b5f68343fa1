// General fused PPF kernel: any supported N, runtime T (1..64), any input dtype.
//
// One CTA walks a contiguous band of row blocks.  For each block of RB output
// spectra it
//   1. filters (Section 2, Eq. 1): y[s][c] = sum_t h[t*N+c] * x[(s+t)*N+c],
//      two channels per thread, reading the input straight from global memory
//      (the T-1 halo rows of a block were read by the previous block of the
//      same CTA and come back from L1/L2, not HBM);
//   2. writes y into shared memory and transforms every row with the
//      Stockham passes of ppf_device.cuh, in place;
//   3. stores the spectra from the last pass, coalesced.
// Filtered data never leaves the chip.  This kernel also serves the FIR-only
// test hook (it then stores y instead of transforming it).
#pragma once

#include "ppf_device.cuh"

namespace ppf {

constexpr int kGenericThreads = 256;
__host__ __device__ constexpr int generic_rows(int N) { return N >= 4096 ? 1 : 4096 / N; }
__host__ __device__ constexpr int generic_smem_bytes(int N)
{
    return generic_rows(N) * fft_row_stride(N) * (int)sizeof(float2);
}

// One Stockham pass over RB rows held in `buf` (in place).  The last pass
// writes the spectra to global memory instead.
template <int N, int RB, int NT, int P, class OT>
__device__ __forceinline__ void fft_pass_block(float2* buf, const float2* __restrict__ tw,
                                               OT* __restrict__ Yb, int rows)
{
    constexpr int R = fft_radix(N, P);
    constexpr int NS = fft_ns(N, P);
    constexpr bool LAST = (P == fft_npass(N) - 1);
    constexpr int IN_NS = P == 0 ? 0 : fft_ns(N, P - 1);
    constexpr int IN_R = P == 0 ? 1 : fft_radix(N, P - 1);
    constexpr int BPR = N / R;
    constexpr int NB = RB * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) pass_load<N, R, IN_NS, IN_R>(buf, b / BPR, b % BPR, v[k]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            const int row = b / BPR, j = b % BPR;
            pass_twiddle<N, R, NS>(tw, j, v[k]);
            dft<R>(v[k]);
            if constexpr (LAST) {
                if (row < rows) {
                    OT* o = Yb + (int64_t)row * N + j;
#pragma unroll
                    for (int q = 0; q < R; ++q) st_bin(o + q * NS, v[k][q]);
                }
            } else {
                pass_store<N, R, NS>(buf, row, j, v[k]);
            }
        }
    }
    if constexpr (!LAST) __syncthreads();
}

template <int N, int RB, int NT, int P = 0, class OT>
__device__ __forceinline__ void fft_block(float2* buf, const float2* __restrict__ tw,
                                          OT* __restrict__ Yb, int rows)
{
    if constexpr (P < fft_npass(N)) {
        fft_pass_block<N, RB, NT, P>(buf, tw, Yb, rows);
        fft_block<N, RB, NT, P + 1>(buf, tw, Yb, rows);
    }
}

template <int N, class In, class Cf = typename Coef<In>::type, class OT = float2>
__global__ void __launch_bounds__(kGenericThreads)
ppf_generic_kernel(const typename In::raw* __restrict__ x,
                   const Cf* __restrict__ h,
                   const float2* __restrict__ tw, OT* __restrict__ Y,
                   int T, int64_t S, int fir_only)
{
    constexpr int NT = kGenericThreads;
    constexpr int RB = generic_rows(N);
    constexpr int RS = fft_row_stride(N);
    constexpr int HALF = N / 2;
    extern __shared__ float4 smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    using PV = typename Pair<In>::vec;

    const int64_t nblk = (S + RB - 1) / RB;
    const int64_t b0 = nblk * blockIdx.x / gridDim.x;
    const int64_t b1 = nblk * (blockIdx.x + 1) / gridDim.x;

    for (int64_t b = b0; b < b1; ++b) {
        const int64_t s0 = b * RB;
        const int rows = (int)(S - s0 < RB ? S - s0 : RB);
        for (int i = threadIdx.x; i < RB * HALF; i += NT) {
            const int row = i / HALF;
            const int c = 2 * (i % HALF);
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
            if (row < rows) {
                const typename In::raw* xp = x + (s0 + row) * (int64_t)N + c;
                for (int t = 0; t < T; ++t) {
                    const PV pv = __ldg(reinterpret_cast<const PV*>(xp + (int64_t)t * N));
                    float2 v0, v1;
                    Pair<In>::split(pv, v0, v1);
                    const float h0 = coef_f(h[t * N + c]);
                    const float h1 = coef_f(h[t * N + c + 1]);
                    a0.x = fmaf(h0, v0.x, a0.x);
                    a0.y = fmaf(h0, v0.y, a0.y);
                    a1.x = fmaf(h1, v1.x, a1.x);
                    a1.y = fmaf(h1, v1.y, a1.y);
                }
            }
            if (fir_only) {
                if (row < rows) {
                    float2* o = reinterpret_cast<float2*>(Y) + (s0 + row) * (int64_t)N + c;
                    o[0] = a0;
                    o[1] = a1;
                }
            } else {
                if (PPF_INBOUNDS(row * RS + c + 2 <= RB * RS))
                    *reinterpret_cast<float4*>(buf + row * RS + c) = make_float4(a0.x, a0.y, a1.x, a1.y);
            }
        }
        if (fir_only) continue;
        __syncthreads();
        fft_block<N, RB, NT>(buf, tw, Y + s0 * N, rows);
    }
}

}  // namespace ppf
