// Fused PPF kernel for large N*T: groups of CTAs pass filtered rows through L2.
//
// When the T-row FIR window of all N channels does not fit one SM, a group of
// P co-resident CTAs shares each band of spectra.  CTA p of a group
//   * filters the contiguous channel slice [p*N/P, (p+1)*N/P) (Section 2,
//     Eq. 1) from a shared-memory ring fed by 1-D bulk copies, so every input
//     sample is read from HBM once;
//   * writes the filtered slice of each row into the group's exchange rows in
//     global memory (a few hundred KiB per group, so they stay in the 129 MB
//     L2 and never reach HBM), then signals the group's FIR counter;
//   * takes full N-point FFTs (Stockham passes in shared memory, as in the
//     ring kernel) of the rows i of the block with i mod P == p, reading them
//     back from L2 once every CTA's slice is there, stores the spectra as
//     contiguous rows and signals the group's FFT counter.
// The exchange rows are double-buffered and the loop is software-pipelined:
// block b is filtered while block b-1 is transformed.  The grid is launched
// cooperatively so every CTA of a group is resident; every wait on a counter
// is bounded by %globaltimer and records PPF_ERR_TIMEOUT instead of hanging.
#pragma once

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"
#include "ppf_ring.cuh"

namespace ppf {

template <int N_, int T_, class In_, int P_, int NT_, int RB_, int NCH_>
struct SplitCfg {
    static constexpr int N = N_, T = T_, P = P_, NT = NT_, RB = RB_, NCH = NCH_;
    using In = In_;
    using raw = typename In::raw;
    using coef_t = typename Coef<In>::type;
    static constexpr int BPS = In::bytes;
    static constexpr int NC = N / P;  // channels filtered per CTA (contiguous)
    static constexpr int PAIRS = NC / 2;
    static constexpr int G = PAIRS > NT ? PAIRS / NT : 1;
    static constexpr int RG = PAIRS >= NT ? 1 : NT / PAIRS;
    static constexpr int RBT = RB / RG;
    static constexpr int KO = T >= 2 ? (T - 2) / RB + 1 : 0;
    static constexpr int RING_ROWS = NCH * RB;
    static constexpr int ROW_BYTES = NC * BPS;  // one row of the CTA's slice
    static constexpr int CHUNK_BYTES = RB * ROW_BYTES;
    static constexpr int RING_BYTES = NCH * CHUNK_BYTES;
    static constexpr int RF = (RB + P - 1) / P;  // rows each CTA transforms per block (at most)
    static constexpr int RS = fft_row_stride(N);
    static constexpr int FFT_BYTES = 2 * RF * RS * 8;
    static constexpr int SMEM = RING_BYTES + FFT_BYTES + NCH * 8;
    static constexpr size_t XROWS = 2 * RB;  // exchange rows per group (two blocks)
    static_assert(N % P == 0 && NC % 2 == 0 && ROW_BYTES % 16 == 0, "slices of 16-byte multiples");
    static_assert(RB % RG == 0 && RBT >= 1, "rows per block must split over row groups");
    static_assert(NCH >= KO + 2, "ring must hold a block's window plus one chunk in flight");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *ctr >= target (bounded by kWaitLimitNs).
__device__ __forceinline__ bool wait_counter(const int* ctr, int target)
{
    if (ld_acquire_gpu(ctr) >= target) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 1;; ++i) {
        __nanosleep(64);
        if (ld_acquire_gpu(ctr) >= target) return true;
        if ((i & 63u) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
}

// Pass 0 of the FFTs of up to RF exchange rows (row k at xr + k*row_step*N),
// reading the inputs from global memory (L2; ld.global.cg bypasses the
// non-coherent L1) and writing the padded pass-0 output rows of `out`.
template <int N, int NT, int RF>
__device__ __forceinline__ void fft_first_pass_global(const float2* __restrict__ xr, int row_step, int nrows,
                                                      float2* out)
{
    constexpr int R = fft_radix(N, 0);
    constexpr int NS = fft_ns(N, 0);
    constexpr int BPR = N / R;
    constexpr int NB = RF * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
    constexpr bool LAST = fft_npass(N) == 1;
    static_assert(!LAST, "split kernel needs N >= 32");
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT != 0 && b >= NB) continue;
        const int row = b / BPR, j = b % BPR;
        if (row >= nrows) continue;
        const float2* src = xr + (size_t)row * row_step * N;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = __ldcg(src + j + r * (N / R));
        dft<R>(v);
        pass_store<N, R, NS>(out, row, j, v);
    }
    __syncthreads();
}

// Passes 1.. of RF rows held in shared memory (pass 0 already done into `a`);
// local row k is spectrum s0 + first + k*step.  Rows k >= nrows are skipped.
template <int N, int RF, int NT, int PP>
__device__ __forceinline__ void split_pass(const float2* in, float2* out, const PassTwiddles<N, NT>& tw,
                                           float2* __restrict__ Y, int64_t s0, int first, int step, int nrows)
{
    constexpr int R = fft_radix(N, PP);
    constexpr int NS = fft_ns(N, PP);
    constexpr bool LAST = (PP == fft_npass(N) - 1);
    constexpr int IN_NS = fft_ns(N, PP - 1);
    constexpr int IN_R = fft_radix(N, PP - 1);
    constexpr int BPR = N / R;
    constexpr int NB = RF * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT != 0 && b >= NB) continue;
        const int row = b / BPR, j = b % BPR;
        if (row >= nrows) continue;
        float2 v[R];
        pass_load<N, R, IN_NS, IN_R>(in, row, j, v);
        apply_twiddles<R>(tw.template get<PP>(), v);
        dft<R>(v);
        if constexpr (LAST) {
            float2* o = Y + (s0 + first + (int64_t)row * step) * N + j;
#pragma unroll
            for (int q = 0; q < R; ++q) __stcs(o + q * NS, v[q]);
        } else {
            pass_store<N, R, NS>(out, row, j, v);
        }
    }
    if constexpr (!LAST) __syncthreads();
}

template <int N, int RF, int NT, int PP = 1>
__device__ __forceinline__ void fft_rows_rest(float2* a, float2* b, const PassTwiddles<N, NT>& tw,
                                              float2* __restrict__ Y, int64_t s0, int first, int step, int nrows)
{
    if constexpr (PP < fft_npass(N)) {
        split_pass<N, RF, NT, PP>(a, b, tw, Y, s0, first, step, nrows);
        fft_rows_rest<N, RF, NT, PP + 1>(b, a, tw, Y, s0, first, step, nrows);
    }
}

template <class C>
__global__ void __launch_bounds__(C::NT, 1)
ppf_split_kernel(const PpfWork wl, const float2* __restrict__ tw, float2* __restrict__ xbuf, int* __restrict__ ctr,
                 int* __restrict__ err)
{
    constexpr int N = C::N, T = C::T, NT = C::NT, RB = C::RB, NCH = C::NCH, P = C::P, NC = C::NC, RF = C::RF;
    constexpr int G = C::G, RBT = C::RBT, BPS = C::BPS, RING_ROWS = C::RING_ROWS, RS = C::RS;
    using PV = typename Pair<typename C::In>::vec;
    using raw = typename C::raw;
    using coef_t = typename C::coef_t;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float2* fa = reinterpret_cast<float2*>(smem + C::RING_BYTES);
    float2* fb = fa + RF * RS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES + C::FFT_BYTES);

    const int tid = threadIdx.x;
    const int p = blockIdx.x % P, grp = blockIdx.x / P, ngrp = gridDim.x / P;
    float2* xg = xbuf + (size_t)grp * C::XROWS * N;  // this group's exchange rows
    // progress words of the group: fir_done[q] = FIR blocks CTA q has written,
    // fft_done[q] = blocks whose exchange rows CTA q has finished reading
    int* fir_done = ctr + 2 * P * grp;
    int* fft_done = fir_done + P;

    if (tid == 0) {
        for (int i = 0; i < NCH; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t policy = l2_evict_first_policy();

    const int rg = C::PAIRS >= NT ? 0 : tid / C::PAIRS;
    const int pbase = C::PAIRS >= NT ? tid : tid % C::PAIRS;
    const int i0 = rg * RBT;
    PassTwiddles<N, NT> twr;
    twr.load(tw);

    const PpfJob job = wl.one;
    const raw* __restrict__ x = static_cast<const raw*>(job.x);
    const coef_t* __restrict__ h = static_cast<const coef_t*>(job.h);
    float2* __restrict__ Y = job.Y;
    const int64_t S = job.S;
    const int64_t nblk = (S + RB - 1) / RB;
    const int64_t blo = nblk * grp / ngrp, bhi = nblk * (grp + 1) / ngrp;
    const int nb = (int)(bhi - blo);  // the same for every CTA of the group
    const int64_t s_lo = blo * RB;
    const int64_t s_hi = S < bhi * RB ? S : bhi * RB;
    const int64_t in_end = s_hi + T - 1;
    const int nchunks = nb > 0 ? (int)((in_end - s_lo + RB - 1) / RB) : 0;

    int issued = 0;
    auto issue = [&](int k) {
        const int64_t r0 = s_lo + (int64_t)k * RB;
        const int rows = (int)(in_end - r0 < RB ? in_end - r0 : RB);
        const int slot = k % NCH;
        mbar_arrive_expect_tx(&bars[slot], (uint32_t)(rows * C::ROW_BYTES));
        for (int r = 0; r < rows; ++r)
            tma_load_1d(ring + slot * C::CHUNK_BYTES + r * C::ROW_BYTES, x + (r0 + r) * N + p * NC,
                        (uint32_t)C::ROW_BYTES, &bars[slot], policy);
    };
    if (tid == 0) {
        const int first = nchunks < NCH ? nchunks : NCH;
        for (int k = 0; k < first; ++k) issue(k);
        issued = first;
    }

    float hr[G][T][2];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int c = p * NC + 2 * (pbase + g * NT);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            hr[g][t][0] = coef_f(h[t * N + c]);
            hr[g][t][1] = coef_f(h[t * N + c + 1]);
        }
    }

    int waited = 0, rrb = 0;
    bool failed = false;
    for (int b = 0; b <= nb; ++b) {
        if (b < nb) {
            // ---- FIR of block b on this CTA's channel slice
            bool ok = true;
            if (!failed) {
                const int need = (b + C::KO < nchunks ? b + C::KO : nchunks - 1) + 1;
                for (; waited < need; ++waited)
                    if (!mbar_wait_bounded(&bars[waited % NCH], (uint32_t)((waited / NCH) & 1))) {
                        ok = false;
                        break;
                    }
            }
            // exchange rows of parity b&1 were last read by the FFTs of block b-2:
            // thread q < P waits for CTA q of the group
            bool okw = true;
            if (tid < P && b >= 2 && !failed) okw = wait_counter(fft_done + tid, b - 1);
            if (__syncthreads_or(!ok || !okw)) failed = true;
            float2* xo = xg + (size_t)(b & 1) * RB * N;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int cl = 2 * (pbase + g * NT);
                float2 a0[RBT], a1[RBT];
#pragma unroll
                for (int i = 0; i < RBT; ++i) {
                    a0[i] = make_float2(0.f, 0.f);
                    a1[i] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < RBT + T - 1; ++u) {
                    int rr = rrb + i0 + u;
                    rr = rr >= RING_ROWS ? rr - RING_ROWS : rr;
                    const PV pv = *reinterpret_cast<const PV*>(ring + ((size_t)rr * NC + cl) * BPS);
                    float2 v0, v1;
                    Pair<typename C::In>::split(pv, v0, v1);
#pragma unroll
                    for (int i = 0; i < RBT; ++i) {
                        const int t = u - i;
                        if (t >= 0 && t < T) {
                            a0[i].x = fmaf(hr[g][t][0], v0.x, a0[i].x);
                            a0[i].y = fmaf(hr[g][t][0], v0.y, a0[i].y);
                            a1[i].x = fmaf(hr[g][t][1], v1.x, a1[i].x);
                            a1[i].y = fmaf(hr[g][t][1], v1.y, a1[i].y);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < RBT; ++i)
                    __stcg(reinterpret_cast<float4*>(xo + (size_t)(i0 + i) * N + p * NC + cl),
                           make_float4(a0[i].x, a0[i].y, a1[i].x, a1[i].y));
            }
            __syncthreads();
            if (tid == 0) {
                // every thread's slice stores precede this release (barrier above)
                st_release_gpu(fir_done + p, b + 1);
                if (!failed && issued < nchunks && issued == b + NCH) {
                    issue(issued);
                    ++issued;
                }
            }
            rrb += RB;
            rrb = rrb >= RING_ROWS ? rrb - RING_ROWS : rrb;
        }
        if (b >= 1) {
            // ---- FFTs of block b-1: rows i with i mod P == p
            const int bp = b - 1;
            bool okw = true;
            if (tid < P && !failed) okw = wait_counter(fir_done + tid, b);  // every slice of block b-1
            if (__syncthreads_or(!okw)) failed = true;
            const int64_t s0 = s_lo + (int64_t)bp * RB;
            const int rows_blk = (int)(s_hi - s0 < RB ? s_hi - s0 : RB);
            // this CTA's rows of the block: i = p, p + P, ... (< rows_blk)
            const int mine = rows_blk > p ? (rows_blk - p + P - 1) / P : 0;
            const float2* xi = xg + (size_t)(bp & 1) * RB * N;
            fft_first_pass_global<N, NT, RF>(xi + (size_t)p * N, P, mine, fa);
            __syncthreads();
            if (tid == 0) st_release_gpu(fft_done + p, b);  // exchange rows of block b-1 read
            // remaining passes in shared memory; the last stores the spectra
            fft_rows_rest<N, RF, NT>(fa, fb, twr, Y, s0, p, P, mine);
            // the last pass read fa/fb: the next FFT (or FIR, which does not touch them) waits at a barrier
        }
    }
    if (failed && tid == 0) {
        for (int k = waited; k < issued; ++k)
            mbar_wait_bounded(&bars[k % NCH], (uint32_t)((k / NCH) & 1), kWaitLimitNs / 4);
        atomicExch(err, 1);
    }
}

}  // namespace ppf
