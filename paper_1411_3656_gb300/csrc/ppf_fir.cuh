// FIR-only kernel (the first of the paper's two passes, Section 3: a FIR
// kernel writes the filtered spectra, a library FFT transforms them): the
// filtered rows y[s][c] = sum_t h[t*N+c] * x[(s+t)*N+c] (Section 2, Eq. 1)
// go to global memory.  Used by plans made with PPF_FLAG_FIR_ONLY (the
// test hook) and by the two-pass comparison.
//
// No FFT follows, so no CTA needs all N channels of a spectrum: CTA i takes
// channel slice i mod (N/NC) of time band i div (N/NC).  Its ring holds the
// slice of RB-row chunks (1-D bulk copies of each row's slice, every input
// byte read from HBM once per band), every thread filters a channel pair for
// RBT spectra with coefficients in registers and stores the pair of filtered
// bins as one 16-byte store (a warp writes 512 contiguous bytes of a row).
#pragma once

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"

namespace ppf {

template <int N_, int T_, int NC_, int NT_, int RB_, int NCH_>
struct FirCfg {
    static constexpr int N = N_, T = T_, NC = NC_, NT = NT_, RB = RB_, NCH = NCH_;
    static constexpr int SLICES = N / NC;
    static constexpr int UNITS = NC / 2;                      // channel pairs per slice
    static constexpr int G = UNITS > NT ? UNITS / NT : 1;
    static constexpr int RG = UNITS >= NT ? 1 : NT / UNITS;
    static constexpr int RBT = RB / RG;
    static constexpr int KO = T >= 2 ? (T - 2) / RB + 1 : 0;
    static constexpr int SEG_BYTES = NC * 8;
    static constexpr int CHUNK_BYTES = RB * SEG_BYTES;
    static constexpr int RING_BYTES = NCH * CHUNK_BYTES;
    static constexpr int RING_ROWS = NCH * RB;
    static constexpr int SMEM = RING_BYTES + NCH * 8;
    static_assert(N % NC == 0 && NC % 2 == 0 && SEG_BYTES % 16 == 0, "16-byte row slices");
    static_assert(UNITS % NT == 0 || NT % UNITS == 0, "FIR units must tile the threads");
    static_assert(RB % RG == 0 && RBT >= 1, "rows per block must split over row groups");
    static_assert(NCH >= KO + 2, "ring must hold a block's window plus one chunk in flight");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

template <class C>
__global__ void __launch_bounds__(C::NT, 1)
ppf_fir_kernel(const float2* __restrict__ x, const float* __restrict__ h, float2* __restrict__ y, int64_t S,
               int* __restrict__ err)
{
    constexpr int N = C::N, T = C::T, NT = C::NT, RB = C::RB, NCH = C::NCH, NC = C::NC;
    constexpr int G = C::G, RBT = C::RBT, RING_ROWS = C::RING_ROWS;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < NCH; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t policy = l2_evict_first_policy();
    const int slice = (int)(blockIdx.x % C::SLICES);
    const int band = (int)(blockIdx.x / C::SLICES), nbands = (int)(gridDim.x / C::SLICES);
    const int64_t nblk = (S + RB - 1) / RB;
    const int64_t blo = nblk * band / nbands, bhi = nblk * (band + 1) / nbands;
    if (blo >= bhi) return;
    const int nb = (int)(bhi - blo);
    const int64_t s_lo = blo * RB;
    const int64_t s_hi = S < bhi * RB ? S : bhi * RB;
    const int64_t in_end = s_hi + T - 1;
    const int nchunks = (int)((in_end - s_lo + RB - 1) / RB);
    const int rg = C::UNITS >= NT ? 0 : tid / C::UNITS;
    const int pbase = C::UNITS >= NT ? tid : tid % C::UNITS;
    const int i0 = rg * RBT;

    int issued = 0;
    auto issue = [&](int k) {
        const int64_t r0 = s_lo + (int64_t)k * RB;
        const int nrows = (int)(in_end - r0 < RB ? in_end - r0 : RB);
        const int slot = k % NCH;
        const bool ok = PPF_INBOUNDS(slot * C::CHUNK_BYTES + nrows * C::SEG_BYTES <= C::RING_BYTES);
        mbar_arrive_expect_tx(&bars[slot], ok ? (uint32_t)(nrows * C::SEG_BYTES) : 0u);
        for (int q = 0; q < (ok ? nrows : 0); ++q)
            tma_load_1d(ring + slot * C::CHUNK_BYTES + q * C::SEG_BYTES, x + (r0 + q) * N + slice * NC,
                        (uint32_t)C::SEG_BYTES, &bars[slot], policy);
    };
    if (tid == 0) {
        const int first = nchunks < NCH ? nchunks : NCH;
        for (int k = 0; k < first; ++k) issue(k);
        issued = first;
    }

    // coefficients as (h, h) pairs when they fit 128 registers, else scalars
    constexpr bool PK = G * T <= 32 && RBT >= 4;
    float2 hp[PK ? G : 1][PK ? T : 1][2];
    float hr[PK ? 1 : G][PK ? 1 : T][2];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int c = slice * NC + 2 * (pbase + g * NT);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float v0 = h[t * N + c], v1 = h[t * N + c + 1];
            if constexpr (PK) {
                hp[g][t][0] = make_float2(v0, v0);
                hp[g][t][1] = make_float2(v1, v1);
            } else {
                hr[g][t][0] = v0;
                hr[g][t][1] = v1;
            }
        }
    }

    int waited = 0;
    int rrb = 0;
    bool failed = false;
    for (int b = 0; b < nb; ++b) {
        const int need = (b + C::KO < nchunks ? b + C::KO : nchunks - 1) + 1;
        for (; waited < need && !failed; ++waited) {
            if (!mbar_wait_bounded(&bars[waited % NCH], (uint32_t)((waited / NCH) & 1))) {
                failed = true;
                break;
            }
        }
        const int64_t s0 = s_lo + (int64_t)b * RB;
        if (!failed) {
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
                    const size_t ro = ((size_t)rr * NC + cl) * 8;
                    const float4 pv = PPF_INBOUNDS(ro + 16 <= (size_t)C::RING_BYTES)
                                          ? *reinterpret_cast<const float4*>(ring + ro)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float2 v0 = make_float2(pv.x, pv.y), v1 = make_float2(pv.z, pv.w);
#pragma unroll
                    for (int i = 0; i < RBT; ++i) {
                        const int t = u - i;
                        if (t >= 0 && t < T) {
                            if constexpr (PK) {
                                a0[i] = __ffma2_rn(hp[g][t][0], v0, a0[i]);
                                a1[i] = __ffma2_rn(hp[g][t][1], v1, a1[i]);
                            } else {
                                a0[i].x = fmaf(hr[g][t][0], v0.x, a0[i].x);
                                a0[i].y = fmaf(hr[g][t][0], v0.y, a0[i].y);
                                a1[i].x = fmaf(hr[g][t][1], v1.x, a1[i].x);
                                a1[i].y = fmaf(hr[g][t][1], v1.y, a1[i].y);
                            }
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < RBT; ++i) {
                    const int64_t s = s0 + i0 + i;
                    if (s < s_hi)
                        __stcs(reinterpret_cast<float4*>(y + s * N + slice * NC + cl),
                               make_float4(a0[i].x, a0[i].y, a1[i].x, a1[i].y));
                }
            }
        }
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        if (tid == 0 && issued < nchunks && issued == b + NCH) {
            issue(issued);
            ++issued;
        }
        rrb += RB;
        rrb = rrb >= RING_ROWS ? rrb - RING_ROWS : rrb;
    }
    if (failed && tid == 0) {
        for (int k = waited; k < issued; ++k)
            mbar_wait_bounded(&bars[k % NCH], (uint32_t)((k / NCH) & 1), kWaitLimitNs / 4);
        atomicExch(err, 1);
    }
}

}  // namespace ppf
