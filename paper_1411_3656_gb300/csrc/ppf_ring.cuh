// Fused PPF kernel with a TMA-fed shared-memory ring (one CTA per SM).
//
// Each persistent CTA owns a contiguous band of output spectra and walks it in
// blocks of RB spectra.  Input rows arrive through 1-D bulk copies
// (cp.async.bulk, completion on an mbarrier per ring slot) into a ring of NCH
// chunks of RB rows, so every input sample is read from HBM exactly once: the
// T-1 rows a block shares with the next stay in the ring.  Per block:
//
//   1. wait for the chunk holding the block's newest rows (bounded wait);
//   2. FIR (Section 2, Eq. 1): each thread owns channel pairs (2p, 2p+1), or
//      single channels, keeps their coefficients in registers and produces RBT
//      consecutive spectra from RBT+T-1 ring rows (register blocking: each
//      shared-memory read feeds up to RBT multiply-adds per channel);
//   3. refill the ring slot the block no longer needs;
//   4. FFT of the RB filtered rows with Stockham radix-16 passes ping-ponging
//      between two shared buffers (or in place in one); the last pass stores
//      the spectra to global memory (coalesced, streaming).
// Filtered data never leaves the chip.
#pragma once

#include <type_traits>

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"

namespace ppf {

template <int N_, int T_, class In_, int NT_, int RB_, int NCH_, int MINB_ = 1, int CPT_ = 2, class OT_ = float2,
          int R0_ = 16, int NBUF_ = 2>
struct RingCfg {
    using OT = OT_;  // output bin: float2 (complex64) or BinF16
    // radix of the FFT's first pass (8 or 16): 8 splits N = 1024 as 8 x 16 x 8
    // instead of 16 x 16 x 4, evening out the butterflies per thread
    static constexpr int R0 = R0_;
    static constexpr int N = N_, T = T_, NT = NT_, RB = RB_, NCH = NCH_, MINB = MINB_;
    // FIR channels per thread: 2 (a pair, one 2-sample load per row, scalar
    // FMAs) or 1 (one channel, coefficients duplicated as (h, h) so that one
    // packed f32x2 FMA updates a complex accumulator)
    static constexpr int CPT = CPT_;
    using In = In_;
    using raw = typename In::raw;
    using coef_t = typename Coef<In>::type;
    static constexpr int BPS = In::bytes;
    // row stride: room for the first pass's padding (N/R0 slots)
    static constexpr int RS = R0 == 16 ? fft_row_stride(N) : N + N / 8;
    static constexpr int UNITS = N / CPT;                     // FIR work units per row
    static constexpr int G = UNITS > NT ? UNITS / NT : 1;     // units per thread
    static constexpr int RG = UNITS >= NT ? 1 : NT / UNITS;   // row groups
    static constexpr int RBT = RB / RG;                       // spectra per thread per block
    static constexpr int KO = T >= 2 ? (T - 2) / RB + 1 : 0;  // chunks beyond the block's first
    static constexpr int RING_ROWS = NCH * RB;
    static constexpr int CHUNK_BYTES = RB * N * BPS;
    static constexpr int RING_BYTES = NCH * CHUNK_BYTES;
    static constexpr int BUF_SLOTS = RB * RS;
    // FFT buffers: 2 (the passes ping-pong, one barrier per pass) or 1 (every
    // pass in place: loads, barrier, stores, barrier), which frees room for a
    // deeper ring or more spectra per block
    static constexpr int NBUF = NBUF_;
    static constexpr int FFT_BYTES = NBUF * BUF_SLOTS * 8;
    static constexpr int SMEM = RING_BYTES + FFT_BYTES + NCH * 8;
    static_assert(N >= 64, "ring kernel handles N >= 64");
    static_assert(CPT == 1 || CPT == 2, "one channel or a pair per thread");
    static_assert(UNITS % NT == 0 || NT % UNITS == 0, "FIR units must tile the threads");
    static_assert(RB % RG == 0 && RBT >= 1, "rows per block must split over row groups");
    static_assert(NCH >= KO + 2, "ring must hold a block's window plus one chunk in flight");
    static_assert(CHUNK_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
    static_assert(NBUF == 1 || NBUF == 2, "one or two FFT buffers");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

// One Stockham pass from `in` to `out` (or to global memory for the last pass);
// rows of RS slots, first-pass radix R0.
template <int N, int RB, int NT, int R0, int RS, int P, class OT>
__device__ __forceinline__ void fft_pass_pp(const float2* in, float2* out, const PassTwiddlesR<N, NT, R0>& tw,
                                            OT* __restrict__ Yb, int rows)
{
    constexpr int R = fft_radix_r(N, P, R0);
    constexpr int NS = fft_ns_r(N, P, R0);
    constexpr bool LAST = (P == fft_npass_r(N, R0) - 1);
    constexpr int IN_NS = P == 0 ? 0 : fft_ns_r(N, P - 1, R0);
    constexpr int IN_R = P == 0 ? 1 : fft_radix_r(N, P - 1, R0);
    constexpr int BPR = N / R;
    constexpr int NB = RB * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            const int row = b / BPR, j = b % BPR;
            float2 v[R];
            const int bx = row * RS + (IN_NS == 0 ? j : pad_slot<IN_NS, IN_R>(j));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ix = bx + r * (IN_NS == 0 ? N / R : pad_stride<IN_NS, IN_R, N / R>());
                v[r] = PPF_INBOUNDS(ix < RB * RS) ? in[ix] : make_float2(0.f, 0.f);
            }
            if constexpr (P > 0) apply_twiddles<R>(tw.template get<P>(), v);
            dft<R>(v);
            if constexpr (LAST) {
                if (row < rows) {
                    OT* o = Yb + (int64_t)row * N + j;
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        if (PPF_INBOUNDS(j + q * NS < N)) st_bin(o + q * NS, v[q]);
                }
            } else {
                // the R outputs lie in one padding group: one slot computation
                const int ox = row * RS + pad_slot<NS, R>((j / NS) * NS * R + (j % NS));
#pragma unroll
                for (int q = 0; q < R; ++q)
                    if (PPF_INBOUNDS(ox + q * NS < RB * RS)) out[ox + q * NS] = v[q];
            }
        }
    }
    if constexpr (!LAST) __syncthreads();
}

template <int N, int RB, int NT, int R0, int RS, int P = 0, class OT>
__device__ __forceinline__ void fft_rows_pp(float2* a, float2* b, const PassTwiddlesR<N, NT, R0>& tw,
                                            OT* __restrict__ Yb, int rows)
{
    if constexpr (P < fft_npass_r(N, R0)) {
        fft_pass_pp<N, RB, NT, R0, RS, P>(a, b, tw, Yb, rows);
        fft_rows_pp<N, RB, NT, R0, RS, P + 1>(b, a, tw, Yb, rows);
    }
}

// One Stockham pass in place (single FFT buffer): every thread first loads the
// inputs of its butterflies, the CTA synchronises so that no element is
// overwritten before every thread has read it, then the outputs go back to
// the same rows (or, in the last pass, to global memory).  The barrier after
// the last pass's loads also frees the buffer for the next block's FIR; the
// caller's `after_last_read` runs right after it.
template <int N, int RB, int NT, int R0, int RS, int P, int PD, class OT, class F>
__device__ __forceinline__ void fft_pass_ip(float2* buf, const PassTwiddlesR<N, NT, R0>& tw, OT* __restrict__ Yb,
                                            int rows, F&& after_last_read)
{
    constexpr int R = fft_radix_r(N, P, R0);
    constexpr int NS = fft_ns_r(N, P, R0);
    constexpr bool LAST = (P == fft_npass_r(N, R0) - 1);
    constexpr int IN_NS = P == 0 ? 0 : fft_ns_r(N, P - 1, R0);
    constexpr int IN_R = P == 0 ? 1 : fft_radix_r(N, P - 1, R0);
    constexpr int BPR = N / R;
    constexpr int NB = RB * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            const int row = b / BPR, j = b % BPR;
            const int bx = row * RS + (IN_NS == 0 ? j : pad_slot<IN_NS, IN_R, PD>(j));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ix = bx + r * (IN_NS == 0 ? N / R : pad_stride<IN_NS, IN_R, N / R, PD>());
                v[k][r] = PPF_INBOUNDS(ix < RB * RS) ? buf[ix] : make_float2(0.f, 0.f);
            }
        }
    }
    __syncthreads();
    if constexpr (LAST) after_last_read();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT == 0 || b < NB) {
            const int row = b / BPR, j = b % BPR;
            if constexpr (P > 0) apply_twiddles<R>(tw.template get<P>(), v[k]);
            dft<R>(v[k]);
            if constexpr (LAST) {
                if (row < rows) {
                    OT* o = Yb + (int64_t)row * N + j;
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        if (PPF_INBOUNDS(j + q * NS < N)) st_bin(o + q * NS, v[k][q]);
                }
            } else {
                const int ox = row * RS + pad_slot<NS, R, PD>((j / NS) * NS * R + (j % NS));
#pragma unroll
                for (int q = 0; q < R; ++q)
                    if (PPF_INBOUNDS(ox + q * NS < RB * RS)) buf[ox + q * NS] = v[k][q];
            }
        }
    }
    if constexpr (!LAST) __syncthreads();
}

template <int N, int RB, int NT, int R0, int RS, int P = 0, int PD = 1, class OT, class F>
__device__ __forceinline__ void fft_rows_ip(float2* buf, const PassTwiddlesR<N, NT, R0>& tw, OT* __restrict__ Yb,
                                            int rows, F&& after_last_read)
{
    if constexpr (P < fft_npass_r(N, R0)) {
        fft_pass_ip<N, RB, NT, R0, RS, P, PD>(buf, tw, Yb, rows, after_last_read);
        fft_rows_ip<N, RB, NT, R0, RS, P + 1, PD>(buf, tw, Yb, rows, after_last_read);
    }
}

template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB)
ppf_ring_kernel(const PpfWork wl, const float2* __restrict__ tw, int* __restrict__ err)
{
    constexpr int N = C::N, T = C::T, NT = C::NT, RB = C::RB, NCH = C::NCH, RS = C::RS;
    constexpr int G = C::G, RBT = C::RBT, BPS = C::BPS, RING_ROWS = C::RING_ROWS;
    using PV = typename Pair<typename C::In>::vec;
    using raw = typename C::raw;
    using coef_t = typename C::coef_t;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float2* bufA = reinterpret_cast<float2*>(smem + C::RING_BYTES);
    float2* bufB = C::NBUF == 2 ? bufA + C::BUF_SLOTS : bufA;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES + C::FFT_BYTES);

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < NCH; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t policy = l2_evict_first_policy();

    // Thread -> (row group, FIR units: channel pairs or single channels).
    const int rg = C::UNITS >= NT ? 0 : tid / C::UNITS;
    const int pbase = C::UNITS >= NT ? tid : tid % C::UNITS;
    const int i0 = rg * RBT;
    PassTwiddlesR<N, NT, C::R0> twr;
    twr.load(tw);

    // Chunks this CTA issued in earlier bands: ring slots and mbarrier phases
    // continue across bands (every chunk of a band is waited for in that band).
    int cbase = 0;
    // Blocks this CTA has filtered.  With two buffers and an odd number of FFT
    // passes the last pass reads the buffer the FIR wrote, so the FIR alternates
    // between the two buffers from block to block and never writes the one the
    // previous block's last pass may still be reading; no barrier is needed
    // between them.
    constexpr bool ODD = C::NBUF == 2 && fft_npass_r(N, C::R0) % 2 == 1;
    int bcount = 0;
    const int n_items = work_items(wl);
    for (int it = blockIdx.x;; it += gridDim.x) {
        PpfJob job;
        int64_t blo, bhi;
        if (wl.items == nullptr) {
            if (it != (int)blockIdx.x) break;
            job = wl.one;
            const int64_t nblk = (job.S + RB - 1) / RB;
            blo = nblk * blockIdx.x / gridDim.x;
            bhi = nblk * (blockIdx.x + 1) / gridDim.x;
        } else {
            if (it >= n_items) break;
            const PpfItem item = wl.items[it];
            job = wl.jobs[item.job];
            blo = item.blo;
            bhi = item.bhi;
        }
        if (blo >= bhi) continue;
        const raw* __restrict__ x = static_cast<const raw*>(job.x);
        const coef_t* __restrict__ h = static_cast<const coef_t*>(job.h);
        typename C::OT* __restrict__ Y = reinterpret_cast<typename C::OT*>(job.Y);
        const int64_t S = job.S;
        const int nb = (int)(bhi - blo);
        const int64_t s_lo = blo * RB;
        const int64_t s_hi = S < bhi * RB ? S : bhi * RB;
        const int64_t in_end = s_hi + T - 1;  // input rows the band reads: [s_lo, in_end)
        const int nchunks = (int)((in_end - s_lo + RB - 1) / RB);

        int issued = 0;  // chunks of this band issued so far (meaningful in thread 0)
        auto issue = [&](int k) {
            const int64_t r0 = s_lo + (int64_t)k * RB;
            const int64_t rows = in_end - r0 < RB ? in_end - r0 : RB;
            const uint32_t bytes = (uint32_t)(rows * N * BPS);
            const int slot = (cbase + k) % NCH;
            // (a copy the checked build refuses completes the phase with no bytes)
            const bool ok = PPF_INBOUNDS((size_t)slot * C::CHUNK_BYTES + bytes <= (size_t)C::RING_BYTES);
            mbar_arrive_expect_tx(&bars[slot], ok ? bytes : 0u);
            if (ok) tma_load_1d(ring + slot * C::CHUNK_BYTES, x + r0 * N, bytes, &bars[slot], policy);
        };
        if (tid == 0) {
            const int first = nchunks < NCH ? nchunks : NCH;
            for (int k = 0; k < first; ++k) issue(k);
            issued = first;
        }

        // coefficients of this thread's channels, in FP32 registers (CPT = 1
        // keeps each as the pair (h, h))
        // FP16 and int8 input with channel pairs keep each tap's coefficients
        // as one FP16 pair and multiply FP16 samples directly (int8 turned
        // into FP16 exactly: fma_f16_pair, f16_pairs)
        constexpr bool MIX = C::CPT == 2 && !std::is_same<typename C::In, InC32>::value;
        // complex64 channel pairs with G*T <= 32 (at most 128 coefficient
        // registers) and at least 4 spectra per thread keep each coefficient
        // as (h, h) so that one packed FMA updates a complex accumulator (half
        // the FIR instructions, bitwise the scalar result; measured slower
        // with fewer spectra per thread, where the loads dominate)
        constexpr bool PK = C::CPT == 2 && !MIX && G * T <= 32 && RBT >= 4;
        float hr[C::CPT == 2 && !MIX && !PK ? G : 1][C::CPT == 2 && !MIX && !PK ? T : 1][2];
        float2 hp[PK ? G : 1][PK ? T : 1][2];
        uint32_t hq[MIX ? G : 1][MIX ? T : 1];
        float2 hh[C::CPT == 1 ? G : 1][C::CPT == 1 ? T : 1];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int c = C::CPT * (pbase + g * NT);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                if constexpr (MIX) {
                    hq[g][t] = *reinterpret_cast<const uint32_t*>(h + t * N + c);
                } else if constexpr (PK) {
                    const float v0 = coef_f(h[t * N + c]), v1 = coef_f(h[t * N + c + 1]);
                    hp[g][t][0] = make_float2(v0, v0);
                    hp[g][t][1] = make_float2(v1, v1);
                } else if constexpr (C::CPT == 2) {
                    hr[g][t][0] = coef_f(h[t * N + c]);
                    hr[g][t][1] = coef_f(h[t * N + c + 1]);
                } else {
                    const float v = coef_f(h[t * N + c]);
                    hh[g][t] = make_float2(v, v);
                }
            }
        }

        int waited = 0;                    // chunks of this band every thread has waited for
        int rrb = (cbase % NCH) * RB;      // ring row of the block's first input row
        bool failed = false;
        for (int b = 0; b < nb; ++b) {
            // 1. the block needs chunks b .. b+KO; every thread waits itself (a
            //    failure spreads over the CTA at the barrier after the FIR)
            const int need = (b + C::KO < nchunks ? b + C::KO : nchunks - 1) + 1;
            for (; waited < need && !failed; ++waited) {
                const int gk = cbase + waited;
                if (!mbar_wait_bounded(&bars[gk % NCH], (uint32_t)((gk / NCH) & 1))) {
                    failed = true;
                    break;  // this chunk stays "not waited for": the drain below waits for it
                }
            }
            float2* const fb = (ODD && (bcount & 1)) ? bufB : bufA;  // FIR output, FFT pass 0 input
            float2* const ob = (ODD && (bcount & 1)) ? bufA : bufB;

            // 2. FIR over the ring (Eq. 1), RBT spectra x CPT channels per unit.
            //    With one row group the window starts at a chunk boundary, so
            //    row u lies in the window's chunk u / RB at row u % RB: the
            //    chunk bases are computed once per block and every load is a
            //    base plus a compile-time offset (no per-row wrap test).
            constexpr int NW = (RBT + T - 2) / RB + 1;  // chunks the window spans
            uint32_t cbase_off[C::RG == 1 ? NW : 1];
            if constexpr (C::RG == 1) {
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    int sl = rrb / RB + w;
                    sl -= sl >= NCH ? NCH : 0;
                    cbase_off[w] = (uint32_t)(sl * C::CHUNK_BYTES);
                }
            }
            // byte offset in the ring of window row u for channel (pair) c
            auto ring_off = [&](int u, int c) -> size_t {
                if constexpr (C::RG == 1) {
                    return (size_t)cbase_off[u / RB] + ((size_t)(u % RB) * N + c) * BPS;
                } else {
                    int rr = rrb + i0 + u;
                    rr = rr >= RING_ROWS ? rr - RING_ROWS : rr;
                    return ((size_t)rr * N + c) * BPS;
                }
            };
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int c = C::CPT * (pbase + g * NT);
                if constexpr (C::CPT == 2) {
                    float2 a0[RBT], a1[RBT];
#pragma unroll
                    for (int i = 0; i < RBT; ++i) {
                        a0[i] = make_float2(0.f, 0.f);
                        a1[i] = make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < RBT + T - 1; ++u) {
                        const size_t ro = ring_off(u, c);
                        const PV pv = PPF_INBOUNDS(ro + sizeof(PV) <= (size_t)C::RING_BYTES)
                                          ? *reinterpret_cast<const PV*>(ring + ro)
                                          : PV{};
                        if constexpr (MIX) {
                            const uint2 xq = f16_pairs(pv);
#pragma unroll
                            for (int i = 0; i < RBT; ++i) {
                                const int t = u - i;
                                if (t >= 0 && t < T) fma_f16_pair(hq[g][t], xq, a0[i], a1[i]);
                            }
                        } else if constexpr (PK) {
                            float2 v0, v1;
                            Pair<typename C::In>::split(pv, v0, v1);
#pragma unroll
                            for (int i = 0; i < RBT; ++i) {
                                const int t = u - i;
                                if (t >= 0 && t < T) {
                                    a0[i] = __ffma2_rn(hp[g][t][0], v0, a0[i]);
                                    a1[i] = __ffma2_rn(hp[g][t][1], v1, a1[i]);
                                }
                            }
                        } else {
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
                    }
#pragma unroll
                    for (int i = 0; i < RBT; ++i)
                        if (PPF_INBOUNDS((i0 + i) * RS + c + 2 <= C::BUF_SLOTS))
                            *reinterpret_cast<float4*>(fb + (i0 + i) * RS + c) =
                                make_float4(a0[i].x, a0[i].y, a1[i].x, a1[i].y);
                } else {
                    float2 a[RBT];
#pragma unroll
                    for (int i = 0; i < RBT; ++i) a[i] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < RBT + T - 1; ++u) {
                        const size_t ro = ring_off(u, c);
                        const float2 v = PPF_INBOUNDS(ro + sizeof(raw) <= (size_t)C::RING_BYTES)
                                             ? decode(*reinterpret_cast<const raw*>(ring + ro))
                                             : make_float2(0.f, 0.f);
#pragma unroll
                        for (int i = 0; i < RBT; ++i) {
                            const int t = u - i;
                            if (t >= 0 && t < T) a[i] = __ffma2_rn(hh[g][t], v, a[i]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < RBT; ++i)
                        if (PPF_INBOUNDS((i0 + i) * RS + c + 1 <= C::BUF_SLOTS)) fb[(i0 + i) * RS + c] = a[i];
                }
            }
            if (__syncthreads_or(failed)) {
                failed = true;
                break;
            }

            // 3. chunk b is no longer needed: refill its slot
            if (tid == 0 && issued < nchunks && issued == b + NCH) {
                issue(issued);
                ++issued;
            }
            rrb += RB;
            rrb = rrb >= RING_ROWS ? rrb - RING_ROWS : rrb;

            // 4. FFT of the RB rows; the last pass stores the spectra
            const int64_t s0 = s_lo + (int64_t)b * RB;
            const int rows = (int)(s_hi - s0 < RB ? s_hi - s0 : RB);
            if constexpr (C::NBUF == 2) fft_rows_pp<N, RB, NT, C::R0, RS>(fb, ob, twr, Y + s0 * N, rows);
            else fft_rows_ip<N, RB, NT, C::R0, RS>(fb, twr, Y + s0 * N, rows, [] {});
            ++bcount;
        }
        if (failed) {
            if (tid == 0) {
                // let the copies still in flight land before the CTA exits
                for (int k = waited; k < issued; ++k) {
                    const int gk = cbase + k;
                    mbar_wait_bounded(&bars[gk % NCH], (uint32_t)((gk / NCH) & 1), kWaitLimitNs / 4);
                }
                atomicExch(err, 1);
            }
            return;
        }
        cbase += nchunks;
    }
}

}  // namespace ppf
