// Fused PPF kernel with warp-specialised FIR and FFT roles (one CTA per SM).
//
// The ring kernel runs the FIR (Section 2, Eq. 1) and the DFT of a block one
// after the other in the same warps, so the FMA-heavy FIR and the
// shared-memory-heavy, barrier-separated FFT passes never overlap: each alone
// keeps pace with HBM, together they take their sum.  Here the CTA's warps
// are split into two roles that work on consecutive blocks at the same time:
//
//   FIR warps (NF threads): wait for the ring rows of block b (1-D bulk
//     copies, one mbarrier per ring chunk, every input byte read from HBM
//     once), filter them with coefficients held in registers and write the
//     RB filtered rows into FFT buffer b mod 2; then refill the ring chunk the
//     block no longer needs;
//   FFT warps (NX threads): take the N-point DFTs of the rows in buffer
//     b mod 2 with Stockham passes in place and store the spectra.
//
// Block b+1 is filtered into the other buffer while block b is transformed.
// The hand-over uses named barriers: FULL[j] (FIR warps arrive after writing
// buffer j, FFT warps wait) and EMPTY[j] (FFT warps arrive after the last read
// of buffer j, FIR warps wait before writing it again).  Both roles walk the
// same blocks, so every barrier sees the same number of arrivals on each side,
// also when a bounded ring wait gives up (the FIR warps then skip the work but
// keep the barrier schedule).
#pragma once

#include <type_traits>

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"

namespace ppf {

// Named barrier ids of the warp-specialised kernels (0 is __syncthreads).
enum : int { kBarFir = 1, kBarFft = 2, kBarFull0 = 3, kBarEmpty0 = 5 };

template <int N_, int T_, class In_, int NF_, int NX_, int RB_, int NCH_, int CPT_ = 2, class OT_ = float2,
          int PD_ = 1, int RC_ = 16>
struct WsCfg {
    using OT = OT_;  // output bin: float2 (complex64) or BinF16
    using In = In_;
    using raw = typename In::raw;
    using coef_t = typename Coef<In>::type;
    static constexpr int N = N_, T = T_, NF = NF_, NX = NX_, RB = RB_, NCH = NCH_, CPT = CPT_, PD = PD_;
    // FFT passes of radix up to RC: 16, or 32 (1024 = 32 x 32, 512 = 32 x 16:
    // two passes instead of three, one shared-memory round trip less)
    static constexpr int RC = RC_;
    static constexpr int NT = NF + NX;
    static constexpr int BPS = In::bytes;
    // FFT buffer row stride: room for the first pass's padding (one slot per
    // RC elements, or per 2*RC with PD = 2)
    static constexpr int RS = N + (N / (RC * PD) > 2 ? N / (RC * PD) : 2);
    static_assert(RC == 16 || RC == 32, "pass radix cap 16 or 32");
    static_assert(RC == 16 || fft_radix_r(N, 0, RC, RC) == 32, "radix-32 plans start with a radix-32 pass");
    static constexpr int UNITS = N / CPT;                     // FIR work units per row
    static constexpr int G = UNITS > NF ? UNITS / NF : 1;     // units per FIR thread
    static constexpr int RG = UNITS >= NF ? 1 : NF / UNITS;   // row groups
    static constexpr int RBT = RB / RG;                       // spectra per FIR thread per block
    static constexpr int KO = T >= 2 ? (T - 2) / RB + 1 : 0;  // chunks beyond the block's first
    static constexpr int RING_ROWS = NCH * RB;
    static constexpr int CHUNK_BYTES = RB * N * BPS;
    static constexpr int RING_BYTES = NCH * CHUNK_BYTES;
    static constexpr int BUF_SLOTS = RB * RS;
    static constexpr int FFT_BYTES = 2 * BUF_SLOTS * 8;
    static constexpr int SMEM = RING_BYTES + FFT_BYTES + NCH * 8;
    static_assert(N >= 64, "warp-specialised kernel handles N >= 64");
    static_assert(NF % 32 == 0 && NX % 32 == 0 && NT <= 1024, "whole warps per role");
    static_assert(CPT == 1 || CPT == 2, "one channel or a pair per FIR thread");
    static_assert(UNITS % NF == 0 || NF % UNITS == 0, "FIR units must tile the FIR threads");
    static_assert(RB % RG == 0 && RBT >= 1, "rows per block must split over row groups");
    static_assert(NCH >= KO + 2, "ring must hold a block's window plus one chunk in flight");
    static_assert(CHUNK_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
    static_assert(RS % 2 == 0, "16-byte aligned channel pairs in the FFT buffer");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

// Twiddles of passes P.. for the butterflies an FFT thread (role index lt)
// takes in every block: butterfly lt + k*NX of a pass has j = (lt + k*NX) mod
// N/R, which cycles through J = max(1, (N/R)/NX) values, so J sets of R-1
// twiddles per pass are loaded once into registers.
template <int N, int NX, int RC = 16, int P = 1, bool ANY = (P < fft_npass_r(N, RC, RC))>
struct WsTwiddles {
    static constexpr int R = fft_radix_r(N, P, RC, RC);
    static constexpr int NS = fft_ns_r(N, P, RC, RC);
    static constexpr int BPR = N / R;
    static constexpr int J = NX >= BPR ? 1 : BPR / NX;
    static_assert(NX % BPR == 0 || BPR % NX == 0, "FFT threads must tile the butterflies of a row");
    float2 w[J][R - 1];
    WsTwiddles<N, NX, RC, P + 1> next;
    __device__ __forceinline__ void load(const float2* __restrict__ tw, int lt)
    {
        constexpr int step = N / (NS * R);
#pragma unroll
        for (int q = 0; q < J; ++q) {
            const int k = ((lt + q * NX) % BPR) % NS;
#pragma unroll
            for (int r = 1; r < R; ++r) w[q][r - 1] = __ldg(tw + k * r * step);
        }
        next.load(tw, lt);
    }
    template <int Q>
    __device__ __forceinline__ const float2* get(int q) const
    {
        if constexpr (Q == P) return w[q % J];
        else return next.template get<Q>(q);
    }
};
template <int N, int NX, int RC, int P>
struct WsTwiddles<N, NX, RC, P, false> {
    __device__ __forceinline__ void load(const float2* __restrict__, int) {}
    template <int Q>
    __device__ __forceinline__ const float2* get(int) const { return nullptr; }
};

// One Stockham pass in place over RB rows of `buf`, run by the NX FFT threads
// (role index lt): loads, FFT barrier, then twiddles, DFT and stores (the last
// pass stores the spectra to global memory and does not touch `buf` again,
// so it needs no barrier; `after_last_read` runs right after its loads).
template <int N, int RB, int NX, int RS, int PD, int RC, int P, class OT, class F>
__device__ __forceinline__ void ws_fft_pass(float2* buf, const WsTwiddles<N, NX, RC>& tw, OT* __restrict__ Yb,
                                            int rows, int lt, F&& after_last_read)
{
    constexpr int R = fft_radix_r(N, P, RC, RC);
    constexpr int NS = fft_ns_r(N, P, RC, RC);
    constexpr bool LAST = (P == fft_npass_r(N, RC, RC) - 1);
    constexpr int IN_NS = P == 0 ? 0 : fft_ns_r(N, P - 1, RC, RC);
    constexpr int IN_R = P == 0 ? 1 : fft_radix_r(N, P - 1, RC, RC);
    constexpr int BPR = N / R;
    constexpr int NB = RB * BPR;
    constexpr int PER = (NB + NX - 1) / NX;
    float2 v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = lt + k * NX;
        if (NB % NX == 0 || b < NB) {
            const int row = b / BPR, j = b % BPR;
            const int bx = row * RS + (IN_NS == 0 ? j : pad_slot<IN_NS, IN_R, PD>(j));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ix = bx + r * (IN_NS == 0 ? N / R : pad_stride<IN_NS, IN_R, N / R, PD>());
                v[k][r] = PPF_INBOUNDS(ix < RB * RS) ? buf[ix] : make_float2(0.f, 0.f);
            }
        }
    }
    if constexpr (LAST) after_last_read();
    else nbar_sync(kBarFft, NX);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = lt + k * NX;
        if (NB % NX == 0 || b < NB) {
            const int row = b / BPR, j = b % BPR;
            if constexpr (P > 0) apply_twiddles<R>(tw.template get<P>(k), v[k]);
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
    if constexpr (!LAST) nbar_sync(kBarFft, NX);
}

template <int N, int RB, int NX, int RS, int PD, int RC = 16, int P = 0, class OT, class F>
__device__ __forceinline__ void ws_fft_rows(float2* buf, const WsTwiddles<N, NX, RC>& tw, OT* __restrict__ Yb,
                                            int rows, int lt, F&& after_last_read)
{
    if constexpr (P < fft_npass_r(N, RC, RC)) {
        ws_fft_pass<N, RB, NX, RS, PD, RC, P>(buf, tw, Yb, rows, lt, after_last_read);
        ws_fft_rows<N, RB, NX, RS, PD, RC, P + 1>(buf, tw, Yb, rows, lt, after_last_read);
    }
}

// The band of blocks [blo, bhi) of work item `it` (or of the one job), as in
// the ring kernel; false when the CTA has no further item.
__device__ __forceinline__ bool ws_item(const PpfWork& wl, int it, int rb, PpfJob& job, int64_t& blo, int64_t& bhi)
{
    if (wl.items == nullptr) {
        if (it != (int)blockIdx.x) return false;
        job = wl.one;
        const int64_t nblk = (job.S + rb - 1) / rb;
        blo = nblk * blockIdx.x / gridDim.x;
        bhi = nblk * (blockIdx.x + 1) / gridDim.x;
        return true;
    }
    if (it >= work_items(wl)) return false;
    const PpfItem item = wl.items[it];
    job = wl.jobs[item.job];
    blo = item.blo;
    bhi = item.bhi;
    return true;
}

// ------------------------------------------------------------------ FIR role
template <class C>
__device__ __forceinline__ void ws_fir_role(const PpfWork& wl, unsigned char* ring, float2* X, uint64_t* bars,
                                            int* __restrict__ err)
{
    constexpr int N = C::N, T = C::T, NF = C::NF, RB = C::RB, NCH = C::NCH;
    constexpr int G = C::G, RBT = C::RBT, BPS = C::BPS, RING_ROWS = C::RING_ROWS, RS = C::RS;
    using PV = typename Pair<typename C::In>::vec;
    using raw = typename C::raw;
    using coef_t = typename C::coef_t;
    const int tid = threadIdx.x;
    const uint64_t policy = l2_evict_first_policy();
    const int rg = C::UNITS >= NF ? 0 : tid / C::UNITS;
    const int pbase = C::UNITS >= NF ? tid : tid % C::UNITS;
    const int i0 = rg * RBT;

    int cbase = 0;  // ring chunks issued in earlier items (slots and phases continue)
    int gb = 0;     // blocks this CTA has filtered (FFT buffer gb mod 2)
    bool failed = false;
    for (int it = blockIdx.x;; it += gridDim.x) {
        PpfJob job;
        int64_t blo, bhi;
        if (!ws_item(wl, it, RB, job, blo, bhi)) break;
        if (blo >= bhi) continue;
        const raw* __restrict__ x = static_cast<const raw*>(job.x);
        const coef_t* __restrict__ h = static_cast<const coef_t*>(job.h);
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
            const bool ok = PPF_INBOUNDS((size_t)slot * C::CHUNK_BYTES + bytes <= (size_t)C::RING_BYTES);
            mbar_arrive_expect_tx(&bars[slot], ok ? bytes : 0u);
            if (ok) tma_load_1d(ring + slot * C::CHUNK_BYTES, x + r0 * N, bytes, &bars[slot], policy);
        };
        if (tid == 0 && !failed) {
            const int first = nchunks < NCH ? nchunks : NCH;
            for (int k = 0; k < first; ++k) issue(k);
            issued = first;
        }

        // coefficients in registers, as in the ring kernel: channel pairs with
        // packed (h, h) pairs (G*T <= 32, at least 4 spectra per thread),
        // FP16 pairs with the mixed-precision FMA for FP16/int8 input, scalar
        // FP32 otherwise; one channel per thread keeps (h, h) pairs
        constexpr bool MIX = C::CPT == 2 && !std::is_same<typename C::In, InC32>::value;
        constexpr bool PK = C::CPT == 2 && !MIX && G * T <= 32 && RBT >= 4;
        float hr[C::CPT == 2 && !MIX && !PK ? G : 1][C::CPT == 2 && !MIX && !PK ? T : 1][2];
        float2 hp[PK ? G : 1][PK ? T : 1][2];
        uint32_t hq[MIX ? G : 1][MIX ? T : 1];
        float2 hh[C::CPT == 1 ? G : 1][C::CPT == 1 ? T : 1];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int c = C::CPT * (pbase + g * NF);
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

        int waited = 0;
        int rrb = (cbase % NCH) * RB;  // ring row of the block's first input row
        for (int b = 0; b < nb; ++b, ++gb) {
            const int need = (b + C::KO < nchunks ? b + C::KO : nchunks - 1) + 1;
            for (; waited < need && !failed; ++waited) {
                const int gk = cbase + waited;
                if (!mbar_wait_bounded(&bars[gk % NCH], (uint32_t)((gk / NCH) & 1))) {
                    failed = true;
                    break;  // this chunk stays "not waited for": the drain below waits for it
                }
            }
            const int j = gb & 1;
            // the FFT warps have read buffer j for the block before last
            if (gb >= 2) nbar_sync(kBarEmpty0 + j, C::NT);
            float2* const fb = X + j * C::BUF_SLOTS;

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
            auto ring_off = [&](int u, int c) -> size_t {
                if constexpr (C::RG == 1) {
                    return (size_t)cbase_off[u / RB] + ((size_t)(u % RB) * N + c) * BPS;
                } else {
                    int rr = rrb + i0 + u;
                    rr = rr >= RING_ROWS ? rr - RING_ROWS : rr;
                    return ((size_t)rr * N + c) * BPS;
                }
            };
            if (!failed) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int c = C::CPT * (pbase + g * NF);
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
            }
            // buffer j holds block b: hand it to the FFT warps
            nbar_arrive(kBarFull0 + j, C::NT);
            // every FIR thread's reads of chunk b are done: refill its slot
            failed = nbar_sync_or(kBarFir, NF, failed);
            if (tid == 0 && !failed && issued < nchunks && issued == b + NCH) {
                issue(issued);
                ++issued;
            }
            rrb += RB;
            rrb = rrb >= RING_ROWS ? rrb - RING_ROWS : rrb;
        }
        if (failed && tid == 0) {
            // let the copies still in flight land before the CTA moves on or exits
            for (int k = waited; k < issued; ++k) {
                const int gk = cbase + k;
                mbar_wait_bounded(&bars[gk % NCH], (uint32_t)((gk / NCH) & 1), kWaitLimitNs / 4);
            }
        }
        cbase += nchunks;
    }
    // the FFT warps arrive on EMPTY after every block; the arrivals of the
    // last two blocks have no later block waiting for them: take them here
    for (int g = gb - 2 < 0 ? 0 : gb - 2; g < gb; ++g) nbar_sync(kBarEmpty0 + (g & 1), C::NT);
    if (failed && tid == 0) atomicExch(err, 1);
}

// ------------------------------------------------------------------ FFT role
template <class C>
__device__ __forceinline__ void ws_fft_role(const PpfWork& wl, float2* X, const float2* __restrict__ tw)
{
    constexpr int N = C::N, RB = C::RB, NX = C::NX;
    const int lt = threadIdx.x - C::NF;
    WsTwiddles<N, NX, C::RC> twr;
    twr.load(tw, lt);
    int gb = 0;
    for (int it = blockIdx.x;; it += gridDim.x) {
        PpfJob job;
        int64_t blo, bhi;
        if (!ws_item(wl, it, RB, job, blo, bhi)) break;
        if (blo >= bhi) continue;
        typename C::OT* __restrict__ Y = reinterpret_cast<typename C::OT*>(job.Y);
        const int64_t S = job.S;
        const int nb = (int)(bhi - blo);
        const int64_t s_lo = blo * RB;
        const int64_t s_hi = S < bhi * RB ? S : bhi * RB;
        for (int b = 0; b < nb; ++b, ++gb) {
            const int j = gb & 1;
            nbar_sync(kBarFull0 + j, C::NT);
            const int64_t s0 = s_lo + (int64_t)b * RB;
            const int rows = (int)(s_hi - s0 < RB ? s_hi - s0 : RB);
            ws_fft_rows<N, RB, NX, C::RS, C::PD, C::RC>(X + j * C::BUF_SLOTS, twr, Y + s0 * N, rows, lt,
                                                 [&] { nbar_arrive(kBarEmpty0 + j, C::NT); });
        }
    }
}

template <class C>
__global__ void __launch_bounds__(C::NT, 1)
ppf_ws_kernel(const PpfWork wl, const float2* __restrict__ tw, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float2* X = reinterpret_cast<float2*>(smem + C::RING_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES + C::FFT_BYTES);
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::NCH; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // warps 0 .. NF/32-1 filter, the others transform (role boundaries fall
    // on warp boundaries, so every named barrier is executed warp-uniformly)
    if (threadIdx.x < C::NF) ws_fir_role<C>(wl, ring, X, bars, err);
    else ws_fft_role<C>(wl, X, tw);
}

}  // namespace ppf
