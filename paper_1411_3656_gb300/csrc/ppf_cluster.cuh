// Fused PPF kernel for large N*T: a thread-block cluster splits the channels.
//
// One SM cannot hold the T-row FIR window of every channel when N*T is large
// (N = 4096, T = 32 needs 1 MiB), so a cluster of P CTAs shares the work of
// each spectrum with the four-step form of the DFT.  With N = N1 * N2,
// channel c = c1 + N1*c2 and bin k = k2 + N2*k1:
//
//   Y[k2 + N2*k1] = sum_c1 W_N1^{c1*k1} * ( W_N^{c1*k2} * sum_c2 y[c1 + N1*c2] W_N2^{c2*k2} ).
//
// CTA `rank` owns the input channels with c1 in [rank*C1, (rank+1)*C1)
// (C1 = N1/P, all c2): a strided slice that a 3-D TMA tensor map
// (dims N1 x N2 x rows, box C1 x N2 x RB) lands densely in its ring.  Per
// block of RB spectra each CTA
//   1. filters its channels (Section 2, Eq. 1) from the ring;
//   2. takes the N2-point DFTs over c2 for each of its c1 (Stockham passes in
//      shared memory, element stride C1);
//   3. multiplies by W_N^{c1*k2} and stores each result into the shared
//      memory of the CTA that owns bin group k2 (st.async into distributed
//      shared memory, K2 = N2/P bins per CTA, completion counted in bytes on
//      the owner's mbarrier, so no cluster-wide fence is needed);
//   4. once its mbarrier has seen every byte, takes the N1-point DFTs over
//      c1 of its K2 bin groups and stores the spectra (runs of K2
//      consecutive bins); after its last read of the exchange buffer it
//      arrives on each peer's "buffer free" mbarrier.
// The exchange buffer is double-buffered per block parity.
// Input is read from HBM once, filtered data never leaves the cluster.
#pragma once

#include <cuda.h>

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"

namespace ppf {

__host__ __device__ constexpr int cl_max(int a, int b) { return a > b ? a : b; }

// Row stride of the stage-2 buffer: room for the first pass's padding and
// congruent to 16/K2 modulo 16 slots, so a half-warp (K2 bin groups x 16/K2
// butterflies) touches 16 distinct 8-byte bank slots.
__host__ __device__ constexpr int stage2_stride(int N1, int K2, int R0 = 16)
{
    const int base = N1 + cl_max(N1 / R0, 1) + 1;
    const int want = K2 >= 16 ? 1 : 16 / K2;
    int s = base;
    while (s % 16 != want % 16) ++s;
    return s;
}

template <int N_, int T_, class In_, int P_, int N1_, int NT_, int RB_, int NCH_, int MINB_ = 1, int CPT_ = 2,
          class OT_ = float2, int R0_ = 16>
struct ClusterCfg {
    using OT = OT_;  // output bin: float2 (complex64) or BinF16
    // radix of the first pass of each stage's transforms (8 or 16); R0 = 8
    // keeps every thread busy in that pass when RB*C1*N2/16 < threads
    static constexpr int R0 = R0_;
    static constexpr int N = N_, T = T_, P = P_, N1 = N1_, NT = NT_, RB = RB_, NCH = NCH_, MINB = MINB_;
    // FIR channels per thread: 2 (a pair, one 2-sample load per row, scalar
    // FMAs) or 1 (one channel, coefficients duplicated as (h, h) so that one
    // packed f32x2 FMA updates a complex accumulator)
    static constexpr int CPT = CPT_;
    using In = In_;
    using raw = typename In::raw;
    using coef_t = typename Coef<In>::type;
    static constexpr int BPS = In::bytes;
    static constexpr int N2 = N / N1;
    static constexpr int C1 = N1 / P;  // input channels c1 per CTA
    static constexpr int K2 = N2 / P;  // bin groups k2 per CTA
    static constexpr int NC = N / P;   // channels per CTA
    static constexpr int UNITS = NC / CPT;  // FIR work units per row
    static constexpr int G = UNITS > NT ? UNITS / NT : 1;
    static constexpr int RG = UNITS >= NT ? 1 : NT / UNITS;
    static constexpr int RBT = RB / RG;
    static constexpr int KO = T >= 2 ? (T - 2) / RB + 1 : 0;
    static constexpr int RING_ROWS = NCH * RB;
    static constexpr int CHUNK_BYTES = RB * NC * BPS;
    static constexpr int RING_BYTES = NCH * CHUNK_BYTES;
    static constexpr int RSB = (N2 + cl_max(N2 / R0, 1) + 1) * C1 + ((N2 + cl_max(N2 / R0, 1) + 1) * C1) % 2;
    static constexpr int A_SLOTS = RB * RSB;
    static constexpr int RS1 = stage2_stride(N1, K2, R0);
    static constexpr int X_SLOTS = RB * K2 * RS1;
    static constexpr int XBYTES = RB * K2 * N1 * 8;  // bytes each CTA receives per block
    static constexpr int SMEM = RING_BYTES + (A_SLOTS + 2 * X_SLOTS) * 8 + (NCH + 4) * 8;
    static_assert(P >= 2 && P <= 16, "cluster sizes 2..16 (above 8 needs the non-portable opt-in)");
    static_assert(CPT == 1 || CPT == 2, "one channel or a pair per thread");
    static_assert(UNITS % NT == 0 || NT % UNITS == 0, "FIR units must tile the threads");
    static_assert(C1 >= 2 && C1 % 2 == 0 && (C1 * BPS) % 16 == 0, "TMA box rows must be 16-byte multiples");
    static_assert(K2 >= 1 && N2 <= 256 && C1 <= 256 && RB <= 256, "TMA box limits");
    static_assert(RB % RG == 0 && RBT >= 1, "rows per block must split over row groups");
    static_assert(NCH >= KO + 2, "ring must hold a block's window plus one chunk in flight");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

// Twiddles W_{NS*R}^{(j mod NS)*r} of passes P.. of a length-L transform
// whose butterfly index is j = (tid mod (M*L/R)) / M (M transforms
// interleaved element-wise); kept in registers for the whole kernel.
template <int L, int M, int NT, int R0 = 16, int P = 1, bool ANY = (P < fft_npass_r(L, R0))>
struct StageTwiddles {
    static constexpr int R = fft_radix_r(L, P, R0);
    static constexpr int NS = fft_ns_r(L, P, R0);
    static_assert(NT % (M * L / R) == 0, "thread count must be a multiple of the butterflies per row");
    float2 w[R - 1];
    StageTwiddles<L, M, NT, R0, P + 1> next;
    __device__ __forceinline__ void load(const float2* __restrict__ tw, int N)
    {
        const int j = (threadIdx.x % (M * L / R)) / M;
        const int k = j % NS;
        const int step = N / (NS * R);
#pragma unroll
        for (int r = 1; r < R; ++r) w[r - 1] = __ldg(tw + k * r * step);
        next.load(tw, N);
    }
    template <int Q>
    __device__ __forceinline__ const float2* get() const
    {
        if constexpr (Q == P) return w;
        else return next.template get<Q>();
    }
};
template <int L, int M, int NT, int R0, int P>
struct StageTwiddles<L, M, NT, R0, P, false> {
    __device__ __forceinline__ void load(const float2* __restrict__, int) {}
    template <int Q>
    __device__ __forceinline__ const float2* get() const { return nullptr; }
};

// Per-thread data of the last stage-1 pass: four-step twiddles W_N^{c1*k2}
// and the cluster addresses its R outputs go to (row 0 of the X buffer).
template <class C>
struct Stage1Out {
    static constexpr int L = C::N2;
    static constexpr int PL = fft_npass_r(L, C::R0) - 1;
    static constexpr int R = fft_radix_r(L, PL, C::R0);
    static constexpr int NS = fft_ns_r(L, PL, C::R0);
    static_assert(C::NT % (C::C1 * (L / R)) == 0, "thread count must be a multiple of the butterflies per row");
    float2 w[R];
    uint32_t addr[R];
    uint32_t rbar[R];  // the owner's "exchange full" mbarrier for block parity 0 (+8 for parity 1)
    __device__ __forceinline__ void load(const float2* __restrict__ tw, float2* X, uint64_t* xfull, int rank)
    {
        constexpr int BPR = C::C1 * (L / R);
        const int rem = threadIdx.x % BPR;
        const int c1l = rem % C::C1, j = rem / C::C1;
        const int c1 = rank * C::C1 + c1l;
        const uint32_t xbase = smem_u32(X);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int k2 = j + q * NS;
            w[q] = __ldg(tw + (int)(((int64_t)c1 * k2) % C::N));
            const int dst = k2 / C::K2, k2l = k2 % C::K2;
            addr[q] = map_shared_rank(xbase + (uint32_t)((k2l * C::RS1 + c1) * 8), (uint32_t)dst);
            rbar[q] = map_shared_rank(smem_u32(xfull), (uint32_t)dst);
        }
    }
};

// Stage 1, pass PP: N2-point transforms over c2 in A (element stride C1, in
// place).  The last pass sends its outputs to the owning CTAs' X buffers.
template <class C, int PP>
__device__ __forceinline__ void stage1_pass(float2* A, const StageTwiddles<C::N2, C::C1, C::NT, C::R0>& tw,
                                            const Stage1Out<C>& so, uint32_t xoff, uint32_t boff)
{
    constexpr int L = C::N2, NT = C::NT, C1 = C::C1, RB = C::RB, RSB = C::RSB;
    constexpr int R = fft_radix_r(L, PP, C::R0), NS = fft_ns_r(L, PP, C::R0);
    constexpr bool LAST = (PP == fft_npass_r(L, C::R0) - 1);
    constexpr int IN_NS = PP == 0 ? 0 : fft_ns_r(L, PP - 1, C::R0);
    constexpr int IN_R = PP == 0 ? 1 : fft_radix_r(L, PP - 1, C::R0);
    constexpr int BPR = C1 * (L / R);
    constexpr int NB = RB * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT != 0 && b >= NB) continue;
        const int row = b / BPR, rem = b % BPR, c1l = rem % C1, j = rem / C1;
        const float2* a = A + row * RSB + c1l;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int idx = j + r * (L / R);
            if constexpr (IN_NS == 0) v[k][r] = a[idx * C1];
            else v[k][r] = a[pad_slot<IN_NS, IN_R>(idx) * C1];
        }
    }
    if constexpr (!LAST) __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT != 0 && b >= NB) continue;
        const int row = b / BPR, rem = b % BPR, c1l = rem % C1, j = rem / C1;
        if constexpr (PP > 0) apply_twiddles<R>(tw.template get<PP>(), v[k]);
        dft<R>(v[k]);
        if constexpr (!LAST) {
            float2* a = A + row * RSB + c1l;
            const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int q = 0; q < R; ++q) a[pad_slot<NS, R>(base + q * NS) * C1] = v[k][q];
        } else {
            const uint32_t roff = xoff + (uint32_t)(row * C::K2 * C::RS1 * 8);
#pragma unroll
            for (int q = 0; q < R; ++q) st_async_f2(so.addr[q] + roff, cmul(v[k][q], so.w[q]), so.rbar[q] + boff);
        }
    }
    if constexpr (!LAST) __syncthreads();
}

template <class C, int PP = 0>
__device__ __forceinline__ void stage1_upto_last(float2* A, const StageTwiddles<C::N2, C::C1, C::NT, C::R0>& tw,
                                                 const Stage1Out<C>& so)
{
    if constexpr (PP < fft_npass_r(C::N2, C::R0) - 1) {
        stage1_pass<C, PP>(A, tw, so, 0, 0);
        stage1_upto_last<C, PP + 1>(A, tw, so);
    }
}

// Stage 2, pass PP: N1-point transforms over c1 of rows (row, k2l) in X (in
// place); bin group k2l varies fastest across threads so the last pass stores
// runs of K2 consecutive bins.
template <class C, int PP, class F>
__device__ __forceinline__ void stage2_pass(float2* X, const StageTwiddles<C::N1, C::K2, C::NT, C::R0>& tw,
                                            typename C::OT* __restrict__ Yb, int rows, int rank,
                                            F&& after_last_read)
{
    constexpr int L = C::N1, NT = C::NT, K2 = C::K2, RB = C::RB, RS1 = C::RS1;
    constexpr int R = fft_radix_r(L, PP, C::R0), NS = fft_ns_r(L, PP, C::R0);
    constexpr bool LAST = (PP == fft_npass_r(L, C::R0) - 1);
    constexpr int IN_NS = PP == 0 ? 0 : fft_ns_r(L, PP - 1, C::R0);
    constexpr int IN_R = PP == 0 ? 1 : fft_radix_r(L, PP - 1, C::R0);
    constexpr int BPR = K2 * (L / R);
    constexpr int NB = RB * BPR;
    constexpr int PER = (NB + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT != 0 && b >= NB) continue;
        const int row = b / BPR, rem = b % BPR, k2l = rem % K2, j = rem / K2;
        const float2* x = X + (row * K2 + k2l) * RS1;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int idx = j + r * (L / R);
            if constexpr (IN_NS == 0) v[k][r] = x[idx];
            else v[k][r] = x[pad_slot<IN_NS, IN_R>(idx)];
        }
    }
    if constexpr (!LAST) __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT != 0 && b >= NB) continue;
        if constexpr (PP > 0) apply_twiddles<R>(tw.template get<PP>(), v[k]);
        dft<R>(v[k]);
    }
    if constexpr (LAST) after_last_read();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = threadIdx.x + k * NT;
        if (NB % NT != 0 && b >= NB) continue;
        const int row = b / BPR, rem = b % BPR, k2l = rem % K2, j = rem / K2;
        if constexpr (!LAST) {
            float2* x = X + (row * K2 + k2l) * RS1;
            const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int q = 0; q < R; ++q) x[pad_slot<NS, R>(base + q * NS)] = v[k][q];
        } else if (row < rows) {
            typename C::OT* o = Yb + (int64_t)row * C::N + rank * K2 + k2l;
#pragma unroll
            for (int q = 0; q < R; ++q) st_bin(o + (int64_t)C::N2 * (j + q * NS), v[k][q]);
        }
    }
    if constexpr (!LAST) __syncthreads();
}

template <class C, int PP = 0, class F>
__device__ __forceinline__ void stage2(float2* X, const StageTwiddles<C::N1, C::K2, C::NT, C::R0>& tw,
                                       typename C::OT* __restrict__ Yb, int rows, int rank, F&& after_last_read)
{
    if constexpr (PP < fft_npass_r(C::N1, C::R0)) {
        stage2_pass<C, PP>(X, tw, Yb, rows, rank, after_last_read);
        stage2<C, PP + 1>(X, tw, Yb, rows, rank, after_last_read);
    }
}

template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB)
ppf_cluster_kernel(const __grid_constant__ CUtensorMap xmap, const PpfWork wl, const float2* __restrict__ tw,
                   int* __restrict__ err)
{
    constexpr int N = C::N, T = C::T, NT = C::NT, RB = C::RB, NCH = C::NCH, P = C::P;
    constexpr int G = C::G, RBT = C::RBT, BPS = C::BPS, RING_ROWS = C::RING_ROWS, NC = C::NC, C1 = C::C1;
    using PV = typename Pair<typename C::In>::vec;
    using raw = typename C::raw;
    using coef_t = typename C::coef_t;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float2* A = reinterpret_cast<float2*>(smem + C::RING_BYTES);
    float2* X = A + C::A_SLOTS;  // two buffers of X_SLOTS
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES + (C::A_SLOTS + 2 * C::X_SLOTS) * 8);
    uint64_t* xfull = bars + NCH;      // [2]: every byte of X[parity] has arrived
    uint64_t* xfree = bars + NCH + 2;  // [2]: every owner has finished reading its X[parity]

    const int tid = threadIdx.x;
    const int rank = (int)cluster_ctarank();
    const int cid = blockIdx.x / P, ncl = gridDim.x / P;

    if (tid == 0) {
        for (int i = 0; i < NCH; ++i) mbar_init(&bars[i], 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&xfull[i], 1);
            mbar_init(&xfree[i], P);
        }
        fence_mbar_init();
    }
    // every CTA of the cluster is running, with its mbarriers initialised,
    // before any distributed-memory store or remote arrive
    cluster_arrive_release();
    cluster_wait_acquire();
    const uint64_t policy = l2_evict_first_policy();

    // FIR ownership: unit pp is channel pair (c1l, c1l+1) at c2 of this CTA's
    // slice (CPT = 2) or the single channel at ring offset pp (CPT = 1)
    const int rg = C::UNITS >= NT ? 0 : tid / C::UNITS;
    const int pbase = C::UNITS >= NT ? tid : tid % C::UNITS;
    const int i0 = rg * RBT;
    StageTwiddles<C::N2, C1, NT, C::R0> tw1;
    tw1.load(tw, N);
    StageTwiddles<C::N1, C::K2, NT, C::R0> tw2;
    tw2.load(tw, N);
    Stage1Out<C> so;
    so.load(tw, X, xfull, rank);

    int cbase = 0;  // ring chunks this CTA issued in earlier bands (slots and phases continue)
    int gbase = 0;  // blocks this cluster exchanged in earlier bands (X parity and phases continue)
    bool failed = false;
    // Every CTA of a cluster walks the same items, so the cluster keeps one
    // schedule of exchanges and nobody waits on a peer that has moved on.
    for (int it = cid;; it += ncl) {
        PpfJob job;
        const void* tmap;
        int64_t blo, bhi;
        if (wl.items == nullptr) {
            if (it != cid) break;
            job = wl.one;
            tmap = &xmap;
            const int64_t nblk = (job.S + RB - 1) / RB;
            blo = nblk * cid / ncl;
            bhi = nblk * (cid + 1) / ncl;
        } else {
            if (it >= wl.n_items) break;
            const PpfItem item = wl.items[it];
            job = wl.jobs[item.job];
            tmap = job.tmap;
            blo = item.blo;
            bhi = item.bhi;
        }
        if (blo >= bhi) continue;
        const coef_t* __restrict__ h = static_cast<const coef_t*>(job.h);
        typename C::OT* __restrict__ Y = reinterpret_cast<typename C::OT*>(job.Y);
        const int64_t S = job.S;
        const int nb = (int)(bhi - blo);
        const int64_t s_lo = blo * RB;
        const int64_t s_hi = S < bhi * RB ? S : bhi * RB;
        const int64_t in_end = s_hi + T - 1;
        const int nchunks = (int)((in_end - s_lo + RB - 1) / RB);

        int issued = 0;
        auto issue = [&](int k) {
            const int slot = (cbase + k) % NCH;
            mbar_arrive_expect_tx(&bars[slot], (uint32_t)C::CHUNK_BYTES);
            tma_load_3d(ring + slot * C::CHUNK_BYTES, tmap, rank * C1, 0, (int)(s_lo + (int64_t)k * RB), &bars[slot],
                        policy);
        };
        if (tid == 0 && !failed) {
            const int first = nchunks < NCH ? nchunks : NCH;
            for (int k = 0; k < first; ++k) issue(k);
            issued = first;
        }

        // coefficients of the owned channels, in registers for the whole item
        // (CPT = 1 keeps each as the pair (h, h))
        float hr[C::CPT == 2 ? G : 1][C::CPT == 2 ? T : 1][2];
        float2 hh[C::CPT == 1 ? G : 1][C::CPT == 1 ? T : 1];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int pp = pbase + g * NT;
            if constexpr (C::CPT == 2) {
                const int c1l = 2 * (pp % (C1 / 2)), c2 = pp / (C1 / 2);
                const int c = rank * C1 + c1l + C::N1 * c2;
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    hr[g][t][0] = coef_f(h[t * N + c]);
                    hr[g][t][1] = coef_f(h[t * N + c + 1]);
                }
            } else {
                const int c = rank * C1 + pp % C1 + C::N1 * (pp / C1);
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float v = coef_f(h[t * N + c]);
                    hh[g][t] = make_float2(v, v);
                }
            }
        }

        int waited = 0, rrb = (cbase % NCH) * RB;
        // Software pipeline: iteration b filters and sends block b, then
        // finishes block b-1, whose exchange data arrived meanwhile.
        for (int b = 0; b <= nb; ++b) {
            if (b < nb) {
                bool ok = true;
                if (!failed) {
                    const int need = (b + C::KO < nchunks ? b + C::KO : nchunks - 1) + 1;
                    for (; waited < need; ++waited) {
                        const int gk = cbase + waited;
                        if (!mbar_wait_bounded(&bars[gk % NCH], (uint32_t)((gk / NCH) & 1))) {
                            ok = false;
                            break;
                        }
                    }
                }
                // A failed wait is recorded and the cluster keeps its schedule (no
                // early exit, so no CTA waits on one that has left); the flag
                // spreads over the CTA at the barrier after the FIR.  Every thread
                // waits for the chunks itself, so no barrier is needed here, except
                // after block 0, whose stage-1 reads of A no stage-2 barrier has
                // yet ordered before this block's FIR writes.
                if (!ok) failed = true;
                if (b == 1) __syncthreads();

                // 1. FIR over the ring
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int pp = pbase + g * NT;
                    if constexpr (C::CPT == 2) {
                        const int l = (pp / (C1 / 2)) * C1 + 2 * (pp % (C1 / 2));
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
                            const PV pv = *reinterpret_cast<const PV*>(ring + ((size_t)rr * NC + l) * BPS);
                            float2 v0, v1;
                            split_cvt<typename C::In>(pv, v0, v1);
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
                            *reinterpret_cast<float4*>(A + (i0 + i) * C::RSB + l) =
                                make_float4(a0[i].x, a0[i].y, a1[i].x, a1[i].y);
                    } else {
                        const int l = pp;
                        float2 a[RBT];
#pragma unroll
                        for (int i = 0; i < RBT; ++i) a[i] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int u = 0; u < RBT + T - 1; ++u) {
                            int rr = rrb + i0 + u;
                            rr = rr >= RING_ROWS ? rr - RING_ROWS : rr;
                            const float2 v = decode_cvt(*reinterpret_cast<const raw*>(ring + ((size_t)rr * NC + l) * BPS));
#pragma unroll
                            for (int i = 0; i < RBT; ++i) {
                                const int t = u - i;
                                if (t >= 0 && t < T) a[i] = __ffma2_rn(hh[g][t], v, a[i]);
                            }
                        }
#pragma unroll
                        for (int i = 0; i < RBT; ++i) A[(i0 + i) * C::RSB + l] = a[i];
                    }
                }
                if (__syncthreads_or(failed)) failed = true;
                if (tid == 0 && !failed && issued < nchunks && issued == b + NCH) {
                    issue(issued);
                    ++issued;
                }
                rrb += RB;
                rrb = rrb >= RING_ROWS ? rrb - RING_ROWS : rrb;

                // 2-3. N2-point DFTs, four-step twiddle, send to the owning CTAs
                const int gb = gbase + b, par = gb & 1;
                if (tid == 0) mbar_arrive_expect_tx(&xfull[par], (uint32_t)C::XBYTES);
                stage1_upto_last<C>(A, tw1, so);
                // the owners have finished reading X[par] of exchange gb-2 (each
                // thread waits before its own sends)
                if (gb >= 2 && !failed && !mbar_wait_bounded(&xfree[par], (uint32_t)(((gb >> 1) - 1) & 1)))
                    failed = true;
                stage1_pass<C, fft_npass_r(C::N2, C::R0) - 1>(A, tw1, so, (uint32_t)(par * C::X_SLOTS * 8),
                                                     (uint32_t)(par * 8));
            }
            if (b >= 1) {
                // 4. block b-1: once every byte of X[par] is here, N1-point DFTs and store
                const int bp = b - 1, gb = gbase + bp, par = gb & 1;
                // each thread waits before its own reads of X[par]
                if (!failed && !mbar_wait_bounded(&xfull[par], (uint32_t)((gb >> 1) & 1))) failed = true;
                const int64_t s0 = s_lo + (int64_t)bp * RB;
                const int rows = (int)(s_hi - s0 < RB ? s_hi - s0 : RB);
                stage2<C>(X + par * C::X_SLOTS, tw2, Y + s0 * N, rows, rank, [&] {
                    // every thread's last reads of X[par] have returned; free it for the senders
                    __syncthreads();
                    if (tid < P) mbar_arrive_remote(map_shared_rank(smem_u32(&xfree[par]), (uint32_t)tid));
                });
            }
        }
        if (failed && tid == 0) {
            for (int k = waited; k < issued; ++k) {
                const int gk = cbase + k;
                mbar_wait_bounded(&bars[gk % NCH], (uint32_t)((gk / NCH) & 1), kWaitLimitNs / 4);
            }
        }
        cbase += nchunks;
        gbase += nb;
    }
    const bool any_failed = __syncthreads_or(failed);
    // no CTA leaves while a peer may still store into its shared memory
    cluster_arrive_release();
    cluster_wait_acquire();
    if (any_failed && tid == 0) atomicExch(err, 1);
}

}  // namespace ppf
