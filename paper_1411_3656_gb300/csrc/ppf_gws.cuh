// Fused PPF kernel for N*T too large for one SM, with warp-specialised FIR
// and FFT roles: the cluster exchange of the gather kernel (ppf_gather.cuh)
// run by two groups of warps in every CTA that work on consecutive rounds at
// the same time.
//
// A cluster of P CTAs splits the channels into P contiguous slices; spectra
// go in rounds of P*RB, block q of a round (RB consecutive spectra) belongs to
// CTA q.  In every CTA
//   FIR warps (NF threads): wait for the ring chunks of round k (1-D bulk
//     copies of this CTA's slice of each input row, every input byte read
//     from HBM once), filter the slice for the round's P*RB spectra (Section
//     2, Eq. 1) with coefficients in registers, wait until every owner has
//     freed the FFT buffer the round goes to, and st.async each filtered
//     channel pair (16 bytes) into the owning CTA's buffer, completion
//     counted in bytes on the owner's "full" mbarrier; then refill the ring
//     chunk the round no longer needs;
//   FFT warps (NX threads): wait until their own buffer holds all N channels
//     of the round's RB rows, take the N-point DFTs (Section 2) with
//     Stockham passes in place, arrive on every CTA's "free" mbarrier right
//     after the last pass's loads, and store the spectra.
// With one FFT buffer the FIR warps compute round k+1 while the FFT warps
// transform round k and store it once the owners have freed the buffer; with
// two, round k+1 is stored into the other buffer at once.
//
// Ordering: a CTA's "full" mbarrier for round k takes its local arrival
// (with the expected byte count) only after every owner freed the buffer
// from round k-NXB, which implies that this CTA's FFT warps observed the
// completion of that earlier phase; peers' bytes for round k may arrive
// before the local arrival (the phase cannot complete without it).
#pragma once

#include <type_traits>

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"
#include "ppf_ws.cuh"

namespace ppf {

template <int N_, int T_, class In_, int P_, int NF_, int NX_, int RB_, int NCH_, int NXB_ = 1, class OT_ = float2,
          int PD_ = 1, int RF_ = 0, int RX_ = 0, int ER_ = 0, int PF_ = 0>
struct GwsCfg {
    using OT = OT_;  // output bin: float2 (complex64) or BinF16
    using In = In_;
    using raw = typename In::raw;
    using coef_t = typename Coef<In>::type;
    static constexpr int N = N_, T = T_, P = P_, NF = NF_, NX = NX_, RB = RB_, NCH = NCH_, NXB = NXB_, PD = PD_;
    static constexpr int NT = NF + NX;
    static constexpr int BPS = In::bytes;
    static constexpr int NC = N / P;                     // channels per CTA
    static constexpr int ROWS = P * RB;                  // spectra per round = input rows per ring chunk
    static constexpr int UNITS = NC / 2;                 // FIR units (channel pairs) per row
    static constexpr int G = UNITS > NF ? UNITS / NF : 1;
    static constexpr int RG = UNITS >= NF ? 1 : NF / UNITS;
    static constexpr int RBT = ROWS / RG;                // spectra per FIR thread per round
    static constexpr int KO = T >= 2 ? (T - 2) / ROWS + 1 : 0;
    // early refill (ER, one row group whose window runs past its first
    // chunk): chunks are waited for as the window reaches them and the first
    // is refilled mid-round, at the cost of a second FIR barrier per round
    static constexpr bool EARLY = ER_ != 0 && RG == 1 && RBT + T - 1 > ROWS;
    static_assert(ER_ == 0 || EARLY, "early refill needs one row group and a window past its first chunk");
    // L2 prefetch distance (PF > 0): when chunk k of an item is copied into
    // the ring, chunk k + PF is prefetched into L2, so PF more chunks of the
    // stream are in flight than the ring itself holds
    static constexpr int PF = PF_;
    static constexpr int RING_ROWS = NCH * ROWS;
    static constexpr int SEG_BYTES = NC * BPS;           // one input row's slice
    static constexpr int CHUNK_BYTES = ROWS * SEG_BYTES;
    static constexpr int RING_BYTES = NCH * CHUNK_BYTES;
    static constexpr int RS = PD == 1 ? fft_row_stride(N) : N + (N / 32 > 2 ? N / 32 : 2);
    static constexpr int X_SLOTS = RB * RS;              // one FFT buffer
    static constexpr int XBYTES = RB * N * 8;            // bytes a buffer receives per round
    static constexpr int SMEM = RING_BYTES + NXB * X_SLOTS * 8 + (NCH + 2 * NXB) * 8;
    // Register split (RF > 0): at launch every thread gets the same count
    // (LREG, the launch bound's share of the 64K-register file); the FIR
    // warpgroups then raise theirs to RF and the FFT warpgroups lower theirs
    // to RX, so the FIR's coefficients and accumulators need not spill to fit
    // the FFT threads' count.  The host refuses the tile if the compiled
    // kernel was given fewer than LREG registers a thread at launch.
    static constexpr int RF = RF_, RX = RX_;
    static constexpr int LREG = (65536 / NT) / 8 * 8 > 255 ? 255 : (65536 / NT) / 8 * 8;
    static_assert(RF == 0 || (NF % 128 == 0 && NX % 128 == 0), "register split: whole warpgroups per role");
    static_assert(RF == 0 || (RF % 8 == 0 && RX % 8 == 0 && RX >= 24 && RF <= 256),
                  "register split: FIR count up, FFT count down, multiples of 8");
    static_assert(RF == 0 || NF * RF + NX * RX <= NT * LREG, "register split exceeds the launch pool");
    static_assert(P >= 2 && P <= 8, "portable cluster sizes");
    static_assert(N % (2 * P) == 0 && SEG_BYTES % 16 == 0, "16-byte row slices");
    static_assert(NF % 32 == 0 && NX % 32 == 0 && NT <= 1024, "whole warps per role");
    static_assert(UNITS % NF == 0 || NF % UNITS == 0, "FIR units must tile the FIR threads");
    static_assert(ROWS % RG == 0 && RBT >= 1, "spectra per round must split over row groups");
    // the ring holds a round's window; a deeper ring keeps refills in flight
    static_assert(NCH >= KO + 1, "ring must hold a round's window");
    static_assert(NXB == 1 || NXB == 2, "one or two FFT buffers");
    static_assert(RS % 2 == 0, "16-byte aligned channel pairs in the FFT buffer");
    static_assert(XBYTES < (1 << 20), "mbarrier transaction count");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

// The band of rounds [blo, bhi) of work item `it` (or of the one job) for
// cluster `cid` of `ncl`; false when the cluster has no further item.
__device__ __forceinline__ bool gws_item(const PpfWork& wl, int it, int cid, int ncl, int rows, PpfJob& job,
                                         int64_t& blo, int64_t& bhi)
{
    if (wl.items == nullptr) {
        if (it != cid) return false;
        job = wl.one;
        const int64_t nround = (job.S + rows - 1) / rows;
        blo = nround * cid / ncl;
        bhi = nround * (cid + 1) / ncl;
        return true;
    }
    if (it >= work_items(wl)) return false;
    const PpfItem item = wl.items[it];
    job = wl.jobs[item.job];
    blo = item.blo;
    bhi = item.bhi;
    return true;
}

// Buffer and mbarrier phase of global round gk.
template <class C>
__device__ __forceinline__ int gws_buf(int gk)
{
    return C::NXB == 1 ? 0 : (gk & 1);
}
template <class C>
__device__ __forceinline__ uint32_t gws_phase(int gk)
{
    return (uint32_t)((C::NXB == 1 ? gk : (gk >> 1)) & 1);
}

// ------------------------------------------------------------------ FIR role
template <class C>
__device__ __forceinline__ void gws_fir_role(const PpfWork& wl, unsigned char* ring, uint32_t xbase,
                                             uint64_t* bars, uint64_t* xfull, uint64_t* xfree, int rank, int cid,
                                             int ncl, bool& failed)
{
    constexpr int N = C::N, T = C::T, NF = C::NF, RB = C::RB, NCH = C::NCH, P = C::P;
    constexpr int G = C::G, RBT = C::RBT, BPS = C::BPS, RING_ROWS = C::RING_ROWS, NC = C::NC, ROWS = C::ROWS;
    using PV = typename Pair<typename C::In>::vec;
    using raw = typename C::raw;
    using coef_t = typename C::coef_t;
    const int tid = threadIdx.x;
    const uint64_t policy = l2_evict_first_policy();
    const uint32_t fullbase = smem_u32(xfull);
    const int rg = C::UNITS >= NF ? 0 : tid / C::UNITS;
    const int pbase = C::UNITS >= NF ? tid : tid % C::UNITS;
    const int i0 = rg * RBT;

    int cbase = 0;  // ring chunks this CTA issued in earlier items (slots and phases continue)
    int gbase = 0;  // rounds this cluster ran in earlier items (mbarrier phases continue)
    for (int it = cid;; it += ncl) {
        PpfJob job;
        int64_t blo, bhi;
        if (!gws_item(wl, it, cid, ncl, ROWS, job, blo, bhi)) break;
        if (blo >= bhi) continue;
        const raw* __restrict__ x = static_cast<const raw*>(job.x);
        const coef_t* __restrict__ h = static_cast<const coef_t*>(job.h);
        const int64_t S = job.S;
        const int nr = (int)(bhi - blo);
        const int64_t s_lo = blo * ROWS;
        const int64_t s_hi = S < bhi * ROWS ? S : bhi * ROWS;
        const int64_t in_end = s_hi + T - 1;  // input rows the item reads: [s_lo, in_end)
        const int nchunks = (int)((in_end - s_lo + ROWS - 1) / ROWS);

        int issued = 0;  // chunks of this item issued so far (meaningful in thread 0)
        // L2 prefetch of chunk k's rows (only rows the item reads)
        auto prefetch = [&](int k) {
            const int64_t r0 = s_lo + (int64_t)k * ROWS;
            const int nrows = (int)(in_end - r0 < ROWS ? in_end - r0 : ROWS);
            for (int q = 0; q < nrows; ++q) l2_prefetch_1d(x + (r0 + q) * N + rank * NC, (uint32_t)C::SEG_BYTES);
        };
        auto issue = [&](int k) {
            const int64_t r0 = s_lo + (int64_t)k * ROWS;
            const int nrows = (int)(in_end - r0 < ROWS ? in_end - r0 : ROWS);
            const int slot = (cbase + k) % NCH;
            // (copies the checked build refuses complete the phase with no bytes)
            const bool ok = PPF_INBOUNDS(slot * C::CHUNK_BYTES + nrows * C::SEG_BYTES <= C::RING_BYTES);
            mbar_arrive_expect_tx(&bars[slot], ok ? (uint32_t)(nrows * C::SEG_BYTES) : 0u);
            for (int q = 0; q < (ok ? nrows : 0); ++q)
                tma_load_1d(ring + slot * C::CHUNK_BYTES + q * C::SEG_BYTES, x + (r0 + q) * N + rank * NC,
                            (uint32_t)C::SEG_BYTES, &bars[slot], policy);
            if constexpr (C::PF > 0) {
                // (chunks of the ring's first fill are copied at once)
                if (k + C::PF < nchunks && k + C::PF >= NCH) prefetch(k + C::PF);
            }
        };
        if (tid == 0 && !failed) {
            const int first = nchunks < NCH ? nchunks : NCH;
            for (int k = 0; k < first; ++k) issue(k);
            issued = first;
        }

        // coefficients of the owned channel pairs, in registers for the whole
        // item: for complex64 input one (h[c], h[c+1]) pair per tap, which a
        // packed FMA applies to the pair's real parts and to its imaginary
        // parts (each lane the scalar FMA, so bitwise the scalar result, in
        // half the instructions and no more registers); FP16 pairs for FP16
        // and int8 input (mixed-precision FMA on FP16 samples, int8 turned
        // into FP16 exactly)
        constexpr bool MIX = !std::is_same<typename C::In, InC32>::value;
        float2 hs[MIX ? 1 : G][MIX ? 1 : T];
        uint32_t hq[MIX ? G : 1][MIX ? T : 1];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int c = rank * NC + 2 * (pbase + g * NF);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                if constexpr (MIX) {
                    hq[g][t] = *reinterpret_cast<const uint32_t*>(h + t * N + c);
                } else {
                    hs[g][t] = make_float2(coef_f(h[t * N + c]), coef_f(h[t * N + c + 1]));
                }
            }
        }

        int waited = 0;
        // every thread waits itself for the item's chunks up to `upto`
        auto wait_chunks = [&](int upto) {
            const int need = (upto < nchunks ? upto : nchunks - 1) + 1;
            for (; waited < need && !failed; ++waited) {
                const int gc = cbase + waited;
                if (!mbar_wait_bounded(&bars[gc % NCH], (uint32_t)((gc / NCH) & 1))) {
                    failed = true;
                    break;  // this chunk stays "not waited for": the drain below waits for it
                }
            }
        };
        // once every FIR thread is past the round's first chunk, its slot
        // takes the next chunk of the item (in order)
        auto refill = [&](int k) {
            failed = nbar_sync_or(kBarFir, NF, failed);
            if (tid == 0 && !failed && issued < nchunks && issued == k + NCH) {
                issue(issued);
                ++issued;
            }
        };
        for (int k = 0; k < nr; ++k) {
            const int gk = gbase + k;
            const int b = gws_buf<C>(gk);
            const int rrb = ((cbase + k) % NCH) * ROWS;
            // 1. the round reads chunks k .. k+KO.  With one row group (every
            //    thread filters all of the round's spectra) each chunk is
            //    waited for right before the window first reaches it, and the
            //    first chunk's slot is refilled as soon as every thread has
            //    passed it (EARLY), so a refill has more than a round to land;
            //    otherwise all are waited for here and the refill follows the
            //    round.
            if constexpr (!C::EARLY) wait_chunks(k + C::KO);
            // 2. FIR over the ring; row i of the round goes to CTA i / RB.
            //    With one row group the window starts at a chunk boundary, so
            //    the chunk bases are computed once per round.
            constexpr int NW = (RBT + T - 2) / ROWS + 1;  // chunks the window spans
            uint32_t cbase_off[C::RG == 1 ? NW : 1];
            if constexpr (C::RG == 1) {
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    int sl = rrb / ROWS + w;
                    sl -= sl >= NCH ? NCH : 0;
                    cbase_off[w] = (uint32_t)(sl * C::CHUNK_BYTES);
                }
            }
            auto ring_off = [&](int u, int cl) -> size_t {
                if constexpr (C::RG == 1) {
                    return (size_t)cbase_off[u / ROWS] + ((size_t)(u % ROWS) * NC + cl) * BPS;
                } else {
                    int rr = rrb + i0 + u;
                    rr = rr >= RING_ROWS ? rr - RING_ROWS : rr;
                    return ((size_t)rr * NC + cl) * BPS;
                }
            };
            bool freed = gk < C::NXB;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int cl = 2 * (pbase + g * NF);
                float2 a0[RBT], a1[RBT];
#pragma unroll
                for (int i = 0; i < RBT; ++i) {
                    a0[i] = make_float2(0.f, 0.f);
                    a1[i] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < RBT + T - 1; ++u) {
                    if constexpr (C::EARLY) {
                        if (g == 0 && u % ROWS == 0) wait_chunks(k + u / ROWS);
                        if (g == G - 1 && u == ROWS) refill(k);
                    }
                    const size_t ro = ring_off(u, cl);
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
                    } else {
                        // a0[i] holds (re c, re c+1), a1[i] (im c, im c+1)
                        float2 v0, v1;
                        Pair<typename C::In>::split(pv, v0, v1);
                        const float2 xr = make_float2(v0.x, v1.x), xi = make_float2(v0.y, v1.y);
#pragma unroll
                        for (int i = 0; i < RBT; ++i) {
                            const int t = u - i;
                            if (t >= 0 && t < T) {
                                a0[i] = __ffma2_rn(hs[g][t], xr, a0[i]);
                                a1[i] = __ffma2_rn(hs[g][t], xi, a1[i]);
                            }
                        }
                    }
                }
                // 3. every owner has freed buffer b from round gk - NXB (each
                //    thread waits before its own stores; thread 0 then opens
                //    this CTA's phase of the buffer for round gk)
                if (!freed) {
                    if (!failed && !mbar_wait_cluster_bounded(&xfree[b], gws_phase<C>(gk - C::NXB))) failed = true;
                    freed = true;
                }
                // (after a failure the phase is left alone: the owners' bounded
                // waits for it give up)
                if (g == 0 && tid == 0 && !failed) mbar_arrive_expect_tx(&xfull[b], (uint32_t)C::XBYTES);
                if (!failed) {
#pragma unroll
                    for (int i = 0; i < RBT; ++i) {
                        const int row = i0 + i, q = row / RB, rr = row % RB;
                        const uint32_t off = (uint32_t)((rr * C::RS + rank * NC + cl) * 8);
                        const float4 y = MIX ? make_float4(a0[i].x, a0[i].y, a1[i].x, a1[i].y)
                                             : make_float4(a0[i].x, a1[i].x, a0[i].y, a1[i].y);
                        if (PPF_INBOUNDS(off + 16 <= (uint32_t)C::X_SLOTS * 8 && q < P))
                            st_async_f4(map_shared_rank(xbase + b * C::X_SLOTS * 8 + off, (uint32_t)q), y,
                                        map_shared_rank(fullbase + b * 8, (uint32_t)q));
                    }
                }
            }
            // 4. every FIR thread's reads of chunk k are done: refill its slot
            if constexpr (!C::EARLY) refill(k);
        }
        if (failed && tid == 0) {
            // let the copies still in flight land before the CTA moves on or exits
            for (int k = waited; k < issued; ++k) {
                const int gc = cbase + k;
                mbar_wait_bounded(&bars[gc % NCH], (uint32_t)((gc / NCH) & 1), kWaitLimitNs / 4);
            }
        }
        cbase += nchunks;
        gbase += nr;
    }
}

// ------------------------------------------------------------------ FFT role
template <class C>
__device__ __forceinline__ void gws_fft_role(const PpfWork& wl, float2* X, const float2* __restrict__ tw,
                                             uint64_t* xfull, uint64_t* xfree, int rank, int cid, int ncl,
                                             bool& failed)
{
    constexpr int N = C::N, NX = C::NX, RB = C::RB, P = C::P, ROWS = C::ROWS;
    const int lt = threadIdx.x - C::NF;
    const uint32_t freebase = smem_u32(xfree);
    WsTwiddles<N, NX> twr;
    twr.load(tw, lt);
    int gbase = 0;
    for (int it = cid;; it += ncl) {
        PpfJob job;
        int64_t blo, bhi;
        if (!gws_item(wl, it, cid, ncl, ROWS, job, blo, bhi)) break;
        if (blo >= bhi) continue;
        typename C::OT* __restrict__ Y = reinterpret_cast<typename C::OT*>(job.Y);
        const int64_t S = job.S;
        const int nr = (int)(bhi - blo);
        const int64_t s_lo = blo * ROWS;
        const int64_t s_hi = S < bhi * ROWS ? S : bhi * ROWS;
        for (int k = 0; k < nr; ++k) {
            const int gk = gbase + k;
            const int b = gws_buf<C>(gk);
            // this CTA's block of the round: all N channels of its RB rows
            if (!failed && !mbar_wait_bounded(&xfull[b], gws_phase<C>(gk))) failed = true;
            const int64_t s0 = s_lo + (int64_t)k * ROWS + rank * RB;
            const int64_t left = s_hi - s0;
            const int rows = (int)(left < 0 ? 0 : (left < RB ? left : RB));
            ws_fft_rows<N, RB, NX, C::RS, C::PD>(X + b * C::X_SLOTS, twr, Y + (rows > 0 ? s0 : 0) * N, rows, lt,
                                                 [&] {
                // every FFT thread's last read of the buffer is done: free it on every CTA
                nbar_sync(kBarFft, NX);
                if (lt < P) mbar_arrive_cluster(map_shared_rank(freebase + b * 8, (uint32_t)lt));
            });
        }
        gbase += nr;
    }
}

template <class C>
__global__ void __launch_bounds__(C::NT, 1)
ppf_gws_kernel(const PpfWork wl, const float2* __restrict__ tw, int* __restrict__ err)
{
    constexpr int P = C::P;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float2* X = reinterpret_cast<float2*>(smem + C::RING_BYTES);  // the FFT buffer(s)
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES + C::NXB * C::X_SLOTS * 8);
    uint64_t* xfull = bars + C::NCH;            // [NXB] every byte of this CTA's buffer has arrived
    uint64_t* xfree = bars + C::NCH + C::NXB;   // [NXB] every owner has finished reading its buffer
    const int rank = (int)cluster_ctarank();
    const int cid = blockIdx.x / P, ncl = gridDim.x / P;
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::NCH; ++i) mbar_init(&bars[i], 1);
        for (int b = 0; b < C::NXB; ++b) {
            mbar_init(&xfull[b], 1);
            mbar_init(&xfree[b], P);
        }
        fence_mbar_init();
    }
    // every CTA of the cluster is running, with its mbarriers initialised,
    // before any distributed-memory store or remote arrive
    cluster_arrive_release();
    cluster_wait_acquire();
    bool failed = false;
    // warps 0 .. NF/32-1 filter, the others transform (role boundaries fall
    // on warp boundaries, so every named barrier is executed warp-uniformly)
    if (threadIdx.x < C::NF) {
        if constexpr (C::RF > 0) regs_inc<C::RF>();
        gws_fir_role<C>(wl, ring, smem_u32(X), bars, xfull, xfree, rank, cid, ncl, failed);
    } else {
        if constexpr (C::RF > 0) regs_dec<C::RX>();
        gws_fft_role<C>(wl, X, tw, xfull, xfree, rank, cid, ncl, failed);
    }
    const bool any_failed = __syncthreads_or(failed);
    // no CTA leaves while a peer may still store into its shared memory
    cluster_arrive_release();
    cluster_wait_acquire();
    if (any_failed && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace ppf
