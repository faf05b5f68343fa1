// Fused PPF kernel for N*T too large for one SM: a cluster of P CTAs splits
// the channels into P contiguous slices and gathers every filtered block in
// one CTA for its FFT.
//
// The T-row window over all N channels (N*T*8 bytes for complex64: 256 KiB
// at N*T = 32K) does not fit one SM's shared memory, but a CTA's slice of N/P
// channels does.  Spectra go in rounds of P*RB; block q of a round (RB
// consecutive spectra) belongs to CTA q of the cluster.  Per round every CTA
//   1. filters (Section 2, Eq. 1) its channel slice for the round's P*RB
//      spectra from its ring (1-D bulk copies of its slice of each input row);
//   2. stores each filtered row segment into the FFT buffer of the CTA that
//      owns the row's block (st.async into distributed shared memory, 16
//      bytes per channel pair, completion counted in bytes on the owner's
//      mbarrier, so no cluster-wide fence is needed);
//   3. once its own buffer holds all N channels of its RB rows, takes their
//      N-point DFTs (Section 2) with Stockham passes in place and stores the
//      spectra;
//   4. right after the last pass has read the buffer, arrives on every CTA's
//      "buffer free" mbarrier so the next round's segments may land.
// Input is read from HBM once; filtered rows cross the cluster once and never
// reach HBM.  Unlike the four-step cluster kernel no transform is split
// across CTAs, so there is no twiddle stage and no second exchange.
#pragma once

#include <type_traits>

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"
#include "ppf_ring.cuh"

namespace ppf {

template <int N_, int T_, class In_, int P_, int NT_, int RB_, int NCH_, int MINB_ = 1, class OT_ = float2,
          int NXB_ = 1>
struct GatherCfg {
    using OT = OT_;  // output bin: float2 (complex64) or BinF16
    using In = In_;
    using raw = typename In::raw;
    using coef_t = typename Coef<In>::type;
    static constexpr int N = N_, T = T_, P = P_, NT = NT_, RB = RB_, NCH = NCH_;
    static constexpr int MINB = MINB_;  // CTAs per SM the tile is built for
    // FFT buffers per CTA: 1, or 2 (pipelined: round k+1 is filtered and sent
    // into one buffer while round k is transformed in the other; the first
    // pass's padding is halved, PD = 2, and the ring may be one chunk shorter
    // so that both buffers fit)
    static constexpr int NXB = NXB_;
    static constexpr int PD = NXB_ == 2 ? 2 : 1;
    static constexpr int BPS = In::bytes;
    static constexpr int NC = N / P;                     // channels per CTA
    static constexpr int ROWS = P * RB;                  // spectra per round = input rows per ring chunk
    static constexpr int UNITS = NC / 2;                 // FIR units (channel pairs) per row
    static constexpr int G = UNITS > NT ? UNITS / NT : 1;
    static constexpr int RG = UNITS >= NT ? 1 : NT / UNITS;
    static constexpr int RBT = ROWS / RG;                // spectra per thread per round
    static constexpr int KO = T >= 2 ? (T - 2) / ROWS + 1 : 0;
    static constexpr int RING_ROWS = NCH * ROWS;
    static constexpr int SEG_BYTES = NC * BPS;           // one input row's slice
    static constexpr int CHUNK_BYTES = ROWS * SEG_BYTES;
    static constexpr int RING_BYTES = NCH * CHUNK_BYTES;
    static constexpr int RS = PD == 1 ? fft_row_stride(N) : N + (N / 32 > 2 ? N / 32 : 2);
    static constexpr int X_SLOTS = RB * RS;              // one FFT buffer
    static constexpr int XBYTES = RB * N * 8;            // bytes a buffer receives per round
    static constexpr int SMEM = RING_BYTES + NXB * X_SLOTS * 8 + (NCH + 2 * NXB) * 8;
    static_assert(P >= 2 && P <= 8, "portable cluster sizes");
    static_assert(N % (2 * P) == 0 && SEG_BYTES % 16 == 0, "16-byte row slices");
    static_assert(UNITS % NT == 0 || NT % UNITS == 0, "FIR units must tile the threads");
    static_assert(ROWS % RG == 0 && RBT >= 1, "spectra per round must split over row groups");
    // one chunk in flight beyond the round's window; with two buffers the
    // refill of a slot overlaps the FFT of the previous round instead
    static_assert(NCH >= KO + 3 - NXB, "ring must hold a round's window plus one chunk in flight");
    static_assert(NXB == 1 || NXB == 2, "one or two FFT buffers");
    static_assert(RS % 2 == 0, "16-byte aligned channel pairs in the FFT buffer");
    static_assert(XBYTES < (1 << 20), "mbarrier transaction count");
    static_assert(SMEM <= 232448, "shared memory per CTA");
};

template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB)
ppf_gather_kernel(const PpfWork wl, const float2* __restrict__ tw, int* __restrict__ err)
{
    constexpr int N = C::N, T = C::T, NT = C::NT, RB = C::RB, NCH = C::NCH, P = C::P;
    constexpr int G = C::G, RBT = C::RBT, BPS = C::BPS, RING_ROWS = C::RING_ROWS, NC = C::NC, ROWS = C::ROWS;
    using PV = typename Pair<typename C::In>::vec;
    using raw = typename C::raw;
    using coef_t = typename C::coef_t;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    float2* X = reinterpret_cast<float2*>(smem + C::RING_BYTES);  // the FFT buffer(s)
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::RING_BYTES + C::NXB * C::X_SLOTS * 8);
    uint64_t* xfull = bars + NCH;            // [NXB] every byte of this CTA's buffer has arrived
    uint64_t* xfree = bars + NCH + C::NXB;   // [NXB] every owner has finished reading its buffer

    const int tid = threadIdx.x;
    const int rank = (int)cluster_ctarank();
    const int cid = blockIdx.x / P, ncl = gridDim.x / P;

    if (tid == 0) {
        for (int i = 0; i < NCH; ++i) mbar_init(&bars[i], 1);
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
    const uint64_t policy = l2_evict_first_policy();

    // FIR ownership: unit pp is the channel pair (2pp, 2pp+1) of this CTA's slice
    const int rg = C::UNITS >= NT ? 0 : tid / C::UNITS;
    const int pbase = C::UNITS >= NT ? tid : tid % C::UNITS;
    const int i0 = rg * RBT;
    PassTwiddlesR<N, NT, 16> twr;
    twr.load(tw);
    const uint32_t xbase = smem_u32(X), fullbase = smem_u32(xfull), freebase = smem_u32(xfree);

    int cbase = 0;  // ring chunks this CTA issued in earlier items (slots and phases continue)
    int gbase = 0;  // rounds this cluster ran in earlier items (mbarrier phases continue)
    bool failed = false;
    // Every CTA of a cluster walks the same items, so the cluster keeps one
    // schedule of rounds and nobody waits on a CTA that has moved on.
    const int n_items = work_items(wl);
    for (int it = cid;; it += ncl) {
        PpfJob job;
        int64_t blo, bhi;  // rounds
        if (wl.items == nullptr) {
            if (it != cid) break;
            job = wl.one;
            const int64_t nround = (job.S + ROWS - 1) / ROWS;
            blo = nround * cid / ncl;
            bhi = nround * (cid + 1) / ncl;
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
        const int nr = (int)(bhi - blo);
        const int64_t s_lo = blo * ROWS;
        const int64_t s_hi = S < bhi * ROWS ? S : bhi * ROWS;
        const int64_t in_end = s_hi + T - 1;  // input rows the item reads: [s_lo, in_end)
        const int nchunks = (int)((in_end - s_lo + ROWS - 1) / ROWS);

        int issued = 0;  // chunks of this item issued so far (meaningful in thread 0)
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
        };
        if (tid == 0 && !failed) {
            const int first = nchunks < NCH ? nchunks : NCH;
            for (int k = 0; k < first; ++k) issue(k);
            issued = first;
        }

        // coefficients of the owned channel pairs, in registers for the whole item
        // (channel pairs with G*T <= 32 and at least 4 spectra per thread, of
        // any input type, keep each coefficient as (h, h) so that one packed
        // FMA updates a complex accumulator -- bitwise the scalar result;
        // otherwise FP16 and int8 input keep each tap's coefficients as one
        // FP16 pair and multiply FP16 samples directly, int8 turned into FP16
        // exactly: fma_f16_pair, f16_pairs)
        constexpr bool PK = G * T <= 32 && RBT >= 4;
        constexpr bool MIX = !PK && !std::is_same<typename C::In, InC32>::value;
        float hr[MIX || PK ? 1 : G][MIX || PK ? 1 : T][2];
        float2 hp[PK ? G : 1][PK ? T : 1][2];
        uint32_t hq[MIX ? G : 1][MIX ? T : 1];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int c = rank * NC + 2 * (pbase + g * NT);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                if constexpr (MIX) {
                    hq[g][t] = *reinterpret_cast<const uint32_t*>(h + t * N + c);
                } else if constexpr (PK) {
                    const float v0 = coef_f(h[t * N + c]), v1 = coef_f(h[t * N + c + 1]);
                    hp[g][t][0] = make_float2(v0, v0);
                    hp[g][t][1] = make_float2(v1, v1);
                } else {
                    hr[g][t][0] = coef_f(h[t * N + c]);
                    hr[g][t][1] = coef_f(h[t * N + c + 1]);
                }
            }
        }

        int waited = 0;
        // Round k: its filtered rows go to FFT buffer b of every owner; with one
        // buffer b = 0 and phase parities alternate per round, with two the
        // rounds alternate between the buffers and each buffer's phases
        // advance every second round.
        auto buf_of = [&](int gk) { return C::NXB == 1 ? 0 : (gk & 1); };
        auto phase_of = [&](int gk) { return (uint32_t)((C::NXB == 1 ? gk : (gk >> 1)) & 1); };
        auto fir_round = [&](int k) {
            const int gk = gbase + k;
            const int b = buf_of(gk);
            const int rrb = ((cbase + k) % NCH) * ROWS;
            // 1. the round needs chunks k .. k+KO; every thread waits itself
            //    (a failure spreads over the CTA at the barrier after the FIR)
            const int need = (k + C::KO < nchunks ? k + C::KO : nchunks - 1) + 1;
            for (; waited < need && !failed; ++waited) {
                const int gc = cbase + waited;
                if (!mbar_wait_bounded(&bars[gc % NCH], (uint32_t)((gc / NCH) & 1))) {
                    failed = true;
                    break;  // this chunk stays "not waited for": the drain below waits for it
                }
            }
            // every owner has finished reading buffer b in the round that used it
            // before (each thread waits before its own stores into the buffers;
            // with two buffers only right before the stores, so the FIR overlaps it)
            bool freed = C::NXB == 1 ? true : gk < 2;
            if constexpr (C::NXB == 1) {
                if (gk >= 1 && !failed && !mbar_wait_cluster_bounded(&xfree[0], phase_of(gk - 1))) failed = true;
            }
            if (tid == 0) mbar_arrive_expect_tx(&xfull[b], (uint32_t)C::XBYTES);
            // 2. FIR over the ring; row i of the round goes to CTA i / RB.
            //    With one row group the window starts at a chunk boundary:
            //    row u lies in the window's chunk u / ROWS at row u % ROWS, so
            //    the chunk bases are computed once per round and every load
            //    is a base plus a compile-time offset.
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
                if (!freed) {
                    if (!failed && !mbar_wait_cluster_bounded(&xfree[b], phase_of(gk - 2))) failed = true;
                    freed = true;
                }
                if (!failed) {
#pragma unroll
                    for (int i = 0; i < RBT; ++i) {
                        const int row = i0 + i, q = row / RB, rr = row % RB;
                        const uint32_t off = (uint32_t)((rr * C::RS + rank * NC + cl) * 8);
                        if (PPF_INBOUNDS(off + 16 <= (uint32_t)C::X_SLOTS * 8 && q < P))
                            st_async_f4(map_shared_rank(xbase + b * C::X_SLOTS * 8 + off, (uint32_t)q),
                                    make_float4(a0[i].x, a0[i].y, a1[i].x, a1[i].y),
                                    map_shared_rank(fullbase + b * 8, (uint32_t)q));
                    }
                }
            }
            // every thread's reads of chunk k are done: refill its slot
            if (__syncthreads_or(failed)) failed = true;
            if (tid == 0 && !failed && issued < nchunks && issued == k + NCH) {
                issue(issued);
                ++issued;
            }
        };
        auto fft_round = [&](int k) {
            const int gk = gbase + k;
            const int b = buf_of(gk);
            // 3. this CTA's block of the round: all N channels of its RB rows
            if (!failed && !mbar_wait_bounded(&xfull[b], phase_of(gk))) failed = true;
            const int64_t s0 = s_lo + (int64_t)k * ROWS + rank * RB;
            const int64_t left = s_hi - s0;
            const int rows = (int)(left < 0 ? 0 : (left < RB ? left : RB));
            fft_rows_ip<N, RB, NT, 16, C::RS, 0, C::PD>(X + b * C::X_SLOTS, twr, Y + (rows > 0 ? s0 : 0) * N,
                                                        rows, [&] {
                // 4. every thread's last read of the buffer is done: free it on every CTA
                if (tid < P) mbar_arrive_cluster(map_shared_rank(freebase + b * 8, (uint32_t)tid));
            });
        };
        if constexpr (C::NXB == 1) {
            for (int k = 0; k < nr; ++k) {
                fir_round(k);
                fft_round(k);
            }
        } else {
            // round k+1 is filtered and sent while round k's rows arrive
            if (nr > 0) fir_round(0);
            for (int k = 0; k < nr; ++k) {
                if (k + 1 < nr) fir_round(k + 1);
                fft_round(k);
            }
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
    const bool any_failed = __syncthreads_or(failed);
    // no CTA leaves while a peer may still store into its shared memory
    cluster_arrive_release();
    cluster_wait_acquire();
    if (any_failed && tid == 0) atomicExch(err, 1);
}

}  // namespace ppf
