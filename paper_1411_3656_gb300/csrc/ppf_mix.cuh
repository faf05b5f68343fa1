// One persistent launch over streams of different N and T (complex64 input).
//
// Every CTA (one per SM) has the two warp-specialised roles of ppf_ws.cuh.
// The FIR warps walk the CTA's segment of work items -- (job, band of
// blocks), an equal share of the estimated work cut by the host --,
// dispatch on each job's tile shape, an index into the
// compile-time list MixShapes (N, T, spectra per block, ring chunks, channels
// per FIR thread), and for every block write the filtered rows into FFT
// buffer b mod 2 together with a record of what the FFT warps need (shape,
// output rows, twiddle table).  The FFT warps only follow the records:
// they switch to the record's shape (its pass twiddles stay in registers
// while consecutive blocks keep that shape), transform the rows and store the
// spectra.  A record with shape -1 ends the launch.  Shared memory holds the
// ring at the bottom and two FFT buffer slots, each as large as the largest
// shape's buffer, at the top; a shape's buffer lies at the end of its slot.
// Rings up to the slots' start never touch a buffer, so items of different
// shapes follow each other with no wait; the few rings that reach into slot 0
// (never into the shape's own buffer there) first wait until the FFT warps
// have finished every earlier block.
#pragma once

#include <tuple>
#include <type_traits>

#include "ppf_device.cuh"
#include "ppf_ptx.cuh"
#include "ppf_mix.h"
#include "ppf_ws.cuh"

namespace ppf {

// COST: the shape's time in this kernel for one second of 6.5 GB/s input
// (8.125e8 output samples), in microseconds, measured on a GB300 with one job
// per launch; the host cuts the work into equal-cost segments with it.
template <int N_, int T_, int RB_, int NCH_, int CPT_, int COST_, int PD_ = 1>
struct MixShape {
    static constexpr int N = N_, T = T_, RB = RB_, NCH = NCH_, CPT = CPT_, PD = PD_, COST = COST_;
};

// The tile shapes of the mixed kernel: every complex64 (N, T) with
// 128 <= N <= 2048 whose T-row window fits one SM (N*T <= 16K).
using MixShapeList = std::tuple<
    MixShape<128, 4, 32, 4, 2, 1990>, MixShape<128, 8, 32, 4, 2, 2010>, MixShape<128, 16, 32, 4, 2, 2320>,
    MixShape<128, 32, 32, 4, 2, 3180>,
    MixShape<256, 4, 16, 4, 2, 2000>, MixShape<256, 8, 16, 4, 2, 2000>, MixShape<256, 16, 16, 4, 2, 2130>,
    MixShape<256, 32, 16, 4, 1, 2910>,
    MixShape<512, 4, 8, 4, 2, 2156>, MixShape<512, 8, 8, 4, 2, 2185>, MixShape<512, 16, 8, 4, 2, 2451>,
    MixShape<512, 32, 4, 10, 2, 3694>,
    MixShape<1024, 4, 4, 4, 2, 2265>, MixShape<1024, 8, 4, 4, 2, 2335>, MixShape<1024, 16, 2, 10, 2, 3628>,
    MixShape<2048, 4, 2, 4, 2, 2353>, MixShape<2048, 8, 1, 9, 2, 3520>>;
constexpr int kMixShapes = (int)std::tuple_size<MixShapeList>::value;

// Launch geometry shared by every shape: [ring | slot 0 | slot 1 | records |
// mbarriers].
struct MixGeom {
    static constexpr int NF = 256, NX = 128, NT = NF + NX;
    static constexpr int NCHMAX = 10;
    static constexpr int BUF_BYTES = 34816;   // the largest RB * RS * 8 (RB * N = 4096, RS = N + N/16)
    static constexpr int TAIL = 2 * 32 + NCHMAX * 8 + 16;
    static constexpr int SMEM = 232448;
    static constexpr int SLOT0 = SMEM - TAIL - 2 * BUF_BYTES;  // = the largest ring that needs no wait
    static constexpr int REC_OFF = SLOT0 + 2 * BUF_BYTES;
    static_assert(SLOT0 % 16 == 0 && REC_OFF % 16 == 0, "16-byte aligned regions");
};

// A shape's configuration inside the mixed kernel (the ws layout with the
// shared geometry).
template <class Sh>
struct MixCfg : WsCfg<Sh::N, Sh::T, InC32, MixGeom::NF, MixGeom::NX, Sh::RB, Sh::NCH, Sh::CPT, float2, Sh::PD> {
    using Base = WsCfg<Sh::N, Sh::T, InC32, MixGeom::NF, MixGeom::NX, Sh::RB, Sh::NCH, Sh::CPT, float2, Sh::PD>;
    // a ring beyond slot 0's start drains the FFT warps first
    static constexpr bool DRAIN = Base::RING_BYTES > MixGeom::SLOT0;
    static_assert(Base::BUF_SLOTS * 8 <= MixGeom::BUF_BYTES, "FFT buffer larger than the mixed kernel's");
    static_assert(Base::RING_BYTES <= MixGeom::SLOT0 + MixGeom::BUF_BYTES - Base::BUF_SLOTS * 8,
                  "ring overlaps the shape's own buffer in slot 0");
    static_assert(Sh::NCH <= MixGeom::NCHMAX, "more ring chunks than mbarriers");
};

// Start of a shape's FFT buffer j (RB * RS float2 at the end of slot j).
__device__ __forceinline__ float2* mix_buf(unsigned char* smem, int j, int slots)
{
    return reinterpret_cast<float2*>(smem + MixGeom::SLOT0 + (j + 1) * MixGeom::BUF_BYTES - slots * 8);
}

// The FIR warps wait (EMPTY named barriers, in block order) until the FFT
// warps have finished with every block before `upto`.
__device__ __forceinline__ void mix_consume_empty(int& emptied, int upto)
{
    for (; emptied < upto; ++emptied) nbar_sync(kBarEmpty0 + (emptied & 1), MixGeom::NT);
}

// What the FFT warps need for one block (written by FIR thread 0 next to
// the buffer, read after the FULL barrier).
struct MixRec {
    float2* Y;          // first output row of the block
    const float2* tw;   // the job's twiddles
    int rows;           // valid rows of the block
    int shape;          // MixShapes index, -1: no further block
    int rb;             // spectra per block of the shape (rows the FIR warps wrote)
    int ni;             // index of N in MixFftList
};
static_assert(sizeof(MixRec) == 32, "record size");

// Pass twiddles of the FFT warps for one N: in registers where a thread's
// butterflies need at most 16 distinct complex twiddles in a pass, else read
// per butterfly from the twiddle table (L1).
template <int N, int NX, int P = 1, bool ANY = (P < fft_npass(N))>
struct MixTwiddles {
    static constexpr int R = fft_radix(N, P);
    static constexpr int NS = fft_ns(N, P);
    static constexpr int BPR = N / R;
    static constexpr int J = NX >= BPR ? 1 : BPR / NX;
    static constexpr int JE = NX % NS == 0 ? 1 : J;  // distinct j mod NS over the thread's butterflies
    static constexpr bool REG = JE * (R - 1) <= 16;
    float2 w[REG ? JE : 1][REG ? R - 1 : 1];
    MixTwiddles<N, NX, P + 1> next;
    __device__ __forceinline__ void load(const float2* __restrict__ tw, int lt)
    {
        if constexpr (REG) {
            constexpr int step = N / (NS * R);
#pragma unroll
            for (int q = 0; q < JE; ++q) {
                const int k = ((lt + q * NX) % BPR) % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) w[q][r - 1] = __ldg(tw + k * r * step);
            }
        }
        next.load(tw, lt);
    }
    // twiddles of butterfly k of the thread (j = its index in the row)
    template <int Q>
    __device__ __forceinline__ void apply(const float2* __restrict__ tw, int k, int j, float2 (&v)[fft_radix(N, Q)]) const
    {
        if constexpr (Q == P) {
            if constexpr (REG) {
                apply_twiddles<R>(w[k % JE], v);
            } else {
                constexpr int step = N / (NS * R);
                const int kk = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + kk * r * step));
            }
        } else {
            next.template apply<Q>(tw, k, j, v);
        }
    }
};
template <int N, int NX, int P>
struct MixTwiddles<N, NX, P, false> {
    __device__ __forceinline__ void load(const float2* __restrict__, int) {}
    template <int Q, class V>
    __device__ __forceinline__ void apply(const float2* __restrict__, int, int, V&) const {}
};

// One Stockham pass in place (as ws_fft_pass, twiddles from MixTwiddles).
template <int N, int RB, int NX, int RS, int PD, int P>
__device__ __forceinline__ void mix_fft_pass(float2* buf, const MixTwiddles<N, NX>& twr, const float2* __restrict__ tw,
                                             float2* __restrict__ Yb, int rows, int rb, int lt, int empty_id)
{
    constexpr int R = fft_radix(N, P);
    constexpr int NS = fft_ns(N, P);
    constexpr bool LAST = (P == fft_npass(N) - 1);
    constexpr int IN_NS = P == 0 ? 0 : fft_ns(N, P - 1);
    constexpr int IN_R = P == 0 ? 1 : fft_radix(N, P - 1);
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
    if constexpr (LAST) nbar_arrive(empty_id, MixGeom::NT);  // the buffer may take the block after next
    else nbar_sync(kBarFft, NX);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int b = lt + k * NX;
        if (NB % NX == 0 || b < NB) {
            const int row = b / BPR, j = b % BPR;
            if constexpr (P > 0) twr.template apply<P>(tw, k, j, v[k]);
            dft<R>(v[k]);
            if constexpr (LAST) {
                if (row < rows) {
                    float2* o = Yb + (int64_t)row * N + j;
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

template <int N, int RB, int NX, int RS, int PD, int P = 0>
__device__ __forceinline__ void mix_fft_rows(float2* buf, const MixTwiddles<N, NX>& twr, const float2* __restrict__ tw,
                                             float2* __restrict__ Yb, int rows, int rb, int lt, int empty_id)
{
    if constexpr (P < fft_npass(N)) {
        mix_fft_pass<N, RB, NX, RS, PD, P>(buf, twr, tw, Yb, rows, rb, lt, empty_id);
        mix_fft_rows<N, RB, NX, RS, PD, P + 1>(buf, twr, tw, Yb, rows, rb, lt, empty_id);
    }
}

// The FFT warps' code depends only on N and the spectra per block: one path
// per (N, RB) pair of the shape list.
template <int N_, int RB_, int PD_>
struct MixFft {
    static constexpr int N = N_, RB = RB_, PD = PD_;
    static constexpr int RS = PD == 1 ? fft_row_stride(N) : N + (N / 32 > 2 ? N / 32 : 2);
    static_assert(RB * RS * 8 <= MixGeom::BUF_BYTES, "FFT buffer larger than the mixed kernel's");
};
using MixFftList = std::tuple<MixFft<128, 32, 1>, MixFft<256, 16, 1>, MixFft<512, 8, 1>, MixFft<512, 4, 1>,
                              MixFft<1024, 4, 1>, MixFft<1024, 2, 1>, MixFft<2048, 2, 1>, MixFft<2048, 1, 1>>;
constexpr int kMixFfts = (int)std::tuple_size<MixFftList>::value;

template <int I = 0>
__host__ __device__ constexpr int mix_fft_index(int N, int RB)
{
    if constexpr (I < kMixFfts) {
        using F = typename std::tuple_element<I, MixFftList>::type;
        return F::N == N && F::RB == RB ? I : mix_fft_index<I + 1>(N, RB);
    } else {
        return -1;
    }
}

// ------------------------------------------------------------------ FIR role
// Blocks [blo, bhi) of one job with shape C; the ring restarts at slot 0 (every
// chunk of the previous item has been waited for), `ph` holds each slot's
// phase parity.
template <class C>
__device__ __forceinline__ void mix_fir_item(const MixJob& job, int64_t blo, int64_t bhi, int shape,
                                             unsigned char* ring, MixRec* rec, uint64_t* bars, uint32_t& ph,
                                             int& gb, int& emptied, bool& failed)
{
    constexpr int N = C::N, T = C::T, NF = C::NF, RB = C::RB, NCH = C::NCH;
    constexpr int G = C::G, RBT = C::RBT, BPS = C::BPS, RING_ROWS = C::RING_ROWS, RS = C::RS;
    using PV = typename Pair<InC32>::vec;
    const int tid = threadIdx.x;
    const uint64_t policy = l2_evict_first_policy();
    const int rg = C::UNITS >= NF ? 0 : tid / C::UNITS;
    const int pbase = C::UNITS >= NF ? tid : tid % C::UNITS;
    const int i0 = rg * RBT;
    const float2* __restrict__ x = static_cast<const float2*>(job.x);
    const float* __restrict__ h = static_cast<const float*>(job.h);
    const int64_t S = job.S;
    const int nb = (int)(bhi - blo);
    const int64_t s_lo = blo * RB;
    const int64_t s_hi = S < bhi * RB ? S : bhi * RB;
    const int64_t in_end = s_hi + T - 1;
    const int nchunks = (int)((in_end - s_lo + RB - 1) / RB);
    // this ring reaches into slot 0: every earlier block leaves the buffers first
    if constexpr (C::DRAIN) mix_consume_empty(emptied, gb);

    int issued = 0;
    auto issue = [&](int k) {
        const int64_t r0 = s_lo + (int64_t)k * RB;
        const int64_t rows = in_end - r0 < RB ? in_end - r0 : RB;
        const uint32_t bytes = (uint32_t)(rows * N * BPS);
        const int slot = k % NCH;
        const bool ok = PPF_INBOUNDS((size_t)slot * C::CHUNK_BYTES + bytes <= (size_t)C::RING_BYTES);
        mbar_arrive_expect_tx(&bars[slot], ok ? bytes : 0u);
        if (ok) tma_load_1d(ring + slot * C::CHUNK_BYTES, x + r0 * N, bytes, &bars[slot], policy);
    };
    if (tid == 0 && !failed) {
        const int first = nchunks < NCH ? nchunks : NCH;
        for (int k = 0; k < first; ++k) issue(k);
        issued = first;
    }

    constexpr bool PK = C::CPT == 2 && G * T <= 32 && RBT >= 4;
    float hr[C::CPT == 2 && !PK ? G : 1][C::CPT == 2 && !PK ? T : 1][2];
    float2 hp[PK ? G : 1][PK ? T : 1][2];
    float2 hh[C::CPT == 1 ? G : 1][C::CPT == 1 ? T : 1];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int c = C::CPT * (pbase + g * NF);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if constexpr (PK) {
                const float v0 = h[t * N + c], v1 = h[t * N + c + 1];
                hp[g][t][0] = make_float2(v0, v0);
                hp[g][t][1] = make_float2(v1, v1);
            } else if constexpr (C::CPT == 2) {
                hr[g][t][0] = h[t * N + c];
                hr[g][t][1] = h[t * N + c + 1];
            } else {
                const float v = h[t * N + c];
                hh[g][t] = make_float2(v, v);
            }
        }
    }

    int waited = 0;
    int rrb = 0;
    for (int b = 0; b < nb; ++b, ++gb) {
        const int need = (b + C::KO < nchunks ? b + C::KO : nchunks - 1) + 1;
        for (; waited < need && !failed; ++waited) {
            const int slot = waited % NCH;
            if (!mbar_wait_bounded(&bars[slot], (ph >> slot) & 1u)) {
                failed = true;
                break;
            }
            ph ^= 1u << slot;
        }
        const int j = gb & 1;
        // the FFT warps have finished the block before last (buffer j)
        mix_consume_empty(emptied, gb - 1);
        float2* const fb = mix_buf(ring, j, C::BUF_SLOTS);
        constexpr int NW = (RBT + T - 2) / RB + 1;
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
                        float2 v0, v1;
                        Pair<InC32>::split(pv, v0, v1);
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
                        const float2 v = PPF_INBOUNDS(ro + sizeof(float2) <= (size_t)C::RING_BYTES)
                                             ? *reinterpret_cast<const float2*>(ring + ro)
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
        if (tid == 0) {
            const int64_t s0 = s_lo + (int64_t)b * RB;
            MixRec r;
            r.Y = job.Y + s0 * N;
            r.tw = job.tw;
            r.rows = (int)(s_hi - s0 < RB ? s_hi - s0 : RB);
            r.shape = shape;
            r.rb = RB;
            r.ni = mix_fft_index(N, RB);
            rec[j] = r;
        }
        nbar_arrive(kBarFull0 + j, C::NT);
        failed = nbar_sync_or(kBarFir, NF, failed);
        if (tid == 0 && !failed && issued < nchunks && issued == b + NCH) {
            issue(issued);
            ++issued;
        }
        rrb += RB;
        rrb = rrb >= RING_ROWS ? rrb - RING_ROWS : rrb;
    }
    if (failed && tid == 0) {
        for (int k = waited; k < issued; ++k) {
            const int slot = k % NCH;
            mbar_wait_bounded(&bars[slot], (ph >> slot) & 1u, kWaitLimitNs / 4);
            ph ^= 1u << slot;
        }
    }
}

template <int I = 0>
__device__ __forceinline__ void mix_fir_dispatch(int shape, const MixJob& job, int64_t blo, int64_t bhi,
                                                 unsigned char* ring, MixRec* rec, uint64_t* bars, uint32_t& ph,
                                                 int& gb, int& emptied, bool& failed)
{
    if constexpr (I < kMixShapes) {
        if (shape == I) {
            using Sh = typename std::tuple_element<I, MixShapeList>::type;
            mix_fir_item<MixCfg<Sh>>(job, blo, bhi, I, ring, rec, bars, ph, gb, emptied, failed);
        } else {
            mix_fir_dispatch<I + 1>(shape, job, blo, bhi, ring, rec, bars, ph, gb, emptied, failed);
        }
    }
}

__device__ __forceinline__ void mix_fir_role(const MixWork& w, unsigned char* ring, MixRec* rec, uint64_t* bars,
                                             int* __restrict__ err)
{
    const int tid = threadIdx.x;
    uint32_t ph = 0;
    int gb = 0;       // blocks handed to the FFT warps
    int emptied = 0;  // blocks the FFT warps are known to have finished
    bool failed = false;
    const int n_items = w.n_items_dev ? *w.n_items_dev : w.n_items;
    int* next_item = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(bars) + MixGeom::NCHMAX * 8);
    int par = 0;
    for (int it = blockIdx.x; it < n_items;) {
        // the CTA's next item, asked for now so the answer is there when this one ends
        int pref = 0;
        if (tid == 0) pref = (int)gridDim.x + atomicAdd(w.next, 1);
        const MixItem item = w.items[it];
        const MixJob job = w.jobs[item.job];
        if (item.blo < item.bhi && job.shape >= 0 && job.shape < kMixShapes)
            mix_fir_dispatch(job.shape, job, item.blo, item.bhi, ring, rec, bars, ph, gb, emptied, failed);
        if (tid == 0) next_item[par] = pref;
        nbar_sync(kBarFir, MixGeom::NF);
        it = next_item[par];
        par ^= 1;
    }
    // the end record (in the slot of block gb), then the EMPTY arrivals of
    // the blocks still outstanding
    const int j = gb & 1;
    mix_consume_empty(emptied, gb - 1);
    if (tid == 0) {
        MixRec r{};
        r.shape = -1;
        r.ni = -1;
        rec[j] = r;
    }
    nbar_arrive(kBarFull0 + j, MixGeom::NT);
    mix_consume_empty(emptied, gb);
    if (failed && tid == 0) atomicExch(err, 1);
}

// ------------------------------------------------------------------ FFT role
// Blocks of one FFT path from the record in hand until a record of another
// path (or the end record) arrives, returned in r with gb its block; the
// pass twiddles stay in registers meanwhile.
template <int I>
__device__ __forceinline__ void mix_fft_run(unsigned char* smem, const MixRec* rec, MixRec& r, int& gb)
{
    using F = typename std::tuple_element<I, MixFftList>::type;
    constexpr int N = F::N, NX = MixGeom::NX;
    const int lt = threadIdx.x - MixGeom::NF;
    MixTwiddles<N, NX> twr;
    const float2* tw = r.tw;
    twr.load(tw, lt);
    do {
        if (r.tw != tw) {  // another job: its own twiddle table (the same values)
            tw = r.tw;
            twr.load(tw, lt);
        }
        const int j = gb & 1;
        mix_fft_rows<N, F::RB, NX, F::RS, F::PD>(mix_buf(smem, j, F::RB * F::RS), twr, tw, r.Y, r.rows, r.rb, lt,
                                                 kBarEmpty0 + j);
        ++gb;
        const int jn = gb & 1;
        nbar_sync(kBarFull0 + jn, MixGeom::NT);
        r = rec[jn];
    } while (r.shape >= 0 && r.ni == I);
}

template <int I = 0>
__device__ __forceinline__ void mix_fft_dispatch(unsigned char* smem, const MixRec* rec, MixRec& r, int& gb)
{
    if constexpr (I < kMixFfts) {
        if (r.ni == I) mix_fft_run<I>(smem, rec, r, gb);
        else mix_fft_dispatch<I + 1>(smem, rec, r, gb);
    }
}

__device__ __forceinline__ void mix_fft_role(unsigned char* smem, const MixRec* rec)
{
    int gb = 0;
    nbar_sync(kBarFull0, MixGeom::NT);
    MixRec r = rec[0];
    while (r.shape >= 0 && r.ni >= 0 && r.ni < kMixFfts) mix_fft_dispatch(smem, rec, r, gb);
}

__global__ void __launch_bounds__(MixGeom::NT, 1) ppf_mix_kernel(const MixWork w, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    MixRec* rec = reinterpret_cast<MixRec*>(smem + MixGeom::REC_OFF);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + MixGeom::REC_OFF + 2 * sizeof(MixRec));
    if (threadIdx.x == 0) {
        for (int i = 0; i < MixGeom::NCHMAX; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x < MixGeom::NF) mix_fir_role(w, ring, rec, bars, err);
    else mix_fft_role(smem, rec);
}

}  // namespace ppf
