// Host launchers of the TMA-ring kernel and the variant table shared by the
// per-N translation units (each TU instantiates the variants of one N).
#pragma once

#include <type_traits>

#include <cstdio>

#include "ppf_launch.h"
#include "ppf_ring.cuh"

namespace ppf {
namespace ring_detail {

template <class C>
cudaError_t prepare_ring(PlanView& p)
{
    cudaError_t e = cudaFuncSetAttribute(ppf_ring_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ppf_ring_kernel<C>, C::NT, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    p.grid_cap = occ * p.sms;
    return cudaSuccess;
}

template <class C>
cudaError_t launch_ring(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    const int64_t nblk = (S + C::RB - 1) / C::RB;
    const int grid = (int)(nblk < p.grid_cap ? nblk : p.grid_cap);
    if (grid <= 0) return cudaSuccess;
    PpfWork w{};
    w.one.x = in;
    w.one.Y = out;
    w.one.h = p.h;
    w.one.S = S;
    ppf_ring_kernel<C><<<grid, C::NT, C::SMEM, st>>>(w, p.tw, p.err);
    note_launch();
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_ring_work(const PlanView& p, const PpfWork& w, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    ppf_ring_kernel<C><<<grid, C::NT, C::SMEM, st>>>(w, p.tw, p.err);
    note_launch();
    return cudaGetLastError();
}

template <class C>
KernelEntry entry()
{
    static char name[64];
    std::snprintf(name, sizeof(name), "ring:nt%d:rb%d:nch%d:b%d%s%s%s%s", C::NT, C::RB, C::NCH, C::MINB,
                  C::CPT == 1 ? ":c1" : "", C::R0 == 8 ? ":r8" : "", C::NBUF == 1 ? ":sb" : "",
                  std::is_same<typename C::OT, BinF16>::value ? ":f16" : "");
    KernelEntry e;
    e.name = name;
    e.prepare = prepare_ring<C>;
    e.launch = launch_ring<C>;
    e.launch_work = launch_ring_work<C>;
    e.rows_per_block = C::RB;
    e.cluster = 1;
    return e;
}

}  // namespace ring_detail
}  // namespace ppf

// Walk a variant list: PPF_RV(NN, TT, NT, RB, NCH, MINB) entries for one input type
// (a channel pair per FIR thread); PPF_RV1: the same with one channel per thread.
#define PPF_RV(NN, TT, NT, RB, NCH, MINB)                                                      \
    if (N == NN && T == TT) {                                                                  \
        if (idx == want && out) *out = ring_detail::entry<RingCfg<NN, TT, In, NT, RB, NCH, MINB>>(); \
        ++idx;                                                                                 \
    }
#define PPF_RV1(NN, TT, NT, RB, NCH, MINB)                                                     \
    if (N == NN && T == TT) {                                                                  \
        if (idx == want && out) *out = ring_detail::entry<RingCfg<NN, TT, In, NT, RB, NCH, MINB, 1>>(); \
        ++idx;                                                                                 \
    }
// PPF_RVF(N, T, threads, spectra per block, ring chunks, CTAs per SM, channels per
// FIR thread, first-pass radix): the FP16-output twin of a tile shape.
#define PPF_RVF(NN, TT, NT, RB, NCH, MINB, CPT, R0)                                                \
    if (N == NN && T == TT) {                                                                      \
        if (idx == want && out)                                                                    \
            *out = ring_detail::entry<RingCfg<NN, TT, In, NT, RB, NCH, MINB, CPT, BinF16, R0>>();  \
        ++idx;                                                                                     \
    }
// PPF_RV8(N, T, threads, spectra per block, ring chunks, CTAs per SM, channels per
// FIR thread): a tile shape whose FFT starts with a radix-8 pass.
#define PPF_RV8(NN, TT, NT, RB, NCH, MINB, CPT)                                                   \
    if (N == NN && T == TT) {                                                                     \
        if (idx == want && out)                                                                   \
            *out = ring_detail::entry<RingCfg<NN, TT, In, NT, RB, NCH, MINB, CPT, float2, 8>>();   \
        ++idx;                                                                                    \
    }
// PPF_RVS(N, T, threads, spectra per block, ring chunks, CTAs per SM, channels per
// FIR thread): a tile shape with one FFT buffer (passes in place); PPF_RVFS is
// its FP16-output twin.
#define PPF_RVS(NN, TT, NT, RB, NCH, MINB, CPT)                                                       \
    if (N == NN && T == TT) {                                                                         \
        if (idx == want && out)                                                                       \
            *out = ring_detail::entry<RingCfg<NN, TT, In, NT, RB, NCH, MINB, CPT, float2, 16, 1>>();   \
        ++idx;                                                                                        \
    }
#define PPF_RVFS(NN, TT, NT, RB, NCH, MINB, CPT)                                                      \
    if (N == NN && T == TT) {                                                                         \
        if (idx == want && out)                                                                       \
            *out = ring_detail::entry<RingCfg<NN, TT, In, NT, RB, NCH, MINB, CPT, BinF16, 16, 1>>();   \
        ++idx;                                                                                        \
    }
