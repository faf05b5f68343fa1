// Host launchers of the warp-specialised kernel and its variant macros (each
// input type's translation unit instantiates its own list).
#pragma once

#include <type_traits>

#include <cstdio>

#include "ppf_launch.h"
#include "ppf_ws.cuh"

namespace ppf {
namespace ws_detail {

template <class C>
cudaError_t prepare_ws(PlanView& p)
{
    cudaError_t e = cudaFuncSetAttribute(ppf_ws_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ppf_ws_kernel<C>, C::NT, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    p.grid_cap = occ * p.sms;
    return cudaSuccess;
}

template <class C>
cudaError_t launch_ws(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    const int64_t nblk = (S + C::RB - 1) / C::RB;
    const int grid = (int)(nblk < p.grid_cap ? nblk : p.grid_cap);
    if (grid <= 0) return cudaSuccess;
    PpfWork w{};
    w.one.x = in;
    w.one.Y = out;
    w.one.h = p.h;
    w.one.S = S;
    ppf_ws_kernel<C><<<grid, C::NT, C::SMEM, st>>>(w, p.tw, p.err);
    note_launch();
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_ws_work(const PlanView& p, const PpfWork& w, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    ppf_ws_kernel<C><<<grid, C::NT, C::SMEM, st>>>(w, p.tw, p.err);
    note_launch();
    return cudaGetLastError();
}

template <class C>
KernelEntry entry()
{
    static char name[64];
    std::snprintf(name, sizeof(name), "ws:nf%d:nx%d:rb%d:nch%d%s%s%s%s", C::NF, C::NX, C::RB, C::NCH,
                  C::CPT == 1 ? ":c1" : "", C::PD == 2 ? ":pd2" : "", C::RC == 32 ? ":r32" : "",
                  std::is_same<typename C::OT, BinF16>::value ? ":f16" : "");
    KernelEntry e;
    e.name = name;
    e.prepare = prepare_ws<C>;
    e.launch = launch_ws<C>;
    e.launch_work = launch_ws_work<C>;
    e.rows_per_block = C::RB;
    e.cluster = 1;
    return e;
}

}  // namespace ws_detail
}  // namespace ppf

// PPF_WV(N, T, FIR threads, FFT threads, spectra per block, ring chunks,
// channels per FIR thread, first-pass padding divisor): one tile shape of the
// input type `In` in scope.
#define PPF_WV(NN, TT, NF, NX, RB, NCH, CPT, PD)                                                    \
    if (N == NN && T == TT) {                                                                        \
        if (idx == want && out)                                                                      \
            *out = ws_detail::entry<WsCfg<NN, TT, In, NF, NX, RB, NCH, CPT, float2, PD>>();          \
        ++idx;                                                                                       \
    }
// PPF_WV32: the same with FFT passes of radix up to 32 (N = 512 or 1024 in two
// passes).
#define PPF_WV32(NN, TT, NF, NX, RB, NCH, CPT)                                                      \
    if (N == NN && T == TT) {                                                                       \
        if (idx == want && out)                                                                     \
            *out = ws_detail::entry<WsCfg<NN, TT, In, NF, NX, RB, NCH, CPT, float2, 1, 32>>();      \
        ++idx;                                                                                      \
    }
// PPF_WVF: the FP16-output twin of a tile shape (complex64 input).
#define PPF_WVF(NN, TT, NF, NX, RB, NCH, CPT, PD)                                                   \
    if (N == NN && T == TT) {                                                                        \
        if (idx == want && out)                                                                      \
            *out = ws_detail::entry<WsCfg<NN, TT, In, NF, NX, RB, NCH, CPT, BinF16, PD>>();          \
        ++idx;                                                                                       \
    }
