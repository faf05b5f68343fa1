// Host side of the warp-specialised gather kernel: cluster launch, work-list
// launch and the variant list macro used by ppf_gws*.cu.
#pragma once

#include <cstdio>
#include <cstring>
#include <type_traits>

#include "ppf_gws.cuh"
#include "ppf_launch.h"

namespace ppf {
namespace gws_detail {

template <class C>
cudaLaunchConfig_t launch_config(int grid, cudaStream_t st, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(C::NT, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C::P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class C>
cudaError_t prepare_gws(PlanView& p)
{
    cudaError_t e = cudaFuncSetAttribute(ppf_gws_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    if constexpr (C::RF > 0) {
        // the register split draws on the launch pool: the kernel must have
        // been compiled with the full share, or the FIR warps' request
        // could never be granted
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, ppf_gws_kernel<C>);
        if (e != cudaSuccess) return e;
        if ((long)fa.numRegs * C::NT < (long)C::NF * C::RF + (long)C::NX * C::RX)
            return cudaErrorInvalidConfiguration;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config<C>(C::P * p.sms, nullptr, attr);
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, ppf_gws_kernel<C>, &cfg);
    if (e != cudaSuccess) return e;
    if (ncl < 1) return cudaErrorInvalidConfiguration;
    p.grid_cap = ncl * C::P;
    return cudaSuccess;
}

template <class C>
cudaError_t launch_gws(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    const int64_t nround = (S + C::ROWS - 1) / C::ROWS;
    const int64_t ncl_cap = p.grid_cap / C::P;
    const int ncl = (int)(nround < ncl_cap ? nround : ncl_cap);
    if (ncl <= 0) return cudaSuccess;
    PpfWork w{};
    w.one.x = in;
    w.one.Y = out;
    w.one.h = p.h;
    w.one.S = S;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config<C>(ncl * C::P, st, attr);
    cudaError_t e = cudaLaunchKernelEx(&cfg, ppf_gws_kernel<C>, w, p.tw, p.err);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_gws_work(const PlanView& p, const PpfWork& w, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config<C>(grid, st, attr);
    cudaError_t e = cudaLaunchKernelEx(&cfg, ppf_gws_kernel<C>, w, p.tw, p.err);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class C>
KernelEntry entry()
{
    static char name[112];
    char split[40] = "";
    if (C::RF > 0) std::snprintf(split, sizeof(split), ":r%d/%d", C::RF, C::RX);
    if (C::EARLY) std::snprintf(split + std::strlen(split), sizeof(split) - std::strlen(split), ":er");
    if (C::PF > 0) std::snprintf(split + std::strlen(split), sizeof(split) - std::strlen(split), ":pf%d", C::PF);
    std::snprintf(name, sizeof(name), "gws:p%d:nf%d:nx%d:rb%d:nch%d%s%s%s%s", C::P, C::NF, C::NX, C::RB, C::NCH,
                  C::NXB == 2 ? ":db" : "", C::PD == 2 ? ":pd2" : "", split,
                  std::is_same<typename C::OT, BinF16>::value ? ":f16" : "");
    KernelEntry e;
    e.name = name;
    e.prepare = prepare_gws<C>;
    e.launch = launch_gws<C>;
    e.launch_work = launch_gws_work<C>;
    e.rows_per_block = C::ROWS;  // work items count rounds of P*RB spectra
    e.cluster = C::P;
    return e;
}

}  // namespace gws_detail
}  // namespace ppf

// PPF_GWV(N, T, cluster size, FIR threads, FFT threads, spectra per CTA and
// round, ring chunks, FFT buffers, first-pass padding divisor): one tile shape
// of the input type `In` in scope; PPF_GWVF is its FP16-output twin.
#define PPF_GWV(NN, TT, P, NF, NX, RB, NCH, NXB, PD)                                                     \
    if (N == NN && T == TT) {                                                                            \
        if (idx == want && out)                                                                          \
            *out = gws_detail::entry<GwsCfg<NN, TT, In, P, NF, NX, RB, NCH, NXB, float2, PD>>();         \
        ++idx;                                                                                           \
    }
// PPF_GWVR: the same with a register split, FIR warpgroups at RF registers a
// thread and FFT warpgroups at RX (RF = 0: none), and the early ring refill
// when ER is 1.
#define PPF_GWVR(NN, TT, P, NF, NX, RB, NCH, NXB, PD, RF, RX, ER)                                        \
    if (N == NN && T == TT) {                                                                            \
        if (idx == want && out)                                                                          \
            *out = gws_detail::entry<GwsCfg<NN, TT, In, P, NF, NX, RB, NCH, NXB, float2, PD, RF, RX, ER>>(); \
        ++idx;                                                                                           \
    }
// PPF_GWVP: a PPF_GWVR tile shape with chunks prefetched into L2 PF chunks
// ahead of the ring copies; PPF_GWVPF its FP16-output twin.
#define PPF_GWVP(NN, TT, P, NF, NX, RB, NCH, NXB, PD, RF, RX, ER, PF)                                    \
    if (N == NN && T == TT) {                                                                            \
        if (idx == want && out)                                                                          \
            *out = gws_detail::entry<GwsCfg<NN, TT, In, P, NF, NX, RB, NCH, NXB, float2, PD, RF, RX, ER, PF>>(); \
        ++idx;                                                                                           \
    }
#define PPF_GWVPF(NN, TT, P, NF, NX, RB, NCH, NXB, PD, RF, RX, ER, PF)                                   \
    if (N == NN && T == TT) {                                                                            \
        if (idx == want && out)                                                                          \
            *out = gws_detail::entry<GwsCfg<NN, TT, In, P, NF, NX, RB, NCH, NXB, BinF16, PD, RF, RX, ER, PF>>(); \
        ++idx;                                                                                           \
    }
// PPF_GWVRF: the FP16-output twin of a PPF_GWVR tile shape.
#define PPF_GWVRF(NN, TT, P, NF, NX, RB, NCH, NXB, PD, RF, RX, ER)                                       \
    if (N == NN && T == TT) {                                                                            \
        if (idx == want && out)                                                                          \
            *out = gws_detail::entry<GwsCfg<NN, TT, In, P, NF, NX, RB, NCH, NXB, BinF16, PD, RF, RX, ER>>(); \
        ++idx;                                                                                           \
    }
#define PPF_GWVF(NN, TT, P, NF, NX, RB, NCH, NXB, PD)                                                    \
    if (N == NN && T == TT) {                                                                            \
        if (idx == want && out)                                                                          \
            *out = gws_detail::entry<GwsCfg<NN, TT, In, P, NF, NX, RB, NCH, NXB, BinF16, PD>>();         \
        ++idx;                                                                                           \
    }
