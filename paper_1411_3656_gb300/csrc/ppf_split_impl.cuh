// Host side of the split kernel: cooperative launch, plan scratch, variants.
#pragma once

#include <cstdio>

#include "ppf_launch.h"
#include "ppf_split.cuh"

namespace ppf {
namespace split_detail {

constexpr size_t kCounterBytes = 4096;  // 2*P progress words per group (<= 2*304 ints), rounded

template <class C>
cudaError_t prepare_split(PlanView& p)
{
    cudaError_t e = cudaFuncSetAttribute(ppf_split_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ppf_split_kernel<C>, C::NT, C::SMEM);
    if (e != cudaSuccess) return e;
    const int groups = (occ * p.sms) / C::P;
    if (groups < 1) return cudaErrorInvalidConfiguration;
    p.grid_cap = groups * C::P;
    p.scratch_bytes = kCounterBytes + (size_t)groups * C::XROWS * C::N * sizeof(float2);
    return cudaSuccess;
}

template <class C>
cudaError_t launch_split(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    if (!p.scratch) return cudaErrorInvalidValue;
    const int64_t nblk = (S + C::RB - 1) / C::RB;
    const int64_t gcap = p.grid_cap / C::P;
    const int groups = (int)(nblk < gcap ? nblk : gcap);
    if (groups <= 0) return cudaSuccess;
    int* ctr = static_cast<int*>(p.scratch);
    float2* xbuf = reinterpret_cast<float2*>(static_cast<unsigned char*>(p.scratch) + kCounterBytes);
    cudaError_t e = cudaMemsetAsync(ctr, 0, 2 * sizeof(int) * C::P * groups, st);
    if (e != cudaSuccess) return e;
    PpfWork w{};
    w.one.x = in;
    w.one.Y = out;
    w.one.h = p.h;
    w.one.S = S;
    const float2* tw = p.tw;
    int* err = p.err;
    void* args[] = {(void*)&w, (void*)&tw, (void*)&xbuf, (void*)&ctr, (void*)&err};
    e = cudaLaunchCooperativeKernel((const void*)ppf_split_kernel<C>, dim3(groups * C::P), dim3(C::NT), args, C::SMEM,
                                    st);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class C>
KernelEntry entry()
{
    static char name[80];
    std::snprintf(name, sizeof(name), "split:p%d:nt%d:rb%d:nch%d", C::P, C::NT, C::RB, C::NCH);
    KernelEntry e;
    e.name = name;
    e.prepare = prepare_split<C>;
    e.launch = launch_split<C>;
    e.launch_work = nullptr;  // uses plan scratch: one job at a time
    e.rows_per_block = C::RB;
    e.cluster = C::P;
    return e;
}

}  // namespace split_detail
}  // namespace ppf

// PPF_SV(N, T, group size, threads, spectra per block, ring chunks): one split-kernel variant.
#define PPF_SV(NN, TT, P, NT, RB, NCH)                                                              \
    if (N == NN && T == TT) {                                                                       \
        if (idx == want && out) *out = split_detail::entry<SplitCfg<NN, TT, In, P, NT, RB, NCH>>(); \
        ++idx;                                                                                      \
    }
