// Host side of the FIR-only kernel (ppf_fir.cuh): tile shapes and launch.
#include <cstdio>

#include "ppf_fir.cuh"
#include "ppf_launch.h"

namespace ppf {
namespace {

template <class C>
cudaError_t prepare_fir(PlanView& p)
{
    cudaError_t e = cudaFuncSetAttribute(ppf_fir_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ppf_fir_kernel<C>, C::NT, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    p.grid_cap = occ * p.sms;
    return cudaSuccess;
}

template <class C>
cudaError_t launch_fir(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    if (S <= 0) return cudaSuccess;
    const int64_t nblk = (S + C::RB - 1) / C::RB;
    int bands = p.grid_cap / C::SLICES;
    if (bands < 1) bands = 1;
    if (bands > nblk) bands = (int)nblk;
    ppf_fir_kernel<C><<<bands * C::SLICES, C::NT, C::SMEM, st>>>(static_cast<const float2*>(in),
                                                                  static_cast<const float*>(p.h), out, S, p.err);
    note_launch();
    return cudaGetLastError();
}

template <int N, int T>
KernelEntry fir_entry_nt()
{
    constexpr int NC = N < 512 ? N : 512;
    constexpr int NT = 256;
    constexpr int RG = NC / 2 >= NT ? 1 : NT / (NC / 2);
    constexpr int RB = 8 * RG;
    constexpr int KO = T >= 2 ? (T - 2) / RB + 1 : 0;
    constexpr int NCH = KO + 2 > 3 ? KO + 2 : 3;
    using C = FirCfg<N, T, NC, NT, RB, NCH>;
    static char name[48];
    std::snprintf(name, sizeof(name), "fir:nc%d:rb%d:nch%d", NC, RB, NCH);
    KernelEntry e;
    e.name = name;
    e.prepare = prepare_fir<C>;
    e.launch = launch_fir<C>;
    e.rows_per_block = RB;
    return e;
}

template <int N>
KernelEntry fir_entry_n(int T)
{
    switch (T) {
    case 4: return fir_entry_nt<N, 4>();
    case 8: return fir_entry_nt<N, 8>();
    case 16: return fir_entry_nt<N, 16>();
    case 32: return fir_entry_nt<N, 32>();
    default: return KernelEntry{};
    }
}

}  // namespace

// The FIR-only kernel for (N, T) of complex64 input, or an empty entry (the
// general kernel's FIR-only mode serves every other size and input type).
KernelEntry fir_only_entry(int N, int T, int dtype)
{
    if (dtype != 0) return KernelEntry{};
    switch (N) {
    case 128: return fir_entry_n<128>(T);
    case 256: return fir_entry_n<256>(T);
    case 512: return fir_entry_n<512>(T);
    case 1024: return fir_entry_n<1024>(T);
    case 2048: return fir_entry_n<2048>(T);
    case 4096: return fir_entry_n<4096>(T);
    default: return KernelEntry{};
    }
}

}  // namespace ppf
