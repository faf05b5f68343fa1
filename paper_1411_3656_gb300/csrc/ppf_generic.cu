// Instantiations and host launchers of the general fused PPF kernel.
#include "ppf_generic.cuh"
#include "ppf_launch.h"

namespace ppf {
namespace {

template <int N, class In>
cudaError_t prepare_generic(PlanView& p)
{
    auto kern = ppf_generic_kernel<N, In>;
    constexpr int smem = generic_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGenericThreads, smem);
    if (e != cudaSuccess) return e;
    p.grid_cap = (occ > 0 ? occ : 1) * p.sms;
    return cudaSuccess;
}

template <int N, class In>
cudaError_t launch_generic(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    constexpr int RB = generic_rows(N);
    const int64_t nblk = (S + RB - 1) / RB;
    const int grid = (int)(nblk < p.grid_cap ? nblk : p.grid_cap);
    if (grid <= 0) return cudaSuccess;
    ppf_generic_kernel<N, In><<<grid, kGenericThreads, generic_smem_bytes(N), st>>>(
        static_cast<const typename In::raw*>(in),
        static_cast<const typename Coef<In>::type*>(p.h), p.tw, out, p.T, S, p.fir_only);
    note_launch();
    return cudaGetLastError();
}

template <int N, class In>
KernelEntry make_entry()
{
    KernelEntry e;
    e.name = "generic";
    e.prepare = prepare_generic<N, In>;
    e.launch = launch_generic<N, In>;
    return e;
}

template <class In>
KernelEntry entry_for(int N)
{
    switch (N) {
    case 4: return make_entry<4, In>();
    case 8: return make_entry<8, In>();
    case 16: return make_entry<16, In>();
    case 32: return make_entry<32, In>();
    case 64: return make_entry<64, In>();
    case 128: return make_entry<128, In>();
    case 256: return make_entry<256, In>();
    case 512: return make_entry<512, In>();
    case 1024: return make_entry<1024, In>();
    case 2048: return make_entry<2048, In>();
    case 4096: return make_entry<4096, In>();
    default: return KernelEntry{};
    }
}

}  // namespace

KernelEntry generic_entry(int N, int dtype)
{
    switch (dtype) {
    case 0: return entry_for<InC32>(N);
    case 1: return entry_for<InC16>(N);
    case 2: return entry_for<InCI8>(N);
    default: return KernelEntry{};
    }
}

}  // namespace ppf
