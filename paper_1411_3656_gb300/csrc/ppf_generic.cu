// Instantiations and host launchers of the general fused PPF kernel.
#include <type_traits>

#include "ppf_generic.cuh"
#include "ppf_launch.h"

namespace ppf {
namespace {

template <int N, class In, class OT>
cudaError_t prepare_generic(PlanView& p)
{
    auto kern = ppf_generic_kernel<N, In, typename Coef<In>::type, OT>;
    constexpr int smem = generic_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGenericThreads, smem);
    if (e != cudaSuccess) return e;
    p.grid_cap = (occ > 0 ? occ : 1) * p.sms;
    return cudaSuccess;
}

template <int N, class In, class OT>
cudaError_t launch_generic(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    constexpr int RB = generic_rows(N);
    const int64_t nblk = (S + RB - 1) / RB;
    const int grid = (int)(nblk < p.grid_cap ? nblk : p.grid_cap);
    if (grid <= 0) return cudaSuccess;
    ppf_generic_kernel<N, In, typename Coef<In>::type, OT><<<grid, kGenericThreads, generic_smem_bytes(N), st>>>(
        static_cast<const typename In::raw*>(in),
        static_cast<const typename Coef<In>::type*>(p.h), p.tw, reinterpret_cast<OT*>(out), p.T, S, p.fir_only);
    note_launch();
    return cudaGetLastError();
}

template <int N, class In, class OT>
KernelEntry make_entry()
{
    KernelEntry e;
    e.name = std::is_same<OT, BinF16>::value ? "generic:f16" : "generic";
    e.prepare = prepare_generic<N, In, OT>;
    e.launch = launch_generic<N, In, OT>;
    return e;
}

template <class In, class OT>
KernelEntry entry_for(int N)
{
    switch (N) {
    case 4: return make_entry<4, In, OT>();
    case 8: return make_entry<8, In, OT>();
    case 16: return make_entry<16, In, OT>();
    case 32: return make_entry<32, In, OT>();
    case 64: return make_entry<64, In, OT>();
    case 128: return make_entry<128, In, OT>();
    case 256: return make_entry<256, In, OT>();
    case 512: return make_entry<512, In, OT>();
    case 1024: return make_entry<1024, In, OT>();
    case 2048: return make_entry<2048, In, OT>();
    case 4096: return make_entry<4096, In, OT>();
    default: return KernelEntry{};
    }
}

}  // namespace

KernelEntry generic_entry(int N, int dtype, int out_f16)
{
    switch (dtype * 2 + (out_f16 ? 1 : 0)) {
    case 0: return entry_for<InC32, float2>(N);
    case 1: return entry_for<InC32, BinF16>(N);
    case 2: return entry_for<InC16, float2>(N);
    case 3: return entry_for<InC16, BinF16>(N);
    case 4: return entry_for<InCI8, float2>(N);
    case 5: return entry_for<InCI8, BinF16>(N);
    default: return KernelEntry{};
    }
}

}  // namespace ppf
