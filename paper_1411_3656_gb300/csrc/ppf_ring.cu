// Instantiations and host launchers of the TMA-ring fused PPF kernel.
#include "ppf_launch.h"
#include "ppf_ring.cuh"

namespace ppf {
namespace {

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
    ppf_ring_kernel<C><<<grid, C::NT, C::SMEM, st>>>(static_cast<const typename C::raw*>(in),
                                                      static_cast<const typename C::coef_t*>(p.h), p.tw, out, S,
                                                      p.err);
    note_launch();
    return cudaGetLastError();
}

template <class C>
KernelEntry entry()
{
    KernelEntry e;
    e.name = "ring";
    e.prepare = prepare_ring<C>;
    e.launch = launch_ring<C>;
    return e;
}

// (N, T) -> ring configuration <threads, rows per block, ring chunks>; shared
// memory stays under the 227 KB a CTA may use.
template <class In>
KernelEntry ring_for(int N, int T)
{
#define PPF_RING(NN, TT, NT, RB, NCH) \
    if (N == NN && T == TT) return entry<RingCfg<NN, TT, In, NT, RB, NCH>>();
    PPF_RING(256, 4, 256, 16, 4)
    PPF_RING(256, 8, 256, 16, 4)
    PPF_RING(256, 16, 256, 16, 4)
    PPF_RING(256, 32, 256, 16, 4)
    PPF_RING(512, 4, 256, 8, 4)
    PPF_RING(512, 8, 256, 8, 4)
    PPF_RING(512, 16, 256, 8, 4)
    PPF_RING(1024, 4, 256, 4, 4)
    PPF_RING(1024, 8, 256, 4, 4)
    PPF_RING(2048, 4, 256, 2, 4)
#undef PPF_RING
    return KernelEntry{};
}

}  // namespace

KernelEntry ring_entry(int N, int T, int dtype)
{
    switch (dtype) {
    case 0: return ring_for<InC32>(N, T);
    default: return KernelEntry{};
    }
}

}  // namespace ppf
