// Ring-kernel variants, FP16 I/Q input: the complex64 shapes plus larger N*T that fit once rows are half the size.
#include "ppf_ring_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
#include "ppf_ring_table.inc"
    PPF_RV(512, 32, 256, 8, 6, 1) PPF_RV(1024, 8, 256, 4, 5, 1) PPF_RV(1024, 16, 256, 4, 6, 1)
    PPF_RV(1024, 16, 256, 4, 7, 1) PPF_RV(2048, 8, 256, 2, 6, 1)
#include "ppf_ring_reduced.inc"
    return idx;
}

int ring_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC16>(N, T, want, out);
}

}  // namespace ppf
