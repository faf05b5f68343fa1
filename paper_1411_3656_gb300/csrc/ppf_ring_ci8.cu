// Ring-kernel variants, int8 I/Q input: the complex64 shapes plus larger N*T that fit once rows are a quarter of the size.
#include "ppf_ring_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
#include "ppf_ring_table.inc"
    PPF_RV(512, 32, 256, 8, 6, 1) PPF_RV(512, 32, 256, 4, 10, 2) PPF_RV(1024, 8, 256, 4, 5, 2)
    PPF_RV(1024, 8, 256, 8, 4, 1) PPF_RV(1024, 16, 256, 4, 6, 1) PPF_RV(1024, 16, 256, 4, 7, 1)
    PPF_RV(1024, 32, 256, 4, 10, 1) PPF_RV(2048, 8, 256, 2, 6, 1) PPF_RV(2048, 8, 256, 4, 4, 1)
    PPF_RV(2048, 16, 256, 2, 10, 1)
    // one FFT buffer, rings that fit only with 2-byte samples
    PPF_RVS(4096, 8, 256, 2, 6, 1, 2) PPF_RVS(2048, 16, 256, 4, 6, 1, 2) PPF_RVS(1024, 32, 256, 8, 6, 1, 2)
#include "ppf_ring_reduced.inc"
    return idx;
}

int ring_variants_ci8(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InCI8>(N, T, want, out);
}

}  // namespace ppf
