// Ring-kernel variants for N = 1024 and N = 2048 (complex64 input).
#include "ppf_ring_impl.cuh"

namespace ppf {

template <class In>
static int ring_variants_large(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_RV(1024, 4, 256, 4, 4, 1) PPF_RV(1024, 4, 512, 4, 4, 1) PPF_RV(1024, 4, 256, 2, 4, 2)
    PPF_RV(1024, 8, 256, 4, 4, 1) PPF_RV(1024, 8, 512, 4, 4, 1)
    PPF_RV(2048, 4, 256, 2, 4, 1) PPF_RV(2048, 4, 512, 2, 4, 1)
    return idx;
}

int ring_variants_c32_large(int N, int T, int want, KernelEntry* out)
{
    return ring_variants_large<InC32>(N, T, want, out);
}

}  // namespace ppf
