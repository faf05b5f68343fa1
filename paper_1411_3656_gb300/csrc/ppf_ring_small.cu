// Ring-kernel variants for N = 256 and N = 512 (complex64 input).
#include "ppf_ring_impl.cuh"

namespace ppf {

template <class In>
static int ring_variants_small(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    // N = 256: 128 channel pairs
    PPF_RV(256, 4, 256, 16, 4, 1) PPF_RV(256, 4, 256, 8, 4, 2) PPF_RV(256, 4, 512, 16, 4, 1)
    PPF_RV(256, 8, 256, 16, 4, 1) PPF_RV(256, 8, 256, 8, 4, 2) PPF_RV(256, 8, 512, 16, 4, 1)
    PPF_RV(256, 16, 256, 16, 4, 1) PPF_RV(256, 16, 256, 8, 4, 2) PPF_RV(256, 16, 512, 16, 4, 1)
    PPF_RV(256, 32, 256, 16, 4, 1) PPF_RV(256, 32, 256, 8, 6, 1) PPF_RV(256, 32, 512, 16, 4, 1)
    // N = 512: 256 channel pairs
    PPF_RV(512, 4, 256, 8, 4, 1) PPF_RV(512, 4, 256, 4, 3, 2) PPF_RV(512, 4, 512, 8, 4, 1)
    PPF_RV(512, 8, 256, 8, 4, 1) PPF_RV(512, 8, 256, 4, 4, 2) PPF_RV(512, 8, 512, 8, 4, 1)
    PPF_RV(512, 16, 256, 8, 4, 1) PPF_RV(512, 16, 512, 8, 4, 1)
    return idx;
}

int ring_variants_c32_small(int N, int T, int want, KernelEntry* out)
{
    return ring_variants_small<InC32>(N, T, want, out);
}

}  // namespace ppf
