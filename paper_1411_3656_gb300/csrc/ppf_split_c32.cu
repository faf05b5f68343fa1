// Split-kernel variants, complex64 input (large N*T; groups of co-resident CTAs).
#include "ppf_split_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_SV(512, 32, 2, 256, 8, 6)
    PPF_SV(1024, 8, 2, 256, 8, 3) PPF_SV(1024, 16, 2, 256, 8, 4) PPF_SV(1024, 32, 4, 256, 8, 6)
    PPF_SV(2048, 4, 4, 256, 8, 3) PPF_SV(2048, 8, 4, 256, 8, 3)
    PPF_SV(2048, 16, 4, 256, 8, 4) PPF_SV(2048, 16, 8, 256, 8, 4) PPF_SV(2048, 32, 8, 256, 8, 6)
    PPF_SV(4096, 4, 8, 256, 8, 3) PPF_SV(4096, 8, 8, 256, 8, 3)
    PPF_SV(4096, 16, 8, 256, 8, 4) PPF_SV(4096, 16, 16, 256, 8, 4) PPF_SV(4096, 32, 16, 256, 8, 6)
    return idx;
}

int split_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
