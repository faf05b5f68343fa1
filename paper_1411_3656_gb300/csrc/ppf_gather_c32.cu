// Gather-kernel variants, complex64 input (N*T of 32K and more).
#include "ppf_gather_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_GV(4096, 8, 2, 256, 1, 6, 1) PPF_GV(2048, 16, 2, 256, 2, 6, 1) PPF_GV(1024, 32, 2, 256, 4, 6, 1)
    PPF_GV(4096, 16, 4, 256, 1, 6, 1) PPF_GV(4096, 32, 8, 256, 1, 6, 1) PPF_GV(2048, 32, 4, 256, 2, 6, 1)
    // two FFT buffers per CTA: round k+1 filtered and sent while round k is transformed
    PPF_GV2(4096, 32, 8, 256, 1, 5, 1) PPF_GV2(2048, 32, 4, 256, 2, 5, 1) PPF_GV2(1024, 32, 2, 256, 4, 5, 1)
    PPF_GV2(4096, 16, 4, 256, 1, 5, 1) PPF_GV2(2048, 16, 2, 256, 2, 5, 1) PPF_GV2(4096, 8, 2, 256, 1, 5, 1)
    return idx;
}

int gather_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

// FP16-output twins of the tuned tile shapes (complex64 input).
template <class In>
static int variants_f16_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_GVF(4096, 8, 2, 256, 1, 6, 1) PPF_GVF(2048, 16, 2, 256, 2, 6, 1) PPF_GVF(1024, 32, 2, 256, 4, 6, 1)
    PPF_GVF(4096, 16, 4, 256, 1, 6, 1) PPF_GVF(4096, 32, 8, 256, 1, 6, 1) PPF_GVF(2048, 32, 4, 256, 2, 6, 1)
    PPF_GVF2(4096, 32, 8, 256, 1, 5, 1) PPF_GVF2(2048, 32, 4, 256, 2, 5, 1) PPF_GVF2(1024, 32, 2, 256, 4, 5, 1)
    PPF_GVF2(4096, 16, 4, 256, 1, 5, 1) PPF_GVF2(2048, 16, 2, 256, 2, 5, 1)
    return idx;
}

int gather_variants_f16_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_f16_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
