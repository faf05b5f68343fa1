// Gather-kernel variants for the reduced-precision inputs (FP16 and int8 I/Q) at
// N*T = 64K and more, where even their halved or quartered ring rows do not fit
// one SM (the single-buffer ring kernel covers N*T = 32K).
#include "ppf_gather_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_GV(4096, 16, 4, 256, 1, 6, 1) PPF_GV(4096, 16, 4, 256, 2, 4, 1)
    PPF_GV(2048, 32, 4, 256, 2, 6, 1) PPF_GV(4096, 32, 8, 256, 1, 6, 1)
    // two FFT buffers per CTA (pipelined rounds)
    PPF_GV2(4096, 16, 4, 256, 1, 6, 1) PPF_GV2(2048, 32, 4, 256, 2, 6, 1) PPF_GV2(4096, 32, 8, 256, 1, 6, 1)
    return idx;
}

int gather_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC16>(N, T, want, out);
}
int gather_variants_ci8(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InCI8>(N, T, want, out);
}

}  // namespace ppf
