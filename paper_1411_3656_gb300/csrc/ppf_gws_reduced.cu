// Warp-specialised gather-kernel variants, FP16 and int8 I/Q input (FP16 h):
// FIR threads keep FP16 coefficient pairs and multiply FP16 samples with the
// mixed-precision FMA.
#include "ppf_gws_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_GWV(4096, 32, 8, 256, 256, 1, 6, 1, 1) PPF_GWV(4096, 32, 8, 256, 256, 1, 6, 2, 1)
    PPF_GWV(4096, 16, 8, 256, 256, 1, 4, 2, 1) PPF_GWV(4096, 16, 4, 256, 256, 1, 6, 1, 1)
    PPF_GWV(2048, 32, 4, 256, 256, 2, 6, 1, 1) PPF_GWV(2048, 32, 4, 256, 256, 2, 6, 2, 1)
    PPF_GWV(1024, 32, 2, 256, 256, 4, 6, 1, 1) PPF_GWV(1024, 32, 2, 256, 256, 4, 6, 2, 1)
    PPF_GWV(2048, 16, 2, 256, 256, 2, 6, 2, 1) PPF_GWV(2048, 16, 4, 256, 256, 2, 4, 2, 1)
    PPF_GWV(4096, 8, 2, 256, 256, 1, 6, 2, 1) PPF_GWV(4096, 8, 4, 256, 256, 1, 4, 2, 1)
    // early ring refill
    PPF_GWVR(4096, 8, 2, 256, 256, 1, 6, 2, 1, 0, 0, 1) PPF_GWVR(4096, 8, 4, 256, 256, 1, 4, 2, 1, 0, 0, 1)
    PPF_GWVR(2048, 16, 2, 256, 256, 2, 6, 2, 1, 0, 0, 1) PPF_GWVR(4096, 16, 4, 256, 256, 1, 6, 1, 1, 0, 0, 1)
    return idx;
}

int gws_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC16>(N, T, want, out);
}

int gws_variants_ci8(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InCI8>(N, T, want, out);
}

}  // namespace ppf
