// Warp-specialised kernel variants, FP16 and int8 I/Q input (FP16 h).
#include "ppf_ws_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    (void)N;
    (void)T;
    (void)want;
    (void)out;
    return idx;
}

int ws_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC16>(N, T, want, out);
}

int ws_variants_ci8(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InCI8>(N, T, want, out);
}

}  // namespace ppf
