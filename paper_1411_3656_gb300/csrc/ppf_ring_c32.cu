// Ring-kernel variants, complex64 input.
#include "ppf_ring_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
#include "ppf_ring_table.inc"
    return idx;
}

int ring_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
