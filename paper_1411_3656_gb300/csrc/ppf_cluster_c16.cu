// Cluster-kernel variants, FP16 I/Q input.
#include "ppf_cluster_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
#include "ppf_cluster_table.inc"
    return idx;
}

int cluster_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC16>(N, T, want, out);
}

}  // namespace ppf
