// Cluster-kernel variants, int8 I/Q input.
#include "ppf_cluster_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
#include "ppf_cluster_table.inc"
#include "ppf_cluster_reduced.inc"
    return idx;
}

int cluster_variants_ci8(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InCI8>(N, T, want, out);
}

}  // namespace ppf
