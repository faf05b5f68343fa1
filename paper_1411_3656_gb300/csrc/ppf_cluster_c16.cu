// Cluster-kernel variants, FP16 I/Q input.
#include "ppf_cluster_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
#include "ppf_cluster_table.inc"
    // N1 = 32: longer output runs (K2 = N2/P consecutive bins), 32-byte input rows
    PPF_CV(4096, 4, 8, 32, 256, 4, 3, 1) PPF_CV(4096, 8, 8, 32, 256, 4, 4, 1)
    PPF_CV(4096, 16, 8, 32, 256, 4, 6, 1) PPF_CV(4096, 32, 8, 32, 256, 4, 10, 1)
    PPF_CV(2048, 8, 4, 32, 256, 4, 4, 1) PPF_CV(2048, 16, 4, 32, 256, 4, 6, 1)
#include "ppf_cluster_reduced.inc"
    return idx;
}

int cluster_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC16>(N, T, want, out);
}

}  // namespace ppf
