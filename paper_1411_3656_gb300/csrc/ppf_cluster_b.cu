// Cluster-kernel variants for N = 4096 (complex64 input).
#include "ppf_cluster_impl.cuh"

namespace ppf {

template <class In>
static int cluster_variants_b(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_CV(4096, 4, 4, 64, 256, 4, 3, 1) PPF_CV(4096, 4, 8, 64, 256, 8, 3, 1)
    PPF_CV(4096, 8, 8, 64, 256, 4, 4, 1) PPF_CV(4096, 8, 8, 64, 256, 8, 3, 1) PPF_CV(4096, 8, 8, 64, 256, 4, 5, 1)
    PPF_CV(4096, 8, 8, 128, 256, 4, 5, 1) PPF_CV(4096, 8, 8, 128, 256, 8, 3, 1)
    PPF_CV(4096, 16, 8, 64, 256, 4, 6, 1) PPF_CV(4096, 16, 8, 128, 256, 4, 7, 1)
    PPF_CV(4096, 32, 8, 64, 256, 4, 10, 1) PPF_CV(4096, 32, 8, 128, 256, 4, 10, 1)
    return idx;
}

int cluster_variants_c32_b(int N, int T, int want, KernelEntry* out)
{
    return cluster_variants_b<InC32>(N, T, want, out);
}

}  // namespace ppf
