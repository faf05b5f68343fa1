// Cluster-kernel variants for N = 512, 1024 and 2048 (complex64 input).
#include "ppf_cluster_impl.cuh"

namespace ppf {

template <class In>
static int cluster_variants_a(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_CV(512, 32, 2, 32, 128, 8, 6, 1)
    PPF_CV(1024, 8, 2, 32, 256, 4, 4, 1) PPF_CV(1024, 8, 2, 32, 256, 4, 5, 1) PPF_CV(1024, 8, 4, 32, 256, 8, 3, 1)
    PPF_CV(1024, 16, 2, 32, 256, 4, 6, 1) PPF_CV(1024, 16, 4, 64, 256, 8, 4, 1) PPF_CV(1024, 16, 4, 32, 256, 8, 4, 1)
    PPF_CV(1024, 32, 4, 64, 256, 8, 6, 1)
    PPF_CV(2048, 8, 4, 64, 256, 4, 4, 1) PPF_CV(2048, 8, 4, 64, 256, 8, 3, 1) PPF_CV(2048, 8, 4, 64, 256, 4, 5, 1)
    PPF_CV(2048, 16, 4, 64, 256, 4, 6, 1) PPF_CV(2048, 16, 8, 64, 256, 8, 5, 1)
    PPF_CV(2048, 32, 8, 64, 256, 8, 6, 1) PPF_CV(2048, 32, 8, 64, 128, 4, 10, 2)
    return idx;
}

int cluster_variants_c32_a(int N, int T, int want, KernelEntry* out)
{
    return cluster_variants_a<InC32>(N, T, want, out);
}

}  // namespace ppf
