// FP16-output twins of the cluster-kernel tile shapes the complex64 sweep uses
// (complex64 input); see ppf_ring_f16.cu.
#include "ppf_cluster_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_CVF(2048, 32, 8, 64, 128, 4, 10, 2, 2, 8)
    return idx;
}

int cluster_variants_f16_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
