// Cluster-kernel variants, complex64 input.
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
    // one channel per FIR thread, packed f32x2 FMAs
    PPF_CV1(512, 32, 2, 32, 256, 8, 6, 1)
    PPF_CV1(1024, 16, 4, 64, 256, 8, 4, 1) PPF_CV1(1024, 16, 4, 32, 256, 8, 4, 1)
    PPF_CV1(1024, 32, 4, 64, 256, 4, 10, 1) PPF_CV1(1024, 32, 4, 32, 256, 8, 6, 1)
    PPF_CV1(2048, 8, 8, 64, 256, 8, 3, 1)
    PPF_CV1(2048, 16, 8, 64, 256, 8, 4, 1)
    PPF_CV1(2048, 32, 8, 64, 256, 4, 10, 1)
    // two CTAs per SM: one CTA's barriers and exchange waits overlap the other's work
    PPF_CV1(512, 32, 4, 32, 128, 4, 10, 2)
    PPF_CV(1024, 16, 4, 64, 128, 4, 6, 2) PPF_CV1(1024, 16, 4, 64, 128, 4, 6, 2)
    PPF_CV1(1024, 32, 8, 32, 128, 4, 10, 2) PPF_CV(1024, 32, 8, 32, 128, 4, 10, 2)
    PPF_CV1(2048, 8, 8, 64, 256, 4, 4, 2) PPF_CV(2048, 8, 8, 64, 128, 4, 4, 2)
    PPF_CV(2048, 16, 8, 64, 128, 4, 6, 2)
    PPF_CV(4096, 4, 8, 64, 128, 4, 3, 2)
    PPF_CV(4096, 8, 8, 64, 128, 2, 6, 2)
    PPF_CV(4096, 16, 8, 64, 128, 2, 10, 2)
    // stages starting with a radix-8 pass (every thread busy in the first pass)
    PPF_CV8(1024, 32, 4, 64, 256, 8, 6, 1) PPF_CV8(1024, 32, 4, 32, 256, 8, 6, 1)
    PPF_CV8(2048, 16, 4, 64, 256, 4, 6, 1) PPF_CV8(2048, 16, 8, 64, 128, 4, 6, 2)
    PPF_CV8(2048, 32, 8, 64, 128, 4, 10, 2)
    PPF_CV8(4096, 4, 4, 64, 256, 4, 3, 1) PPF_CV8(4096, 4, 8, 64, 128, 4, 3, 2)
    PPF_CV8(4096, 8, 8, 64, 128, 2, 6, 2) PPF_CV8(4096, 16, 8, 64, 128, 2, 10, 2)
    PPF_CV8(4096, 32, 8, 128, 256, 4, 10, 1) PPF_CV8(4096, 32, 8, 64, 256, 4, 10, 1)
    PPF_CV8(1024, 32, 4, 64, 128, 4, 10, 2)
    // 16-CTA clusters (non-portable size): 256 channels per CTA
    PPF_CV(4096, 32, 16, 64, 128, 4, 10, 2) PPF_CV1(4096, 32, 16, 64, 256, 8, 6, 1)
    PPF_CV1(4096, 32, 16, 64, 256, 4, 10, 1)
    PPF_CV(4096, 16, 16, 64, 128, 4, 6, 2) PPF_CV1(4096, 16, 16, 64, 256, 8, 4, 1)
    PPF_CV(4096, 8, 16, 64, 128, 4, 4, 2)
    PPF_CV(2048, 32, 16, 64, 128, 4, 10, 2)
    return idx;
}

int cluster_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
