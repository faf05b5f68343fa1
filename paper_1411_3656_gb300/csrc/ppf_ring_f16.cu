// FP16-output twins of the ring-kernel tile shapes the complex64 sweep uses
// (complex64 input).  A plan made with PPF_FLAG_OUT_F16 runs the twin of the
// tile shape its complex64 counterpart would run, else the general kernel.
#include "ppf_ring_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_RVF(128, 4, 256, 32, 3, 1, 2, 16) PPF_RVF(128, 8, 256, 16, 3, 2, 2, 16)
    PPF_RVF(128, 16, 256, 16, 3, 2, 2, 16) PPF_RVF(128, 32, 256, 32, 4, 1, 2, 16)
    PPF_RVF(256, 4, 512, 16, 4, 1, 2, 16) PPF_RVF(256, 8, 256, 16, 4, 1, 1, 16)
    PPF_RVF(256, 16, 256, 8, 4, 2, 1, 16) PPF_RVF(256, 32, 256, 16, 4, 1, 1, 16)
    PPF_RVF(512, 4, 256, 4, 3, 2, 2, 16) PPF_RVF(512, 8, 256, 4, 4, 2, 2, 16)
    PPF_RVF(512, 16, 512, 8, 4, 1, 1, 16) PPF_RVFS(512, 32, 256, 8, 6, 1, 2)
    PPF_RVF(1024, 4, 256, 2, 4, 2, 2, 16) PPF_RVF(1024, 8, 256, 4, 4, 1, 2, 16)
    PPF_RVFS(1024, 16, 256, 4, 6, 1, 2)
    PPF_RVF(2048, 4, 512, 2, 4, 1, 1, 16) PPF_RVFS(2048, 8, 256, 2, 6, 1, 2)
    PPF_RVFS(4096, 4, 256, 1, 5, 1, 2)
    return idx;
}

int ring_variants_f16_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
