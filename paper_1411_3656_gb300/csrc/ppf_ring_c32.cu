// Ring-kernel variants, complex64 input.
#include "ppf_ring_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
#include "ppf_ring_table.inc"
    // one channel per FIR thread, packed f32x2 FMAs
    PPF_RV1(256, 8, 256, 16, 4, 1) PPF_RV1(256, 16, 256, 16, 4, 1)
    PPF_RV1(256, 32, 256, 16, 4, 1) PPF_RV1(256, 32, 256, 8, 6, 1)
    PPF_RV1(512, 8, 512, 8, 4, 1) PPF_RV1(512, 8, 256, 8, 4, 1)
    PPF_RV1(512, 16, 512, 8, 4, 1) PPF_RV1(512, 32, 512, 4, 10, 1)
    PPF_RV1(1024, 8, 512, 4, 4, 1) PPF_RV1(1024, 16, 512, 2, 10, 1)
    PPF_RV1(2048, 4, 512, 2, 4, 1)
    PPF_RV1(2048, 8, 512, 1, 9, 1) PPF_RV1(1024, 8, 512, 2, 6, 1) PPF_RV1(512, 16, 512, 4, 6, 1)
    // two CTAs per SM
    PPF_RV1(512, 8, 256, 4, 4, 2) PPF_RV1(1024, 4, 256, 2, 4, 2)
    PPF_RV1(256, 16, 256, 8, 4, 2) PPF_RV1(256, 8, 256, 8, 4, 2)
    // FFT starting with a radix-8 pass
    PPF_RV8(512, 8, 256, 4, 4, 2, 2) PPF_RV8(512, 16, 512, 8, 4, 1, 1) PPF_RV8(512, 32, 512, 4, 10, 1, 1)
    PPF_RV8(1024, 16, 512, 2, 10, 1, 1)
    // one FFT buffer: a ring long enough for 4096 x 4, or twice the spectra per block
    PPF_RVS(4096, 4, 256, 1, 5, 1, 2) PPF_RVS(4096, 4, 256, 1, 6, 1, 2)
    PPF_RVS(2048, 8, 256, 2, 6, 1, 2) PPF_RVS(1024, 16, 256, 4, 6, 1, 2) PPF_RVS(512, 32, 256, 8, 6, 1, 2)
    PPF_RVS(256, 32, 256, 16, 5, 1, 1)
    return idx;
}

int ring_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
