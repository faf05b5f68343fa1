// Warp-specialised kernel variants, complex64 input.
#include "ppf_ws_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    // N = 256 (128 channel pairs): two row groups of FIR threads
    PPF_WV(256, 4, 256, 128, 16, 4, 2, 1) PPF_WV(256, 8, 256, 128, 16, 4, 2, 1)
    PPF_WV(256, 16, 256, 128, 16, 4, 2, 1) PPF_WV(256, 32, 256, 128, 16, 4, 1, 1)
    PPF_WV(256, 32, 256, 128, 16, 4, 2, 1)
    // N = 512
    PPF_WV(512, 4, 256, 128, 8, 4, 2, 1) PPF_WV(512, 8, 256, 128, 8, 4, 2, 1)
    PPF_WV(512, 16, 256, 128, 8, 4, 2, 1) PPF_WV(512, 32, 256, 128, 4, 10, 2, 1)
    PPF_WV(512, 32, 256, 128, 4, 10, 1, 1)
    // N = 1024
    PPF_WV(1024, 4, 256, 128, 4, 4, 2, 1) PPF_WV(1024, 8, 256, 128, 4, 4, 2, 1)
    PPF_WV(1024, 16, 256, 128, 2, 10, 2, 1)
    // N = 2048
    PPF_WV(2048, 4, 256, 128, 2, 4, 2, 1)     PPF_WV(2048, 8, 256, 128, 1, 9, 2, 1)
    // N = 4096: FFT threads a multiple of 256 (fixed pass twiddles)
    PPF_WV(4096, 4, 256, 256, 1, 5, 2, 2) PPF_WV(4096, 4, 128, 256, 1, 5, 2, 2)
    // radix-32 passes: N = 512 as 32 x 16, N = 1024 as 32 x 32
    PPF_WV32(512, 4, 256, 128, 8, 4, 2) PPF_WV32(512, 8, 256, 128, 8, 4, 2)
    PPF_WV32(512, 16, 256, 128, 8, 4, 2) PPF_WV32(512, 32, 256, 128, 4, 10, 2)
    PPF_WV32(1024, 4, 256, 128, 4, 4, 2) PPF_WV32(1024, 8, 256, 128, 4, 4, 2)
    PPF_WV32(1024, 16, 256, 64, 2, 10, 2)
    return idx;
}

int ws_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

// FP16-output twins of the tile shapes the sweep cells default to
int ws_variants_f16_c32(int N, int T, int want, KernelEntry* out)
{
    using In = InC32;
    int idx = 0;
    PPF_WVF(256, 4, 256, 128, 16, 4, 2, 1) PPF_WVF(256, 32, 256, 128, 16, 4, 1, 1)
    PPF_WVF(512, 8, 256, 128, 8, 4, 2, 1) PPF_WVF(512, 16, 256, 128, 8, 4, 2, 1)
    PPF_WVF(1024, 8, 256, 128, 4, 4, 2, 1) PPF_WVF(2048, 4, 256, 128, 2, 4, 2, 1)
    PPF_WVF(4096, 4, 256, 256, 1, 5, 2, 2)
    return idx;
}

}  // namespace ppf
