// Warp-specialised kernel variants, FP16 and int8 I/Q input (FP16 h).
#include "ppf_ws_impl.cuh"

namespace ppf {

// Rows of FP16 (4 bytes per sample) or int8 (2 bytes) input take half or a
// quarter of a complex64 row's ring space, so the shapes below hold more
// spectra per block than their complex64 counterparts, and the N*T = 32K
// windows (4096x8, 2048x16, 1024x32), which complex64 leaves to the cluster
// kernel, fit one SM.  FIR threads keep FP16 coefficient pairs (G*T
// registers) and multiply FP16 samples with the mixed-precision FMA.
template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    constexpr bool I8 = std::is_same<In, InCI8>::value;
    // N = 256
    PPF_WV(256, 4, 256, 128, 16, 4, 2, 1) PPF_WV(256, 8, 256, 128, 16, 4, 2, 1)
    PPF_WV(256, 16, 256, 128, 16, 4, 2, 1) PPF_WV(256, 32, 256, 128, 16, 4, 2, 1)
    // N = 512
    PPF_WV(512, 4, 256, 128, 8, 4, 2, 1) PPF_WV(512, 8, 256, 128, 8, 4, 2, 1)
    PPF_WV(512, 16, 256, 128, 8, 4, 2, 1) PPF_WV(512, 32, 256, 128, 8, 6, 2, 1)
    // N = 1024
    PPF_WV(1024, 4, 256, 128, 4, 4, 2, 1) PPF_WV(1024, 8, 256, 128, 4, 4, 2, 1)
    PPF_WV(1024, 16, 256, 128, 4, 6, 2, 1) PPF_WV(1024, 32, 256, 128, 4, 10, 2, 2)
    PPF_WV(1024, 32, 256, 128, 2, 18, 2, 2)
    // N = 2048
    PPF_WV(2048, 4, 256, 128, 2, 4, 2, 2) PPF_WV(2048, 8, 256, 128, 2, 6, 2, 2)
    PPF_WV(2048, 16, 256, 128, 2, 10, 2, 2) PPF_WV(2048, 16, 256, 128, 1, 17, 2, 2)
    // N = 4096: FFT threads a multiple of 256 (fixed pass twiddles)
    PPF_WV(4096, 4, 256, 256, 1, 5, 2, 2) PPF_WV(4096, 8, 256, 256, 1, 9, 2, 2)
    if constexpr (I8) {
        // int8 rows (8 KiB at N = 4096) leave room for deeper blocks
        PPF_WV(2048, 8, 256, 128, 2, 10, 2, 2)
    }
    // radix-32 passes: N = 512 as 32 x 16, N = 1024 as 32 x 32
    PPF_WV32(512, 4, 256, 128, 8, 4, 2) PPF_WV32(512, 8, 256, 128, 8, 4, 2)
    PPF_WV32(512, 16, 256, 128, 8, 4, 2) PPF_WV32(512, 32, 256, 128, 8, 6, 2)
    PPF_WV32(1024, 4, 256, 128, 4, 4, 2) PPF_WV32(1024, 8, 256, 128, 4, 4, 2)
    PPF_WV32(1024, 16, 256, 128, 4, 6, 2) PPF_WV32(1024, 32, 256, 64, 2, 18, 2)
    return idx;
}

int ws_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC16>(N, T, want, out);
}

int ws_variants_ci8(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InCI8>(N, T, want, out);
}

}  // namespace ppf
