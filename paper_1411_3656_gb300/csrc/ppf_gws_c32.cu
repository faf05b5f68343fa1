// Warp-specialised gather-kernel variants, complex64 input (N*T of 32K and
// more).  256 FIR threads (FP32 coefficient pairs, packed FMAs) and 256 FFT
// threads per CTA: at most 128 registers a thread.
#include "ppf_gws_impl.cuh"

namespace ppf {

template <class In>
static int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    // one FFT buffer (full first-pass padding) or two (halved padding where
    // needed to fit); one channel pair of the CTA's slice per FIR thread
    PPF_GWV(4096, 32, 8, 256, 256, 1, 6, 1, 1) PPF_GWV(4096, 32, 8, 256, 256, 1, 5, 2, 2)
    PPF_GWV(4096, 16, 8, 256, 256, 1, 4, 1, 1) PPF_GWV(4096, 16, 8, 256, 256, 1, 4, 2, 1)
    PPF_GWV(4096, 8, 4, 256, 256, 1, 4, 1, 1) PPF_GWV(4096, 8, 4, 256, 256, 1, 4, 2, 1)
    PPF_GWV(2048, 32, 4, 256, 256, 2, 6, 1, 1) PPF_GWV(2048, 32, 4, 256, 256, 2, 5, 2, 2)
    PPF_GWV(2048, 16, 4, 256, 256, 2, 4, 1, 1) PPF_GWV(2048, 16, 4, 256, 256, 2, 4, 2, 1)
    PPF_GWV(1024, 32, 2, 256, 256, 4, 6, 1, 1)
    // four channel pairs per FIR thread at T = 8
    PPF_GWV(4096, 8, 2, 256, 256, 1, 6, 1, 1)
    // register splits (T = 32): each role allocated on its own (128/128),
    // or the FIR warpgroups raised above the launch share
    PPF_GWVR(4096, 32, 8, 256, 256, 1, 6, 1, 1, 128, 128, 0) PPF_GWVR(4096, 32, 8, 256, 256, 1, 6, 1, 1, 136, 120, 0)
    PPF_GWVR(2048, 32, 4, 256, 256, 2, 6, 1, 1, 128, 128, 0) PPF_GWVR(1024, 32, 2, 256, 256, 4, 6, 1, 1, 128, 128, 0)
    // early ring refill
    PPF_GWVR(4096, 8, 4, 256, 256, 1, 4, 2, 1, 0, 0, 1) PPF_GWVR(4096, 16, 8, 256, 256, 1, 4, 2, 1, 0, 0, 1)
    PPF_GWVR(2048, 16, 4, 256, 256, 2, 4, 2, 1, 0, 0, 1)
    // chunks prefetched into L2 ahead of the ring copies
    PPF_GWVP(4096, 32, 8, 256, 256, 1, 6, 1, 1, 136, 120, 0, 2) PPF_GWVP(4096, 32, 8, 256, 256, 1, 6, 1, 1, 136, 120, 0, 4)
    PPF_GWVP(4096, 32, 8, 256, 256, 1, 6, 1, 1, 136, 120, 0, 8) PPF_GWVP(4096, 32, 8, 256, 256, 1, 5, 2, 2, 136, 120, 0, 4)
    PPF_GWVP(4096, 32, 8, 256, 256, 1, 5, 2, 2, 136, 120, 1, 4)
    PPF_GWVP(2048, 32, 4, 256, 256, 2, 6, 1, 1, 128, 128, 0, 4) PPF_GWVP(1024, 32, 2, 256, 256, 4, 6, 1, 1, 128, 128, 0, 4)
    PPF_GWVP(4096, 8, 4, 256, 256, 1, 4, 2, 1, 0, 0, 1, 4) PPF_GWVP(4096, 16, 8, 256, 256, 1, 4, 2, 1, 0, 0, 0, 4)
    PPF_GWVP(2048, 16, 4, 256, 256, 2, 4, 2, 1, 0, 0, 0, 4)
    return idx;
}

int gws_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_impl<InC32>(N, T, want, out);
}

// FP16-output twins of the tuned tile shapes (complex64 input).
template <class In>
static int variants_f16_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_GWVF(4096, 8, 4, 256, 256, 1, 4, 2, 1) PPF_GWVF(1024, 32, 2, 256, 256, 4, 6, 1, 1)
    PPF_GWVRF(4096, 8, 4, 256, 256, 1, 4, 2, 1, 0, 0, 1) PPF_GWVRF(4096, 32, 8, 256, 256, 1, 6, 1, 1, 136, 120, 0)
    PPF_GWVPF(4096, 32, 8, 256, 256, 1, 6, 1, 1, 136, 120, 0, 4) PPF_GWVPF(1024, 32, 2, 256, 256, 4, 6, 1, 1, 128, 128, 0, 4)
    PPF_GWVPF(4096, 8, 4, 256, 256, 1, 4, 2, 1, 0, 0, 1, 4)
    return idx;
}

int gws_variants_f16_c32(int N, int T, int want, KernelEntry* out)
{
    return variants_f16_impl<InC32>(N, T, want, out);
}

}  // namespace ppf
