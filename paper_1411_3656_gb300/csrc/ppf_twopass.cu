// Host side of the two-pass kernels: chunk loop over plan scratch, variants.
#include <cstdio>

#include "ppf_launch.h"
#include "ppf_twopass.cuh"

namespace ppf {
namespace twopass_detail {

template <int T, class In, int RBT, int CW, int STEPS, int N, int CHUNK_MB>
struct Cfg {
    static constexpr int NT_FIR = 32 * CW;
    static constexpr int ROWS_CTA = RBT * STEPS;  // spectra per FIR CTA
    // spectra per chunk: CHUNK_MB of filtered rows, a multiple of the CTA tile
    static constexpr int64_t K = ((int64_t)CHUNK_MB * (1 << 20) / (N * 8)) / ROWS_CTA * ROWS_CTA;
    static constexpr int FFT_SMEM = generic_smem_bytes(N);
    static_assert(N % NT_FIR == 0, "whole channel tiles");
    static_assert(K >= ROWS_CTA, "chunk holds at least one CTA tile");
};

template <class C, int T, class In, int RBT, int CW, int STEPS, int N>
cudaError_t prepare(PlanView& p)
{
    cudaError_t e = cudaFuncSetAttribute(ppf_fftrows_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::FFT_SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ppf_fftrows_kernel<N>, kFftRowsThreads, C::FFT_SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    p.grid_cap = occ * p.sms;
    p.scratch_bytes = (size_t)C::K * N * sizeof(float2);
    return cudaSuccess;
}

template <class C, int T, class In, int RBT, int CW, int STEPS, int N>
cudaError_t launch(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    if (!p.scratch) return cudaErrorInvalidValue;
    using raw = typename In::raw;
    using coef_t = typename Coef<In>::type;
    const raw* x = static_cast<const raw*>(in);
    const coef_t* h = static_cast<const coef_t*>(p.h);
    float2* ybuf = static_cast<float2*>(p.scratch);
    for (int64_t s0 = 0; s0 < S; s0 += C::K) {
        const int64_t k = S - s0 < C::K ? S - s0 : C::K;
        const dim3 gf(N / C::NT_FIR, (unsigned)((k + C::ROWS_CTA - 1) / C::ROWS_CTA));
        // FIR-only test hook: the filtered rows go straight to the output
        float2* ydst = p.fir_only ? out + s0 * N : ybuf;
        ppf_fir_kernel<T, In, RBT, CW, STEPS><<<gf, C::NT_FIR, 0, st>>>(x + s0 * N, h, ydst, N, k);
        note_launch();
        if (p.fir_only) continue;
        const int64_t nblk = (k + generic_rows(N) - 1) / generic_rows(N);
        const int grid = (int)(nblk < p.grid_cap ? nblk : p.grid_cap);
        ppf_fftrows_kernel<N><<<grid, kFftRowsThreads, C::FFT_SMEM, st>>>(ybuf, p.tw, out + s0 * N, k);
        note_launch();
    }
    return cudaGetLastError();
}

template <int T, class In, int RBT, int CW, int STEPS, int N, int CHUNK_MB>
KernelEntry entry()
{
    using C = Cfg<T, In, RBT, CW, STEPS, N, CHUNK_MB>;
    static char name[64];
    std::snprintf(name, sizeof(name), "twopass:rbt%d:cw%d:st%d:chunk%dmb", RBT, CW, STEPS, CHUNK_MB);
    KernelEntry e;
    e.name = name;
    e.prepare = prepare<C, T, In, RBT, CW, STEPS, N>;
    e.launch = launch<C, T, In, RBT, CW, STEPS, N>;
    e.launch_work = nullptr;  // uses plan scratch: one job at a time
    e.rows_per_block = generic_rows(N);
    e.cluster = 1;
    return e;
}

// PPF_TV(N, T, spectra per thread step, warps across channels, steps per CTA, chunk MiB)
#define PPF_TV(NN, TT, RBT, CW, STEPS, MB)                                              \
    if (N == NN && T == TT) {                                                           \
        if (idx == want && out) *out = entry<TT, In, RBT, CW, STEPS, NN, MB>();          \
        ++idx;                                                                          \
    }

template <class In>
int variants_impl(int N, int T, int want, KernelEntry* out)
{
    int idx = 0;
    PPF_TV(512, 32, 8, 4, 8, 32)
    PPF_TV(1024, 16, 8, 4, 8, 32) PPF_TV(1024, 32, 8, 4, 8, 32)
    PPF_TV(2048, 8, 8, 4, 8, 32) PPF_TV(2048, 16, 8, 4, 8, 32) PPF_TV(2048, 32, 8, 4, 8, 32)
    PPF_TV(4096, 4, 8, 4, 8, 32) PPF_TV(4096, 8, 8, 4, 8, 32)
    PPF_TV(4096, 16, 8, 4, 8, 32) PPF_TV(4096, 16, 8, 4, 8, 64) PPF_TV(4096, 16, 8, 8, 8, 64)
    PPF_TV(4096, 32, 8, 4, 8, 32) PPF_TV(4096, 32, 8, 4, 16, 64) PPF_TV(4096, 32, 4, 4, 16, 64)
    return idx;
}

}  // namespace twopass_detail

int twopass_variants_c32(int N, int T, int want, KernelEntry* out)
{
    return twopass_detail::variants_impl<InC32>(N, T, want, out);
}
int twopass_variants_c16(int N, int T, int want, KernelEntry* out)
{
    return twopass_detail::variants_impl<InC16>(N, T, want, out);
}
int twopass_variants_ci8(int N, int T, int want, KernelEntry* out)
{
    return twopass_detail::variants_impl<InCI8>(N, T, want, out);
}

}  // namespace ppf
