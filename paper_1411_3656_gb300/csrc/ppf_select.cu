// Kernel selection for a plan.  Every (N, T, dtype) has an ordered list of
// compiled variants of the specialised kernels; the default is the variant the
// autotuner measured fastest on GB300 (ppf_tuned.inc), else the first.  When no
// specialised variant exists the plan uses the general kernel, which handles
// every supported size.
#include "ppf.h"
#include "ppf_launch.h"

#include <cstdio>
#include <cstring>

namespace ppf {

int ring_variants_c32(int N, int T, int want, KernelEntry* out);
int ring_variants_c16(int N, int T, int want, KernelEntry* out);
int ring_variants_ci8(int N, int T, int want, KernelEntry* out);
int gather_variants_c32(int N, int T, int want, KernelEntry* out);
int gather_variants_c16(int N, int T, int want, KernelEntry* out);
int gather_variants_ci8(int N, int T, int want, KernelEntry* out);
int ws_variants_c32(int N, int T, int want, KernelEntry* out);
int ws_variants_c16(int N, int T, int want, KernelEntry* out);
int ws_variants_ci8(int N, int T, int want, KernelEntry* out);
int gws_variants_c32(int N, int T, int want, KernelEntry* out);
int gws_variants_c16(int N, int T, int want, KernelEntry* out);
int gws_variants_ci8(int N, int T, int want, KernelEntry* out);
int ring_variants_f16_c32(int N, int T, int want, KernelEntry* out);
int gather_variants_f16_c32(int N, int T, int want, KernelEntry* out);
int ws_variants_f16_c32(int N, int T, int want, KernelEntry* out);
int gws_variants_f16_c32(int N, int T, int want, KernelEntry* out);

using VariantFn = int (*)(int, int, int, KernelEntry*);

// Number of variants for (N, T, dtype); fills *out with variant `want` if it exists.
int variants(int N, int T, int dtype, int want, KernelEntry* out)
{
    static const VariantFn lists[3][4] = {
        {ring_variants_c32, gather_variants_c32, ws_variants_c32, gws_variants_c32},
        {ring_variants_c16, gather_variants_c16, ws_variants_c16, gws_variants_c16},
        {ring_variants_ci8, gather_variants_ci8, ws_variants_ci8, gws_variants_ci8}};
    if (dtype < 0 || dtype > 2) return 0;
    int n = 0;
    for (VariantFn f : lists[dtype]) {
        KernelEntry e;
        const int c = f(N, T, want - n, &e);
        if (want - n >= 0 && want - n < c && out) *out = e;
        n += c;
    }
    return n;
}

// Index of the variant named `name` for (N, T, dtype), or -1.
static int variant_by_name(int N, int T, int dtype, const char* name)
{
    const int n = variants(N, T, dtype, -1, nullptr);
    for (int i = 0; i < n; ++i) {
        KernelEntry e;
        variants(N, T, dtype, i, &e);
        if (e.name && std::strcmp(e.name, name) == 0) return i;
    }
    return -1;
}

static int tuned_variant(int N, int T, int dtype)
{
    // An entry names its tile shape; the recorded index is where the shape
    // stood when it was timed and serves only as a first guess.  A shape that
    // is no longer compiled falls back to variant 0.
#define PPF_TUNED(NN, TT, DT, V, NAME)                                                      \
    if (N == NN && T == TT && dtype == DT) {                                                \
        KernelEntry e;                                                                      \
        if (V < variants(N, T, dtype, -1, nullptr) && (variants(N, T, dtype, V, &e), true) && \
            e.name && std::strcmp(e.name, NAME) == 0)                                      \
            return V;                                                                       \
        const int byname = variant_by_name(N, T, dtype, NAME);                              \
        return byname >= 0 ? byname : 0;                                                    \
    }
#if __has_include("ppf_tuned.inc")
#include "ppf_tuned.inc"
#endif
#undef PPF_TUNED
    return 0;
}

// FP16-output twin of a tile shape: the variant named "<name>:f16" (complex64
// input only); an empty entry when none is compiled.
static KernelEntry f16_twin(int N, int T, int dtype, const char* name)
{
    static const VariantFn lists[] = {ring_variants_f16_c32, gather_variants_f16_c32, ws_variants_f16_c32,
                                      gws_variants_f16_c32};
    if (dtype != 0 || !name) return KernelEntry{};
    char want[112];
    std::snprintf(want, sizeof(want), "%s:f16", name);
    for (VariantFn f : lists) {
        const int c = f(N, T, -1, nullptr);
        for (int i = 0; i < c; ++i) {
            KernelEntry e;
            f(N, T, i, &e);
            if (e.name && std::strcmp(e.name, want) == 0) return e;
        }
    }
    return KernelEntry{};
}

KernelEntry select_fast_entry(int N, int T, int dtype, int variant, int out_f16)
{
    KernelEntry e;
    const int n = variants(N, T, dtype, -1, nullptr);
    if (n == 0) return KernelEntry{};
    int v = variant >= 0 ? variant : tuned_variant(N, T, dtype);
    if (v >= n) v = 0;
    variants(N, T, dtype, v, &e);
    return out_f16 ? f16_twin(N, T, dtype, e.name) : e;
}

}  // namespace ppf

extern "C" int ppf_variant_count(int N, int T, ppf_dtype_t dtype)
{
    return ppf::variants(N, T, (int)dtype, -1, nullptr);
}

extern "C" const char* ppf_variant_name(int N, int T, ppf_dtype_t dtype, int i)
{
    ppf::KernelEntry e;
    if (i < 0 || i >= ppf::variants(N, T, (int)dtype, -1, nullptr)) return nullptr;
    ppf::variants(N, T, (int)dtype, i, &e);
    return e.name;
}
