// Device building blocks of the fused polyphase filter bank (arXiv 1411.3656).
//
//  * complex helpers and the in-register forward DFT of R = 2..16 points;
//  * input decoders for complex64 / half2 / int8 I-Q storage;
//  * one Stockham autosort pass over rows held in shared memory.
//
// The FFT is the DFT stage of the PPF (Section 2: channels are DFT bins;
// Section 3 uses a standard forward FFT): forward sign, unnormalised, natural
// bin order.  A length-N row is transformed by passes of radix R_1, R_2, ...
// with N = R_1 * R_2 * ... .  Pass p has Ns = R_1 * ... * R_{p-1} (the length
// of the sub-transforms already done).  Butterfly j (0 <= j < N/R) of the pass
// reads elements j + r*N/R, multiplies element r by W_{Ns*R}^{(j mod Ns)*r},
// takes an R-point DFT and writes output q to (j div Ns)*Ns*R + (j mod Ns) +
// q*Ns.  After the last pass (Ns*R = N) the row holds the DFT in natural
// order; no bit reversal is needed.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>
#include <type_traits>

// ------------------------------------------------------------------ checked build
// A debug build of the same sources with -DPPF_CHECKED (the tests' stand-in
// for a memory checker) tests the index of every instrumented shared-memory
// and global access against the buffer it addresses before making it.  A
// violation is counted in the translation unit's ppf_check_count_d and the
// access is skipped, so a wrong index shows as a count
// (ppf_check_violations), not as a fault.  In the normal build PPF_INBOUNDS
// is the constant true and the checks compile to nothing.
#ifdef PPF_CHECKED
static __device__ unsigned long long ppf_check_count_d;
#define PPF_INBOUNDS(cond) ((cond) ? true : (atomicAdd(&ppf_check_count_d, 1ull), false))
namespace ppf {
void register_check_counter(unsigned long long (*read)(bool reset));
}
static unsigned long long ppf_read_check_count(bool reset)
{
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, ppf_check_count_d, sizeof(v)) != cudaSuccess) return ~0ull;
    if (reset) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(ppf_check_count_d, &z, sizeof(z));
    }
    return v;
}
static const bool ppf_check_counter_registered = (ppf::register_check_counter(ppf_read_check_count), true);
#else
#define PPF_INBOUNDS(cond) true
#endif

namespace ppf {

// ------------------------------------------------------------------ complex
// Packed FP32 pair arithmetic (sm_100+ f32x2): one instruction per complex
// add/sub/multiply-add, each lane an ordinary round-to-nearest FP32 operation,
// so results are bitwise those of the scalar form.
__device__ __forceinline__ unsigned long long pk2(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
// (h, h) * x + acc for a real coefficient pair hh = (h, h) and complex x.
__device__ __forceinline__ float2 cfma_real(float2 hh, float2 x, float2 acc)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(hh)), "l"(pk2(x)), "l"(pk2(acc)));
    return upk2(d);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 w)
{
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * (-i)
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// cos(pi/8), sin(pi/8), cos(pi/4): exact mathematical constants rounded to float.
#define PPF_C8 0.92387953251128675613f
#define PPF_S8 0.38268343236508977173f
#define PPF_R2 0.70710678118654752440f

// a * W_16^m with W_16 = exp(-2*pi*i/16); m is a compile-time constant after
// unrolling, so the switch folds to the few instructions each case needs.
__device__ __forceinline__ float2 mul_w16(int m, float2 a)
{
    m &= 15;
    const bool neg = m >= 8;           // W^(m+8) = -W^m
    if (neg) m -= 8;
    float2 r;
    switch (m) {
    case 0: r = a; break;
    case 1: r = make_float2(fmaf(a.x, PPF_C8, a.y * PPF_S8), fmaf(a.y, PPF_C8, -a.x * PPF_S8)); break;
    case 2: r = make_float2((a.x + a.y) * PPF_R2, (a.y - a.x) * PPF_R2); break;
    case 3: r = make_float2(fmaf(a.x, PPF_S8, a.y * PPF_C8), fmaf(a.y, PPF_S8, -a.x * PPF_C8)); break;
    case 4: r = make_float2(a.y, -a.x); break;
    case 5: r = make_float2(fmaf(-a.x, PPF_S8, a.y * PPF_C8), fmaf(-a.y, PPF_S8, -a.x * PPF_C8)); break;
    case 6: r = make_float2((a.y - a.x) * PPF_R2, -(a.x + a.y) * PPF_R2); break;
    default: r = make_float2(fmaf(-a.x, PPF_C8, a.y * PPF_S8), fmaf(-a.y, PPF_C8, -a.x * PPF_S8)); break;
    }
    return neg ? make_float2(-r.x, -r.y) : r;
}

// a * W_32^m with W_32 = exp(-2*pi*i/32), m a compile-time constant: even m
// is W_16^(m/2); odd m is W_32^r (r = 1, 3, 5, 7: cos and sin of r*pi/16, the
// pairs of r and 8 - r swapped) turned by m / 8 quarter turns (-i each).
#define PPF_C16 0.98078528040323044913f  // cos(pi/16)
#define PPF_S16 0.19509032201612826785f  // sin(pi/16)
#define PPF_C316 0.83146961230254523708f  // cos(3*pi/16)
#define PPF_S316 0.55557023301960222474f  // sin(3*pi/16)
__device__ __forceinline__ float2 mul_w32(int m, float2 a)
{
    m &= 31;
    if ((m & 1) == 0) return mul_w16(m >> 1, a);
    const int q = m >> 3, r = m & 7;
    float c, sn;  // W_32^r = c - i*sn
    switch (r) {
    case 1: c = PPF_C16; sn = PPF_S16; break;
    case 3: c = PPF_C316; sn = PPF_S316; break;
    case 5: c = PPF_S316; sn = PPF_C316; break;
    default: c = PPF_S16; sn = PPF_C16; break;
    }
    float2 t = make_float2(fmaf(a.x, c, a.y * sn), fmaf(a.y, c, -a.x * sn));
    for (int i = 0; i < q; ++i) t = make_float2(t.y, -t.x);
    return t;
}

// In-register forward DFT of R points (R = 1, 2, 4, 8, 16, 32), natural order
// in and out: v[k] <- sum_r v[r] * W_R^{r*k}.  Radix-2 decimation in time
// over compile-time indices; the even/odd copies are register renames.
template <int R>
__device__ __forceinline__ void dft(float2 (&v)[R])
{
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const float2 t2 = cadd(v[1], v[3]), t3 = cmul_mi(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else {
        static_assert(R == 8 || R == 16 || R == 32, "radix must be 1, 2, 4, 8, 16 or 32");
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft<R / 2>(e);
        dft<R / 2>(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const float2 t = R == 32 ? mul_w32(k, o[k]) : mul_w16(k * (16 / R), o[k]);
            v[k] = cadd(e[k], t);
            v[k + R / 2] = csub(e[k], t);
        }
    }
}

// ------------------------------------------------------------------ inputs
// Storage types of the input samples.
struct InC32 { using raw = float2;  static constexpr int bytes = 8; };
struct InC16 { using raw = __half2; static constexpr int bytes = 4; };
struct InCI8 { using raw = char2;   static constexpr int bytes = 2; };

// int8 -> FP32 without a conversion instruction (conversions issue at a
// quarter of the FP32 rate).  With the byte flipped to u = b + 128 and placed
// under the exponent byte 0x4B, the word is the float 2^23 + u exactly (unit
// spacing at 2^23); subtracting 2^23 + 128 leaves b exactly.  The result is
// bitwise (float)b for every b; one byte permute per value and one packed
// subtract per (I, Q) pair.  `flipped` is the packed bytes XOR 0x80 in each.
__device__ __forceinline__ float2 s8x2_to_f32x2(uint32_t flipped, int k0)
{
    constexpr float kBias = 8388736.0f;  // 2^23 + 128
    const float i = __uint_as_float(__byte_perm(flipped, 0x4B000000u, 0x7440u | k0));
    const float q = __uint_as_float(__byte_perm(flipped, 0x4B000000u, 0x7440u | (k0 + 1)));
    return csub(make_float2(i, q), make_float2(kBias, kBias));
}

__device__ __forceinline__ float2 decode(float2 v) { return v; }
__device__ __forceinline__ float2 decode(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 decode(char2 v)
{
    const uint32_t w = (uint32_t)(uint8_t)v.x | ((uint32_t)(uint8_t)v.y << 8);
    return s8x2_to_f32x2(w ^ 0x8080u, 0);
}

// Two consecutive samples as one vector: 16 B (c32), 8 B (c16), 4 B (ci8).
template <class In> struct Pair;
template <> struct Pair<InC32> {
    using vec = float4;
    __device__ static void split(const vec& p, float2& a, float2& b) { a = make_float2(p.x, p.y); b = make_float2(p.z, p.w); }
};
template <> struct Pair<InC16> {
    using vec = uint2;
    __device__ static void split(const vec& p, float2& a, float2& b)
    {
        __half2 h0 = *reinterpret_cast<const __half2*>(&p.x);
        __half2 h1 = *reinterpret_cast<const __half2*>(&p.y);
        a = __half22float2(h0);
        b = __half22float2(h1);
    }
};
template <> struct Pair<InCI8> {
    using vec = char4;
    __device__ static void split(const vec& p, float2& a, float2& b)
    {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(&p) ^ 0x80808080u;
        a = s8x2_to_f32x2(w, 0);
        b = s8x2_to_f32x2(w, 2);
    }
};

// One FIR tap of a channel pair stored as FP16: h = (h0, h1) and the samples
// x = ((re0, im0), (re1, im1)) as FP16 pairs; a0 += h0 * x0, a1 += h1 * x1 per
// component with the mixed-precision FMA (FP16 operands, FP32 accumulator:
// the product of two FP16 values is exact in FP32 and the sum is rounded
// once), the value fmaf((float)h, (float)x, acc) gives, with no conversions.
__device__ __forceinline__ void fma_f16_pair(uint32_t hh, uint2 x, float2& a0, float2& a1)
{
    asm("{\n\t.reg .f16 h0, h1, r0, i0, r1, i1;\n\t"
        "mov.b32 {h0, h1}, %4;\n\t"
        "mov.b32 {r0, i0}, %5;\n\t"
        "mov.b32 {r1, i1}, %6;\n\t"
        "fma.rn.f32.f16 %0, h0, r0, %0;\n\t"
        "fma.rn.f32.f16 %1, h0, i0, %1;\n\t"
        "fma.rn.f32.f16 %2, h1, r1, %2;\n\t"
        "fma.rn.f32.f16 %3, h1, i1, %3;\n\t}"
        : "+f"(a0.x), "+f"(a0.y), "+f"(a1.x), "+f"(a1.y)
        : "r"(hh), "r"(x.x), "r"(x.y));
}

// Two stored samples as FP16 (I, Q) pairs for fma_f16_pair: FP16 storage as
// is; int8 exactly (with the byte flipped to u = b + 128 under the exponent
// byte 0x64 the FP16 word is 1024 + u, and subtracting 1152 leaves b).
__device__ __forceinline__ uint2 f16_pairs(uint2 p) { return p; }
__device__ __forceinline__ uint2 f16_pairs(char4 p)
{
    const uint32_t f = *reinterpret_cast<const uint32_t*>(&p) ^ 0x80808080u;
    const uint32_t w0 = __byte_perm(f, 0x64646464u, 0x4140u), w1 = __byte_perm(f, 0x64646464u, 0x4342u);
    uint2 r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r.x) : "r"(w0), "r"(0x64806480u));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r.y) : "r"(w1), "r"(0x64806480u));
    return r;
}

// Coefficient storage: FP32 for complex64 input, FP16 for the reduced types.
template <class In> struct Coef { using type = __half; };
template <> struct Coef<InC32> { using type = float; };
__device__ __forceinline__ float coef_f(float v) { return v; }
__device__ __forceinline__ float coef_f(__half v) { return __half2float(v); }

// ------------------------------------------------------------------ outputs
// Output bins are complex64 (float2), or FP16 (I, Q) pairs rounded to nearest
// (kept as their 32-bit pattern) for plans made with PPF_FLAG_OUT_F16.  The
// kernels take the bin type as a template parameter; stores stream past the
// caches (each output is written once).
struct BinF16 {
    uint32_t bits;
};
__device__ __forceinline__ void st_bin(float2* p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_bin(BinF16* p, float2 v)
{
    const __half2 hv = __float22half2_rn(v);
    __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<const unsigned*>(&hv));
}

// ------------------------------------------------------------------ work lists
// One job of a launch: a contiguous input stream (S + T - 1 rows of N samples),
// its S output spectra and its coefficients (each stream may have its own h).
struct PpfJob {
    const void* x;
    float2* Y;
    const void* h;
    int64_t S;
};
// A work item: blocks [blo, bhi) of job `job` (a block is the kernel's RB spectra).
struct PpfItem {
    int job;
    int pad;
    int64_t blo;
    int64_t bhi;
};
// Where a launch's work comes from.  With items == nullptr the launch has the
// one job `one`, split into equal contiguous bands over the grid; otherwise
// CTA (or cluster) i processes items i, i + grid, i + 2*grid, ...
struct PpfWork {
    PpfJob one;
    const PpfJob* jobs;
    const PpfItem* items;
    int n_items;
    // when set, the item count is read from device memory at kernel start
    // (a launch captured in a CUDA graph replays with new tables)
    const int* n_items_dev;
};
__device__ __forceinline__ int work_items(const PpfWork& wl)
{
    return wl.n_items_dev ? *wl.n_items_dev : wl.n_items;
}

// ------------------------------------------------------------------ FFT plan
// Radix of pass p for a length-N row: 16 first (or N itself when N <= 16),
// then 16s, the remainder last.  Every pass after the first has Ns >= 16.
__host__ __device__ constexpr int fft_npass(int N)
{
    int p = 0;
    for (int n = N; n > 1;) {
        const int r = n >= 16 ? 16 : n;
        n /= r;
        ++p;
    }
    return p;
}
__host__ __device__ constexpr int fft_radix(int N, int pass)
{
    int n = N;
    for (int p = 0;; ++p) {
        const int r = n >= 16 ? 16 : n;
        if (p == pass) return r;
        n /= r;
    }
}
__host__ __device__ constexpr int fft_ns(int N, int pass)
{
    int ns = 1;
    for (int p = 0; p < pass; ++p) ns *= fft_radix(N, p);
    return ns;
}

// The same plan with the first pass's radix capped at R0 (8, 16 or 32), the
// later passes' at RC (16 or 32), the remainder last: 64 = 8 x 8, 32 = 8 x 4,
// 128 = 8 x 16 for R0 = 8; 1024 = 32 x 32 and 512 = 32 x 16 for R0 = RC = 32.
// R0 = RC = 16 gives the plan above.
__host__ __device__ constexpr int fft_radix_r(int N, int pass, int R0, int RC = 16)
{
    int n = N;
    for (int p = 0;; ++p) {
        const int cap = p == 0 ? R0 : RC;
        const int r = n >= cap ? cap : n;
        if (p == pass) return r;
        n /= r;
    }
}
__host__ __device__ constexpr int fft_npass_r(int N, int R0, int RC = 16)
{
    int p = 0;
    for (int n = N; n > 1; ++p) n /= fft_radix_r(N, p, R0, RC);
    return p;
}
__host__ __device__ constexpr int fft_ns_r(int N, int pass, int R0, int RC = 16)
{
    int ns = 1;
    for (int p = 0; p < pass; ++p) ns *= fft_radix_r(N, p, R0, RC);
    return ns;
}

// Shared-memory row stride (in float2 slots) of the FFT buffer: N plus the
// padding of the first pass (one slot per 16 elements), at least 2 so that
// rows stay 16-byte aligned for vector stores.
__host__ __device__ constexpr int fft_row_stride(int N) { return N + (N / 16 > 2 ? N / 16 : 2); }

// Physical slot of logical element idx in a buffer written by a pass with
// parameters (NS, R).  With NS < 16 the writes of a half-warp would collide
// in the 16 eight-byte bank slots; padding NS slots after every NS*R
// elements spreads them over distinct slots while the next pass's reads (16
// consecutive elements from a 16-aligned start) stay contiguous.
// PD > 1 pads NS slots after every PD*NS*R elements instead (less room, at
// the price of PD-way conflicts in the writes of passes with NS < 16).
template <int NS, int R, int PD = 1>
__device__ __forceinline__ int pad_slot(int idx)
{
    if constexpr (NS >= 16 || NS * R < 2) return idx;
    else return idx + NS * (idx / (PD * NS * R));
}

// Slots from element j to element j + L of a buffer written by a pass (NS, R),
// for L a multiple of NS*R: the padding grows by L/R, so the R inputs of a
// butterfly (j + r*L) sit at fixed offsets from pad_slot(j) and their
// addresses need no per-element division.
template <int NS, int R, int L, int PD = 1>
__host__ __device__ constexpr int pad_stride()
{
    static_assert(NS >= 16 || NS * R < 2 || L % (PD * NS * R) == 0, "stride must span whole padding groups");
    return (NS >= 16 || NS * R < 2) ? L : L + L / (PD * R);
}

// Load the R inputs of butterfly j of a pass from row `row` of `buf`.
// InNS/InR describe the pass that wrote the buffer (InNS == 0: unpadded).
template <int N, int R, int InNS, int InR>
__device__ __forceinline__ void pass_load(const float2* buf, int row, int j, float2 (&v)[R])
{
    constexpr int RS = fft_row_stride(N);
    const float2* b = buf + row * RS;
    if constexpr (InNS == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = b[j + r * (N / R)];
    } else {
        const float2* bj = b + pad_slot<InNS, InR>(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = bj[r * pad_stride<InNS, InR, N / R>()];
    }
}

// Twiddle W_{NS*R}^{(j mod NS)*r} for r = 1..R-1 from the table tw[m] = W_N^m.
template <int N, int R, int NS>
__device__ __forceinline__ void pass_twiddle(const float2* __restrict__ tw, int j, float2 (&v)[R])
{
    if constexpr (NS > 1) {
        const int k = j % NS;
        constexpr int step = N / (NS * R);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[k * r * step]);
    }
}

// Twiddles of passes P.. of a length-N row for the butterfly index this thread
// keeps in every block (j = threadIdx.x mod N/R; fixed because the block's
// thread count is a multiple of N/R).  Loaded once per kernel into registers.
// R0 is the radix of the first pass (plan of fft_radix_r).
template <int N, int NT, int R0 = 16, int P = 1, bool ANY = (P < fft_npass_r(N, R0))>
struct PassTwiddlesR {
    static constexpr int R = fft_radix_r(N, P, R0);
    static constexpr int NS = fft_ns_r(N, P, R0);
    static_assert(NT % (N / R) == 0, "thread count must be a multiple of N/R");
    float2 w[R - 1];
    PassTwiddlesR<N, NT, R0, P + 1> next;
    __device__ __forceinline__ void load(const float2* __restrict__ tw)
    {
        const int k = (threadIdx.x % (N / R)) % NS;
        constexpr int step = N / (NS * R);
#pragma unroll
        for (int r = 1; r < R; ++r) w[r - 1] = __ldg(tw + k * r * step);
        next.load(tw);
    }
    template <int Q>
    __device__ __forceinline__ const float2* get() const
    {
        if constexpr (Q == P) return w;
        else return next.template get<Q>();
    }
};
template <int N, int NT, int R0, int P>
struct PassTwiddlesR<N, NT, R0, P, false> {
    __device__ __forceinline__ void load(const float2* __restrict__) {}
    template <int Q>
    __device__ __forceinline__ const float2* get() const { return nullptr; }
};
template <int N, int NT>
using PassTwiddles = PassTwiddlesR<N, NT, 16>;

template <int R>
__device__ __forceinline__ void apply_twiddles(const float2* w, float2 (&v)[R])
{
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r - 1]);
}

// Store the R outputs of butterfly j into row `row` of `buf` (padded for NS).
template <int N, int R, int NS>
__device__ __forceinline__ void pass_store(float2* buf, int row, int j, const float2 (&v)[R])
{
    constexpr int RS = fft_row_stride(N);
    // the R outputs lie in one padding group: one slot computation
    float2* b = buf + row * RS + pad_slot<NS, R>((j / NS) * NS * R + (j % NS));
#pragma unroll
    for (int q = 0; q < R; ++q) b[q * NS] = v[q];
}

}  // namespace ppf
