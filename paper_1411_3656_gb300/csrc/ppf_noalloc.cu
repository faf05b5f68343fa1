// ppf_execute_noalloc: the whole PPF without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// filter bank: plug-ins hosted by a framework that owns all device memory and
// forbids direct cudaMalloc/cudaFree, and real-time threads that must not
// block on the allocator (cudaMalloc and cudaFree can synchronise the whole
// device).  For them this entry point runs the general fused kernel with no
// plan: the caller passes the coefficients as a device array, and the one
// piece of scratch memory the kernel needs, the FFT twiddle table, lives in a
// file-scope __device__ array of at most 4096 complex values (32 KiB, held by
// every GPU that loads the library until the process exits).
#include "ppf.h"
#include "ppf_generic.cuh"
#include "ppf_launch.h"

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

namespace {

constexpr int kNoallocMaxN = 4096;  // twiddles W_N^m, m < N, for N up to 4096
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is only a stand-in: the kernel gets the
// device address obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) float2 g_noalloc_twiddles[kNoallocMaxN];

struct DeviceSetup {
    std::mutex mu;
    std::atomic<bool> ready{false};  // set only once a set-up has succeeded
    float2* tw = nullptr;  // device address of g_noalloc_twiddles on this device
    int sms = 0;
    int occ[3][13] = {};   // resident CTAs per SM of the general kernel, [dtype][log2 N]
};
DeviceSetup g_setup[kMaxDevices];

// W_N^m = exp(-2*pi*i*m/N), evaluated in FP64 on the device and rounded to FP32.
__global__ void fill_noalloc_twiddles(float2* tw, int N)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < N) {
        double s, c;
        sincospi(2.0 * (double)m / (double)N, &s, &c);
        tw[m] = make_float2((float)c, (float)-s);
    }
}

template <int N, class In>
cudaError_t setup_one(DeviceSetup& d, int dt)
{
    auto kern = ppf::ppf_generic_kernel<N, In, float>;
    constexpr int smem = ppf::generic_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, ppf::kGenericThreads, smem);
    int lg = 0;
    while ((1 << lg) < N) ++lg;
    d.occ[dt][lg] = occ > 0 ? occ : 1;
    return e;
}

template <class In>
cudaError_t setup_dtype(DeviceSetup& d, int dt)
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = setup_one<4, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<8, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<16, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<32, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<64, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<128, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<256, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<512, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<1024, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<2048, In>(d, dt);
    if (e == cudaSuccess) e = setup_one<4096, In>(d, dt);
    return e;
}

// Once per device, with that device current: the scratch's device address,
// kernel attributes and occupancy.  Allocates nothing.  Only success is
// remembered: a set-up that fails (its error is returned, and cleared from
// CUDA's last-error state unless the context itself is broken) is tried
// again by the next call.
cudaError_t ensure_setup(DeviceSetup& d, int dev)
{
    if (d.ready.load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(d.mu);
    if (d.ready.load(std::memory_order_relaxed)) return cudaSuccess;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&d.tw), g_noalloc_twiddles);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = setup_dtype<ppf::InC32>(d, 0);
    if (e == cudaSuccess) e = setup_dtype<ppf::InC16>(d, 1);
    if (e == cudaSuccess) e = setup_dtype<ppf::InCI8>(d, 2);
    if (e == cudaSuccess) d.ready.store(true, std::memory_order_release);
    else cudaGetLastError();
    return e;
}

template <int N, class In>
cudaError_t launch_n(const DeviceSetup& d, int dt, int T, const float* h, const void* in, float2* out, int64_t S,
                     cudaStream_t st)
{
    constexpr int RB = ppf::generic_rows(N);
    int lg = 0;
    while ((1 << lg) < N) ++lg;
    const int64_t nblk = (S + RB - 1) / RB;
    const int64_t cap = (int64_t)d.occ[dt][lg] * d.sms;
    const int grid = (int)(nblk < cap ? nblk : cap);
    ppf::ppf_generic_kernel<N, In, float><<<grid, ppf::kGenericThreads, ppf::generic_smem_bytes(N), st>>>(
        static_cast<const typename In::raw*>(in), h, d.tw, out, T, S, 0);
    ppf::note_launch();
    return cudaGetLastError();
}

template <class In>
cudaError_t launch_dtype(const DeviceSetup& d, int dt, int N, int T, const float* h, const void* in, float2* out,
                         int64_t S, cudaStream_t st)
{
    switch (N) {
    case 4: return launch_n<4, In>(d, dt, T, h, in, out, S, st);
    case 8: return launch_n<8, In>(d, dt, T, h, in, out, S, st);
    case 16: return launch_n<16, In>(d, dt, T, h, in, out, S, st);
    case 32: return launch_n<32, In>(d, dt, T, h, in, out, S, st);
    case 64: return launch_n<64, In>(d, dt, T, h, in, out, S, st);
    case 128: return launch_n<128, In>(d, dt, T, h, in, out, S, st);
    case 256: return launch_n<256, In>(d, dt, T, h, in, out, S, st);
    case 512: return launch_n<512, In>(d, dt, T, h, in, out, S, st);
    case 1024: return launch_n<1024, In>(d, dt, T, h, in, out, S, st);
    case 2048: return launch_n<2048, In>(d, dt, T, h, in, out, S, st);
    case 4096: return launch_n<4096, In>(d, dt, T, h, in, out, S, st);
    default: return cudaErrorInvalidValue;
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" ppf_status_t ppf_execute_noalloc(int N, int T, ppf_dtype_t dtype, const float* d_h, const void* d_in,
                                            void* d_out, int64_t n_spectra, void* stream)
{
    const int bps = dtype == PPF_IN_C32 ? 8 : dtype == PPF_IN_C16 ? 4 : dtype == PPF_IN_CI8 ? 2 : 0;
    if (bps == 0) return PPF_ERR_UNSUPPORTED;
    // N above kNoallocMaxN would not fit the twiddle scratch.
    if (N < 4 || N > kNoallocMaxN || (N & (N - 1)) != 0 || T < 1 || T > 64) return PPF_ERR_UNSUPPORTED;
    if (n_spectra < 0) return PPF_ERR_INVALID_ARG;
    if (n_spectra == 0) return PPF_OK;
    if (!d_h || !d_in || !d_out) return PPF_ERR_INVALID_ARG;
    if (!aligned16(d_in) || !aligned16(d_out)) return PPF_ERR_MISALIGNED;
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(d_in), o0 = reinterpret_cast<uintptr_t>(d_out);
    const uintptr_t in_bytes = (uintptr_t)(n_spectra + T - 1) * N * bps, out_bytes = (uintptr_t)n_spectra * N * 8;
    const uintptr_t h0 = reinterpret_cast<uintptr_t>(d_h), h_bytes = (uintptr_t)N * T * sizeof(float);
    if (i0 < o0 + out_bytes && o0 < i0 + in_bytes) return PPF_ERR_MISALIGNED;
    if (h0 < o0 + out_bytes && o0 < h0 + h_bytes) return PPF_ERR_MISALIGNED;
    if (cudaPeekAtLastError() != cudaSuccess) return PPF_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PPF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return PPF_ERR_UNSUPPORTED;
    DeviceSetup& d = g_setup[dev];
    if (ensure_setup(d, dev) != cudaSuccess) return PPF_ERR_CUDA;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fill_noalloc_twiddles<<<(N + 255) / 256, 256, 0, st>>>(d.tw, N);
    ppf::note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return PPF_ERR_CUDA;
    float2* out = static_cast<float2*>(d_out);
    switch (dtype) {
    case PPF_IN_C32: e = launch_dtype<ppf::InC32>(d, 0, N, T, d_h, d_in, out, n_spectra, st); break;
    case PPF_IN_C16: e = launch_dtype<ppf::InC16>(d, 1, N, T, d_h, d_in, out, n_spectra, st); break;
    default: e = launch_dtype<ppf::InCI8>(d, 2, N, T, d_h, d_in, out, n_spectra, st); break;
    }
    return e == cudaSuccess ? PPF_OK : PPF_ERR_CUDA;
}
