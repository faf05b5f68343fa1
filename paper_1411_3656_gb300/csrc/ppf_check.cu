// Failure-detection self-check: the device-side bounded wait, made to run
// out; and the violation counters of the checked (-DPPF_CHECKED) build.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/ppf.h"
#include "ppf_launch.h"
#include "ppf_ptx.cuh"

namespace {

// One warp waits on an mbarrier that nothing arrives on, with the same bounded
// wait the PPF kernels use, and reports the give-up through the error word.
__global__ void wait_timeout_kernel(uint64_t limit_ns, int* err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        ppf::mbar_init(&bar, 1);
        ppf::fence_mbar_init();
    }
    __syncwarp();
    const bool ok = ppf::mbar_wait_bounded(&bar, 0, limit_ns);
    if (__any_sync(0xffffffffu, !ok) && threadIdx.x == 0) atomicExch(err, 1);
}

// FP32 throughput probe: every thread runs kChains independent chains of
// packed FMAs (a <- a * m + c on float2 lanes), so each issue has work that
// does not wait on the one before; the result is written only if it matches
// an impossible value, which keeps the chains alive without memory traffic.
constexpr int kChains = 8;
__global__ void __launch_bounds__(512) fma_peak_kernel(int iters, float2* sink)
{
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(1.0f + 1e-3f * threadIdx.x, 1.0f + 1e-3f * k);
    const float2 m = make_float2(0.999999f, 1.000001f), c = make_float2(1e-7f, -1e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], m, c);
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += a[k].x + a[k].y;
    if (acc == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = make_float2(acc, acc);
}

}  // namespace

extern "C" ppf_status_t ppf_fma_peak(int blocks, int iters, void* stream, double* lane_fmas)
{
    if (blocks < 1 || blocks > 65535 || iters < 1 || iters > (1 << 24) || !lane_fmas) return PPF_ERR_INVALID_ARG;
    fma_peak_kernel<<<blocks, 512, 0, static_cast<cudaStream_t>(stream)>>>(iters, nullptr);
    ppf::note_launch();
    if (cudaGetLastError() != cudaSuccess) return PPF_ERR_CUDA;
    *lane_fmas = (double)blocks * 512.0 * (double)iters * kChains * 2.0;
    return PPF_OK;
}

extern "C" ppf_status_t ppf_check_timeout(unsigned limit_us, void* stream)
{
    if (limit_us < 1 || limit_us > 1000000) return PPF_ERR_INVALID_ARG;
    int* h_err = nullptr;
    int* d_err = nullptr;
    cudaError_t e = cudaHostAlloc((void**)&h_err, sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) return PPF_ERR_OUT_OF_MEMORY;
    *h_err = 0;
    e = cudaHostGetDevicePointer((void**)&d_err, h_err, 0);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (e == cudaSuccess) {
        wait_timeout_kernel<<<1, 32, 0, st>>>((uint64_t)limit_us * 1000u, d_err);
        ppf::note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const int flagged = *(volatile int*)h_err;
    cudaFreeHost(h_err);
    if (e != cudaSuccess) return PPF_ERR_CUDA;
    return flagged ? PPF_ERR_TIMEOUT : PPF_OK;
}

namespace ppf {
namespace {
struct CheckRegistry {
    std::mutex m;
    std::vector<unsigned long long (*)(bool)> readers;
};
CheckRegistry& check_registry()
{
    static CheckRegistry r;
    return r;
}
}  // namespace

// Each translation unit of the checked build registers the reader of its
// counter at load time.
void register_check_counter(unsigned long long (*read)(bool reset))
{
    CheckRegistry& r = check_registry();
    std::lock_guard<std::mutex> g(r.m);
    r.readers.push_back(read);
}
}  // namespace ppf

extern "C" int64_t ppf_check_violations(int reset)
{
#ifdef PPF_CHECKED
    ppf::CheckRegistry& r = ppf::check_registry();
    std::lock_guard<std::mutex> g(r.m);
    if (cudaDeviceSynchronize() != cudaSuccess) return -2;
    unsigned long long total = 0;
    for (auto read : r.readers) {
        const unsigned long long v = read(reset != 0);
        if (v == ~0ull) return -2;
        total += v;
    }
    return (int64_t)total;
#else
    (void)reset;
    return -1;
#endif
}
