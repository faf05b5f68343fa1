// Host-side kernel registry shared by the translation units of libppf.so.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "ppf_device.cuh"

namespace ppf {

// What a launcher needs to know about a plan (plain data, no ownership).
struct PlanView {
    int N = 0, T = 0, dtype = 0;
    const void* h = nullptr;      // device coefficients: float (c32) or __half (c16/ci8), [T*N]
    const float2* tw = nullptr;   // device twiddles W_N^m, m = 0..N-1
    int sms = 0;                  // multiprocessors of the plan's device
    int grid_cap = 0;             // resident CTAs for the chosen kernel (set by prepare)
    int fir_only = 0;             // test hook: store y instead of Y
    int out_f16 = 0;              // output bins are FP16 (I, Q) pairs instead of complex64
    int* err = nullptr;           // device-visible error word (mapped host memory)
};

using PrepareFn = cudaError_t (*)(PlanView&);
using LaunchFn = cudaError_t (*)(const PlanView&, const void* in, float2* out, int64_t S,
                                 cudaStream_t stream);
// One launch over a device work list (items/jobs in device memory); `grid`
// CTAs (a multiple of the cluster size).
using LaunchWorkFn = cudaError_t (*)(const PlanView&, const PpfWork& work, int grid, cudaStream_t stream);

struct KernelEntry {
    const char* name = nullptr;
    PrepareFn prepare = nullptr;
    LaunchFn launch = nullptr;
    LaunchWorkFn launch_work = nullptr;  // null: no work-list form (general kernel)
    int rows_per_block = 0;              // spectra per block (RB)
    int cluster = 1;                     // CTAs per cluster
};

// General kernel for (N, dtype), complex64 or (out_f16) FP16 output bins;
// runtime T.  Defined in ppf_generic.cu.
KernelEntry generic_entry(int N, int dtype, int out_f16 = 0);

// Counts kernel launches issued by the library.
void note_launch();

}  // namespace ppf
