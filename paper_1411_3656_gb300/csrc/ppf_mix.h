// Host interface of the mixed-shape persistent kernel (ppf_mix.cu), shared
// by the batch and server translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ppf_launch.h"

namespace ppf {

// A job of a mixed launch: a stream of N-channel rows with its own h and
// twiddles; `shape` indexes MixShapes.
struct MixJob {
    const void* x;
    float2* Y;
    const void* h;
    const float2* tw;
    int64_t S;
    int shape;
    int pad;
};
// Blocks [blo, bhi) of job `job` (a block is the shape's RB spectra).
struct MixItem {
    int job;
    int pad;
    int64_t blo;
    int64_t bhi;
};
// The work of one launch.  CTA c takes item c first; every later item goes to
// the CTA that asks for it next (an atomic counter), so CTAs that finish
// early take more items.  Items are sorted by estimated cost, largest first.
struct MixWork {
    const MixJob* jobs;
    const MixItem* items;
    int n_items;             // used when n_items_dev is null
    int pad;
    const int* n_items_dev;  // item count read on the device (graph replays)
    int* next;               // items handed out beyond the first gridDim.x: zero before each launch
};

// Index of (N, T) in the kernel's shape list (complex64 input and output),
// or -1 when the mixed kernel does not take that size.
int mix_shape(int N, int T);
// Spectra per block of a shape.
int mix_rows_per_block(int shape);
// Measured time of a shape in the mixed kernel for one second of 6.5 GB/s
// input (ms): the relative cost of its samples.
double mix_cost_ms(int shape);
// Kernel attributes; *grid = resident CTAs on `device` (one per SM).
cudaError_t mix_prepare(int device, int* grid);
// Launch `grid` CTAs over the work list.
cudaError_t mix_launch(const MixWork& w, int grid, int* err, cudaStream_t st);

// Host: cut `jobs` into items of about equal estimated cost (output samples
// weighted by the shape's measured cost), about kMixItemsPerCta per CTA of
// `grid` and never shorter than the window's halo calls for, sorted largest
// first.
struct MixJobInfo {
    int N, T;
    int64_t S;
};
constexpr int kMixItemsPerCta = 12;
void mix_items(const MixJobInfo* jobs, int n_jobs, int grid, std::vector<MixItem>& items);

}  // namespace ppf
