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
// CTA c processes items[first[c] .. first[c+1]) in order: the host cuts the
// jobs' blocks, laid end to end, into one segment of equal estimated work per
// CTA (a segment may span several jobs: one item per job piece).
struct MixWork {
    const MixJob* jobs;
    const MixItem* items;
    const int* first;  // [grid + 1]
};

// Index of (N, T) in the kernel's shape list (complex64 input and output),
// or -1 when the mixed kernel does not take that size.
int mix_shape(int N, int T);
// Spectra per block of a shape.
int mix_rows_per_block(int shape);
// Kernel attributes; *grid = resident CTAs on `device` (one per SM).
cudaError_t mix_prepare(int device, int* grid);
// Launch `grid` CTAs over the work list.
cudaError_t mix_launch(const MixWork& w, int grid, int* err, cudaStream_t st);

// Host: split `jobs` into items, one contiguous segment of about equal
// estimated work (output samples weighted by 16 + T/2) per CTA of `grid`;
// items and first (grid + 1 entries) are filled.
struct MixJobInfo {
    int N, T;
    int64_t S;
};
void mix_partition(const MixJobInfo* jobs, int n_jobs, int grid, std::vector<MixItem>& items,
                   std::vector<int>& first);

}  // namespace ppf
