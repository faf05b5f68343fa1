// Host side of the mixed-shape persistent kernel (ppf_mix.cuh): shape lookup,
// launch geometry and the launch itself.
#include "ppf_mix.cuh"
#include "ppf_mix.h"

namespace ppf {

namespace {
template <int I = 0>
int shape_index(int N, int T)
{
    if constexpr (I < kMixShapes) {
        using Sh = typename std::tuple_element<I, MixShapeList>::type;
        if (Sh::N == N && Sh::T == T) return I;
        return shape_index<I + 1>(N, T);
    } else {
        return -1;
    }
}
template <int I = 0>
int shape_rb(int s)
{
    if constexpr (I < kMixShapes) {
        using Sh = typename std::tuple_element<I, MixShapeList>::type;
        return s == I ? Sh::RB : shape_rb<I + 1>(s);
    } else {
        return 0;
    }
}
}  // namespace

int mix_shape(int N, int T) { return shape_index(N, T); }

int mix_rows_per_block(int shape) { return shape_rb(shape); }

cudaError_t mix_prepare(int device, int* grid)
{
    cudaError_t e = cudaFuncSetAttribute(ppf_mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MixGeom::SMEM);
    if (e != cudaSuccess) return e;
    int occ = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ppf_mix_kernel, MixGeom::NT, MixGeom::SMEM);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *grid = occ * sms;
    return cudaSuccess;
}

cudaError_t mix_launch(const MixWork& w, int grid, int* err, cudaStream_t st)
{
    ppf_mix_kernel<<<grid, MixGeom::NT, MixGeom::SMEM, st>>>(w, err);
    note_launch();
    return cudaGetLastError();
}

void mix_partition(const MixJobInfo* jobs, int n_jobs, int grid, std::vector<MixItem>& items, std::vector<int>& first)
{
    items.clear();
    first.assign((size_t)grid + 1, 0);
    std::vector<double> per_block((size_t)n_jobs, 0.0);
    std::vector<int64_t> nblk((size_t)n_jobs, 0);
    double total = 0;
    for (int k = 0; k < n_jobs; ++k) {
        const int shape = mix_shape(jobs[k].N, jobs[k].T);
        if (shape < 0 || jobs[k].S <= 0) continue;
        const int RB = mix_rows_per_block(shape);
        nblk[k] = (jobs[k].S + RB - 1) / RB;
        per_block[k] = (double)RB * jobs[k].N * (16.0 + 0.5 * jobs[k].T);
        total += per_block[k] * (double)nblk[k];
    }
    // walk the blocks of all jobs in order; CTA c takes the blocks whose
    // cumulative work lies in [c, c+1) * total / grid
    int c = 0;
    double done = 0;  // work before the current block
    for (int k = 0; k < n_jobs; ++k) {
        int64_t b = 0;
        while (b < nblk[k]) {
            while (c < grid - 1 && done >= total * (c + 1) / grid) first[(size_t)++c] = (int)items.size();
            // blocks of job k that still fit CTA c's share (at least one)
            const double room = c == grid - 1 ? 1e300 : total * (c + 1) / grid - done;
            int64_t take = (int64_t)(room / per_block[k] + 0.5);
            if (take < 1) take = 1;
            if (take > nblk[k] - b) take = nblk[k] - b;
            MixItem it{};
            it.job = k;
            it.blo = b;
            it.bhi = b + take;
            items.push_back(it);
            b += take;
            done += per_block[k] * (double)take;
        }
    }
    while (c < grid) first[(size_t)++c] = (int)items.size();
}

}  // namespace ppf
