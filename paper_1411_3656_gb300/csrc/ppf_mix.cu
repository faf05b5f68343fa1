// Host side of the mixed-shape persistent kernel (ppf_mix.cuh): shape lookup,
// launch geometry and the launch itself.
#include "ppf_mix.cuh"
#include "ppf_mix.h"

#include <algorithm>

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
template <int I = 0>
int shape_cost(int s)
{
    if constexpr (I < kMixShapes) {
        using Sh = typename std::tuple_element<I, MixShapeList>::type;
        return s == I ? Sh::COST : shape_cost<I + 1>(s);
    } else {
        return 0;
    }
}
}  // namespace

int mix_shape(int N, int T) { return shape_index(N, T); }

int mix_rows_per_block(int shape) { return shape_rb(shape); }

double mix_cost_ms(int shape) { return shape_cost(shape) * 1e-3; }

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

void mix_items(const MixJobInfo* jobs, int n_jobs, int grid, std::vector<MixItem>& items)
{
    items.clear();
    std::vector<double> per_block((size_t)n_jobs, 0.0);
    std::vector<int64_t> nblk((size_t)n_jobs, 0);
    double total = 0;
    for (int k = 0; k < n_jobs; ++k) {
        const int shape = mix_shape(jobs[k].N, jobs[k].T);
        if (shape < 0 || jobs[k].S <= 0) continue;
        const int RB = mix_rows_per_block(shape);
        nblk[k] = (jobs[k].S + RB - 1) / RB;
        per_block[k] = (double)RB * jobs[k].N * mix_cost_ms(shape);
        total += per_block[k] * (double)nblk[k];
    }
    const double target = total / ((double)grid * kMixItemsPerCta);
    std::vector<double> cost;
    for (int k = 0; k < n_jobs; ++k) {
        if (nblk[k] == 0) continue;
        const int RB = mix_rows_per_block(mix_shape(jobs[k].N, jobs[k].T));
        // at least 4T spectra per item: the T-1 halo rows and the ring's
        // fill stay small against the item's work
        const int64_t min_len = std::max<int64_t>(2, (4 * (int64_t)jobs[k].T + RB - 1) / RB);
        int64_t len = std::max<int64_t>(min_len, (int64_t)(target / per_block[k] + 0.5));
        const int64_t pieces = std::max<int64_t>(1, (nblk[k] + len / 2) / len);
        for (int64_t q = 0; q < pieces; ++q) {
            MixItem it{};
            it.job = k;
            it.blo = nblk[k] * q / pieces;
            it.bhi = nblk[k] * (q + 1) / pieces;
            if (it.bhi > it.blo) {
                items.push_back(it);
                cost.push_back(per_block[k] * (double)(it.bhi - it.blo));
            }
        }
    }
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<MixItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    items.swap(sorted);
}

}  // namespace ppf
