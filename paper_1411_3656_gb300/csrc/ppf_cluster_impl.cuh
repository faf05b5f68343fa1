// Host side of the cluster kernel: TMA tensor map of the input, cluster
// launch, and the variant list macro used by ppf_cluster*.cu.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <type_traits>
#include <mutex>

#include "ppf_cluster.cuh"
#include "ppf_launch.h"

namespace ppf {
namespace cluster_detail {

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Input stream as a 3-D tensor (c1: N1, c2: N2, row: rows), element = one sample.
template <class C>
bool encode_input_map(CUtensorMap* m, const void* x, int64_t rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const CUtensorMapDataType dt = C::BPS == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                   : C::BPS == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[3] = {(cuuint64_t)C::N1, (cuuint64_t)C::N2, (cuuint64_t)rows};
    const cuuint64_t strides[2] = {(cuuint64_t)C::N1 * C::BPS, (cuuint64_t)C::N * C::BPS};
    const cuuint32_t box[3] = {(cuuint32_t)C::C1, (cuuint32_t)C::N2, (cuuint32_t)C::RB};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, dt, 3, const_cast<void*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <class C>
cudaLaunchConfig_t launch_config(int grid, cudaStream_t st, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(C::NT, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C::P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class C>
cudaError_t prepare_cluster(PlanView& p)
{
    if (!encode_fn()) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(ppf_cluster_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    if (C::P > 8) {
        e = cudaFuncSetAttribute(ppf_cluster_kernel<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config<C>(C::P * p.sms, nullptr, attr);
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, ppf_cluster_kernel<C>, &cfg);
    if (e != cudaSuccess) return e;
    if (ncl < 1) return cudaErrorInvalidConfiguration;
    p.grid_cap = ncl * C::P;
    return cudaSuccess;
}

template <class C>
cudaError_t launch_cluster(const PlanView& p, const void* in, float2* out, int64_t S, cudaStream_t st)
{
    const int64_t nblk = (S + C::RB - 1) / C::RB;
    const int64_t ncl_cap = p.grid_cap / C::P;
    const int ncl = (int)(nblk < ncl_cap ? nblk : ncl_cap);
    if (ncl <= 0) return cudaSuccess;
    CUtensorMap m;
    if (!encode_input_map<C>(&m, in, S + C::T - 1)) return cudaErrorInvalidValue;
    PpfWork w{};
    w.one.x = in;
    w.one.Y = out;
    w.one.h = p.h;
    w.one.S = S;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config<C>(ncl * C::P, st, attr);
    cudaError_t e = cudaLaunchKernelEx(&cfg, ppf_cluster_kernel<C>, m, w, p.tw, p.err);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_cluster_work(const PlanView& p, const PpfWork& w, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    CUtensorMap unused;
    std::memset(&unused, 0, sizeof(unused));
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = launch_config<C>(grid, st, attr);
    cudaError_t e = cudaLaunchKernelEx(&cfg, ppf_cluster_kernel<C>, unused, w, p.tw, p.err);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class C>
bool encode_job_map(void* tmap128, const void* x, int64_t rows)
{
    return encode_input_map<C>(static_cast<CUtensorMap*>(tmap128), x, rows);
}

template <class C>
KernelEntry entry()
{
    static char name[80];
    std::snprintf(name, sizeof(name), "cluster:p%d:n1_%d:nt%d:rb%d:nch%d:b%d%s%s%s", C::P, C::N1, C::NT, C::RB,
                  C::NCH, C::MINB, C::CPT == 1 ? ":c1" : "", C::R0 == 8 ? ":r8" : "",
                  std::is_same<typename C::OT, BinF16>::value ? ":f16" : "");
    KernelEntry e;
    e.name = name;
    e.prepare = prepare_cluster<C>;
    e.launch = launch_cluster<C>;
    e.launch_work = launch_cluster_work<C>;
    e.encode = encode_job_map<C>;
    e.rows_per_block = C::RB;
    e.cluster = C::P;
    return e;
}

}  // namespace cluster_detail
}  // namespace ppf

// PPF_CV(N, T, P, N1, NT, RB, NCH, MINB): one cluster-kernel variant (a
// channel pair per FIR thread); PPF_CV1: the same with one channel per thread.
#define PPF_CV(NN, TT, P, N1, NT, RB, NCH, MINB)                                                        \
    if (N == NN && T == TT) {                                                                           \
        if (idx == want && out)                                                                         \
            *out = cluster_detail::entry<ClusterCfg<NN, TT, In, P, N1, NT, RB, NCH, MINB>>();           \
        ++idx;                                                                                          \
    }
#define PPF_CV1(NN, TT, P, N1, NT, RB, NCH, MINB)                                                       \
    if (N == NN && T == TT) {                                                                           \
        if (idx == want && out)                                                                         \
            *out = cluster_detail::entry<ClusterCfg<NN, TT, In, P, N1, NT, RB, NCH, MINB, 1>>();        \
        ++idx;                                                                                          \
    }
// PPF_CVF(N, T, P, N1, NT, RB, NCH, MINB, channels per FIR thread, first-pass
// radix): the FP16-output twin of a tile shape.
#define PPF_CVF(NN, TT, P, N1, NT, RB, NCH, MINB, CPT, R0)                                                   \
    if (N == NN && T == TT) {                                                                                \
        if (idx == want && out)                                                                              \
            *out = cluster_detail::entry<ClusterCfg<NN, TT, In, P, N1, NT, RB, NCH, MINB, CPT, BinF16, R0>>(); \
        ++idx;                                                                                               \
    }
// PPF_CV81(N, T, P, N1, NT, RB, NCH, MINB): one channel per FIR thread and a
// radix-8 first pass.
#define PPF_CV81(NN, TT, P, N1, NT, RB, NCH, MINB)                                                     \
    if (N == NN && T == TT) {                                                                         \
        if (idx == want && out)                                                                       \
            *out = cluster_detail::entry<ClusterCfg<NN, TT, In, P, N1, NT, RB, NCH, MINB, 1, float2, 8>>(); \
        ++idx;                                                                                        \
    }
// PPF_CV8(N, T, P, N1, NT, RB, NCH, MINB): a tile shape whose stages start with
// a radix-8 pass.
#define PPF_CV8(NN, TT, P, N1, NT, RB, NCH, MINB)                                                      \
    if (N == NN && T == TT) {                                                                         \
        if (idx == want && out)                                                                       \
            *out = cluster_detail::entry<ClusterCfg<NN, TT, In, P, N1, NT, RB, NCH, MINB, 2, float2, 8>>(); \
        ++idx;                                                                                        \
    }
