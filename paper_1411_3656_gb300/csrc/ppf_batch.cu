// Batches of independent streams (see include/ppf.h): complex64 jobs whose
// window fits one SM share one persistent launch of the mixed-shape kernel;
// the other jobs are grouped by specialised kernel, each group one persistent
// launch over a device work list.
#include "ppf.h"
#include "ppf_launch.h"
#include "ppf_mix.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

namespace ppf {
// Plan internals this file needs (defined in ppf_api.cu).
bool plan_info(ppf_plan_t plan, PlanView* view, KernelEntry* entry, int* sample_bytes);
bool plan_mixable(ppf_plan_t plan);
int plan_device(ppf_plan_t plan);
}  // namespace ppf

struct ppf_batch_s {
    struct Group {
        ppf::PlanView view;   // launch parameters of the group's first plan (twiddles, error word)
        ppf::KernelEntry entry;
        ppf::PpfWork work{};  // device job/item tables
        int grid = 0;
    };
    struct Single {            // a job on the general kernel
        ppf::PlanView view;
        ppf::KernelEntry entry;
        ppf_job_t job;
    };
    std::vector<Group> groups;
    std::vector<Single> singles;
    // jobs of the mixed-shape kernel: one persistent launch for all of them
    bool has_mix = false;
    ppf::MixWork mix{};
    int mix_grid = 0;
    int* mix_err = nullptr;
    void* dev = nullptr;      // one allocation holding every table
    unsigned flags = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

namespace {

ppf_status_t from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return PPF_OK;
    if (e == cudaErrorMemoryAllocation) return PPF_ERR_OUT_OF_MEMORY;
    return PPF_ERR_CUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

ppf_status_t enqueue(ppf_batch_s* b, cudaStream_t st)
{
    if (b->has_mix) {
        // the mixed kernel's item counter starts from zero every execution
        cudaError_t e = cudaMemsetAsync(b->mix.next, 0, sizeof(int), st);
        if (e == cudaSuccess) e = ppf::mix_launch(b->mix, b->mix_grid, b->mix_err, st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    for (auto& g : b->groups) {
        cudaError_t e = g.entry.launch_work(g.view, g.work, g.grid, st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    for (auto& s : b->singles) {
        cudaError_t e = s.entry.launch(s.view, s.job.d_in, static_cast<float2*>(s.job.d_out), s.job.n_spectra, st);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return PPF_OK;
}

}  // namespace

extern "C" {

ppf_status_t ppf_batch_create(ppf_batch_t* out, const ppf_job_t* jobs, int n_jobs, unsigned flags)
{
    if (!out || n_jobs < 0 || (n_jobs > 0 && !jobs)) return PPF_ERR_INVALID_ARG;
    if (flags & ~(PPF_BATCH_GRAPH | PPF_BATCH_PER_KERNEL)) return PPF_ERR_INVALID_ARG;
    *out = nullptr;
    ppf_batch_s* b = new (std::nothrow) ppf_batch_s();
    if (!b) return PPF_ERR_OUT_OF_MEMORY;
    b->flags = flags;

    // 1. validate and group by kernel instantiation (same launch function)
    struct Pending {
        ppf::PlanView view;
        ppf::KernelEntry entry;
        std::vector<int> jobs;
    };
    std::map<std::string, Pending> by_kernel;
    std::vector<std::string> order;
    std::vector<int> mix_jobs;
    for (int i = 0; i < n_jobs; ++i) {
        const ppf_job_t& j = jobs[i];
        ppf::PlanView v;
        ppf::KernelEntry e;
        int bps = 0;
        if (!j.plan || j.n_spectra < 0 || !ppf::plan_info(j.plan, &v, &e, &bps)) {
            delete b;
            return PPF_ERR_INVALID_ARG;
        }
        if (j.n_spectra == 0) continue;
        if (!j.d_in || !j.d_out) {
            delete b;
            return PPF_ERR_INVALID_ARG;
        }
        if (!aligned16(j.d_in) || !aligned16(j.d_out)) {
            delete b;
            return PPF_ERR_MISALIGNED;
        }
        if (!(flags & PPF_BATCH_PER_KERNEL) && ppf::plan_mixable(j.plan) && ppf::mix_shape(v.N, v.T) >= 0) {
            mix_jobs.push_back(i);
            continue;
        }
        if (!e.launch_work) {
            b->singles.push_back({v, e, j});
            continue;
        }
        char key[160];
        std::snprintf(key, sizeof(key), "%d:%d:%d:%s", v.N, v.T, v.dtype, e.name);
        auto it = by_kernel.find(key);
        if (it == by_kernel.end()) {
            by_kernel[key] = Pending{v, e, {i}};
            order.push_back(key);
        } else {
            it->second.jobs.push_back(i);
        }
    }

    if (!mix_jobs.empty()) {
        cudaError_t e = ppf::mix_prepare(ppf::plan_device(jobs[mix_jobs[0]].plan), &b->mix_grid);
        if (e != cudaSuccess) {
            delete b;
            return from_cuda(e);
        }
    }

    // 2. bands: about one item per resident CTA (or cluster) of the group
    struct Layout {
        std::vector<ppf::PpfJob> jobs;
        std::vector<ppf::PpfItem> items;
    };
    std::vector<Layout> lay(order.size());
    size_t bytes = 0;
    for (size_t gi = 0; gi < order.size(); ++gi) {
        Pending& pg = by_kernel[order[gi]];
        const int RB = pg.entry.rows_per_block;
        const int units = std::max(1, pg.view.grid_cap / pg.entry.cluster);
        int64_t total_blocks = 0;
        for (int ji : pg.jobs) total_blocks += (jobs[ji].n_spectra + RB - 1) / RB;
        const int64_t target = std::max<int64_t>(1, (total_blocks + units - 1) / units);
        Layout& L = lay[gi];
        for (int ji : pg.jobs) {
            const ppf_job_t& j = jobs[ji];
            ppf::PpfJob pj{};
            pj.x = j.d_in;
            pj.Y = static_cast<float2*>(j.d_out);
            ppf::PlanView v;
            ppf::KernelEntry e;
            int bps = 0;
            ppf::plan_info(j.plan, &v, &e, &bps);
            pj.h = v.h;
            pj.S = j.n_spectra;
            const int jid = (int)L.jobs.size();
            L.jobs.push_back(pj);
            const int64_t nblk = (j.n_spectra + RB - 1) / RB;
            const int64_t pieces = std::max<int64_t>(1, (nblk + target / 2) / target);
            for (int64_t k = 0; k < pieces; ++k) {
                ppf::PpfItem it{};
                it.job = jid;
                it.blo = nblk * k / pieces;
                it.bhi = nblk * (k + 1) / pieces;
                if (it.bhi > it.blo) L.items.push_back(it);
            }
        }
        bytes += sizeof(ppf::PpfJob) * L.jobs.size() + sizeof(ppf::PpfItem) * L.items.size() + 256;
    }

    // 2b. the mixed-shape launch: the jobs cut into items of about equal
    // estimated cost, largest first
    std::vector<ppf::MixJob> mjobs;
    std::vector<ppf::MixItem> mitems;
    if (!mix_jobs.empty()) {
        std::vector<ppf::MixJobInfo> info;
        for (int ji : mix_jobs) {
            const ppf_job_t& j = jobs[ji];
            ppf::PlanView v;
            ppf::KernelEntry e2;
            int bps = 0;
            ppf::plan_info(j.plan, &v, &e2, &bps);
            ppf::MixJob mj{};
            mj.x = j.d_in;
            mj.Y = static_cast<float2*>(j.d_out);
            mj.h = v.h;
            mj.tw = v.tw;
            mj.S = j.n_spectra;
            mj.shape = ppf::mix_shape(v.N, v.T);
            mjobs.push_back(mj);
            info.push_back({v.N, v.T, j.n_spectra});
            if (!b->mix_err) b->mix_err = v.err;
        }
        ppf::mix_items(info.data(), (int)info.size(), b->mix_grid, mitems);
        b->has_mix = !mitems.empty();
        bytes += sizeof(ppf::MixJob) * mjobs.size() + sizeof(ppf::MixItem) * mitems.size() + 16 + 256;
    }

    // 3. one device allocation for every table
    if (bytes > 0) {
        cudaError_t e = cudaMalloc(&b->dev, bytes);
        if (e != cudaSuccess) {
            delete b;
            return from_cuda(e);
        }
    }
    std::vector<unsigned char> host(bytes, 0);
    size_t off = 0;
    auto place = [&](size_t n, size_t align) {
        off = (off + align - 1) / align * align;
        const size_t at = off;
        off += n;
        return at;
    };
    for (size_t gi = 0; gi < order.size(); ++gi) {
        Pending& pg = by_kernel[order[gi]];
        Layout& L = lay[gi];
        const size_t jobs_at = place(sizeof(ppf::PpfJob) * L.jobs.size(), 16);
        std::memcpy(&host[jobs_at], L.jobs.data(), sizeof(ppf::PpfJob) * L.jobs.size());
        const size_t items_at = place(sizeof(ppf::PpfItem) * L.items.size(), 16);
        std::memcpy(&host[items_at], L.items.data(), sizeof(ppf::PpfItem) * L.items.size());
        ppf_batch_s::Group g;
        g.view = pg.view;
        g.entry = pg.entry;
        g.work.jobs = reinterpret_cast<const ppf::PpfJob*>(static_cast<unsigned char*>(b->dev) + jobs_at);
        g.work.items = reinterpret_cast<const ppf::PpfItem*>(static_cast<unsigned char*>(b->dev) + items_at);
        g.work.n_items = (int)L.items.size();
        const int units = std::max(1, pg.view.grid_cap / pg.entry.cluster);
        g.grid = std::min<int>(units, g.work.n_items) * pg.entry.cluster;
        b->groups.push_back(g);
    }
    if (b->has_mix) {
        unsigned char* dev = static_cast<unsigned char*>(b->dev);
        const size_t jobs_at = place(sizeof(ppf::MixJob) * mjobs.size(), 16);
        std::memcpy(&host[jobs_at], mjobs.data(), sizeof(ppf::MixJob) * mjobs.size());
        const size_t items_at = place(sizeof(ppf::MixItem) * mitems.size(), 16);
        std::memcpy(&host[items_at], mitems.data(), sizeof(ppf::MixItem) * mitems.size());
        const size_t next_at = place(sizeof(int), 16);
        b->mix.jobs = reinterpret_cast<const ppf::MixJob*>(dev + jobs_at);
        b->mix.items = reinterpret_cast<const ppf::MixItem*>(dev + items_at);
        b->mix.n_items = (int)mitems.size();
        b->mix.n_items_dev = nullptr;
        b->mix.next = reinterpret_cast<int*>(dev + next_at);
    }
    if (bytes > 0) {
        cudaError_t e = cudaMemcpy(b->dev, host.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(b->dev);
            delete b;
            return from_cuda(e);
        }
    }
    b->launches = (int)(b->groups.size() + b->singles.size()) + (b->has_mix ? 1 : 0);
    *out = b;
    return PPF_OK;
}

ppf_status_t ppf_batch_execute(ppf_batch_t b, void* stream)
{
    if (!b) return PPF_ERR_INVALID_ARG;
    if (cudaPeekAtLastError() != cudaSuccess) return PPF_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!(b->flags & PPF_BATCH_GRAPH)) return enqueue(b, st);
    if (!b->exec) {
        cudaError_t e = cudaSuccess;
        if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return from_cuda(e);
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return from_cuda(e);
        const ppf_status_t s = enqueue(b, b->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (s != PPF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return from_cuda(e);
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return from_cuda(cudaGraphLaunch(b->exec, st));
}

int ppf_batch_launches(ppf_batch_t b) { return b ? b->launches : -1; }

ppf_status_t ppf_batch_destroy(ppf_batch_t b)
{
    if (!b) return PPF_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->dev) cudaFree(b->dev);
    delete b;
    return from_cuda(e);
}

}  // extern "C"
