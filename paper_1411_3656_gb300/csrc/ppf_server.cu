// Serving loop core: many continuous streams admitted by device memory,
// their chunks batched into one set of launches per tick (see include/ppf.h),
// replayed from a captured CUDA graph.
//
// Per stream the server owns two device buffers (ping-pong) of capacity
// 8*T*N + 4*max_chunk + 2*N samples holding the FIR history (Section 2: each
// output needs the newest sample and T-1 past samples of its channel) plus
// newly arrived samples.  A tick
//   1. copies every queued chunk behind its stream's history (one batched
//      copy launch for all streams),
//   2. runs the PPF on every stream's newly complete spectra (one launch of
//      the mixed-shape kernel for every stream whose window fits one SM, one
//      persistent work-list launch per other specialised kernel),
//   3. copies each stream's new history to the front of its other buffer
//      (one batched copy launch) and swaps the buffers.
// The kernels of a tick are captured once into a CUDA graph (re-captured when
// a stream is admitted or released); every kernel reads its tables and item
// counts from a fixed device area, so a tick uploads the new tables (pinned
// staging, two slots alternating so the host can build tick k+1 while tick k
// runs) and replays the graph.  Streams on the general kernel keep direct
// launches.
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
bool plan_info(ppf_plan_t plan, PlanView* view, KernelEntry* entry, int* sample_bytes);
bool plan_mixable(ppf_plan_t plan);
int plan_device(ppf_plan_t plan);
}

namespace {

// One contiguous device-to-device copy piece (at most kSeg bytes).
struct CopySeg {
    const unsigned char* src;
    unsigned char* dst;
    int64_t bytes;
};
constexpr int64_t kSeg = 64 * 1024;

// Batched copy: CTA i copies segments i, i + grid, ...; 16-byte vectors when
// both ends are 16-byte aligned, else 4-, 2- or 1-byte elements.  The count
// is n, or *n_dev when given (a launch captured in the tick's CUDA graph).
__global__ void __launch_bounds__(256) batched_copy(const CopySeg* __restrict__ segs, int n, const int* n_dev)
{
    if (n_dev) n = *n_dev;
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        const CopySeg c = segs[s];
        const uintptr_t a = reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst);
        if ((a & 15u) == 0 && (c.bytes & 15) == 0) {
            const int64_t n16 = c.bytes / 16;
            const uint4* src = reinterpret_cast<const uint4*>(c.src);
            uint4* dst = reinterpret_cast<uint4*>(c.dst);
            for (int64_t i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldcs(src + i);
        } else if ((a & 3u) == 0 && (c.bytes & 3) == 0) {
            const int64_t n4 = c.bytes / 4;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(c.src);
            uint32_t* dst = reinterpret_cast<uint32_t*>(c.dst);
            for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = src[i];
        } else {
            for (int64_t i = threadIdx.x; i < c.bytes; i += blockDim.x) c.dst[i] = c.src[i];
        }
    }
}

ppf_status_t from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return PPF_OK;
    if (e == cudaErrorMemoryAllocation) return PPF_ERR_OUT_OF_MEMORY;
    return PPF_ERR_CUDA;
}

}  // namespace

struct ppf_server_s {
    struct Sub {
        const void* chunk;
        int64_t n;
        void* out;
        int64_t cap;
    };
    struct Slot {
        bool used = false;
        ppf_plan_t plan = nullptr;
        ppf::PlanView view;
        ppf::KernelEntry entry;
        int bps = 0;
        unsigned char* buf[2] = {nullptr, nullptr};
        int64_t cap = 0;       // samples per buffer
        int cur = 0;
        int64_t held = 0;      // samples in buf[cur]
        int64_t base = 0;      // stream index of buf[cur][0]
        int64_t pushed = 0;
        int64_t emitted = 0;
        int64_t max_chunk = 0;
        size_t bytes = 0;      // device bytes reserved by the slot
        std::vector<Sub> queue;
        std::vector<int64_t> done;  // spectra written per submission of the last tick
        bool mix = false;           // runs on the mixed-shape kernel
    };
    std::vector<Slot> slots;
    size_t budget = 0;
    size_t reserved = 0;
    int sms = 0;
    // staging: two pinned host slots + their device mirrors
    unsigned char* host_stage[2] = {nullptr, nullptr};
    unsigned char* dev_stage[2] = {nullptr, nullptr};
    size_t stage_cap = 0;
    cudaEvent_t stage_free[2] = {nullptr, nullptr};
    int stage_idx = 0;
    // groups of a tick run concurrently on these streams (fork/join with events)
    static constexpr int kLanes = 4;
    cudaStream_t lane[kLanes] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kLanes] = {};
    int64_t ticks = 0;
    int last_launches = 0;
    // the tick as a CUDA graph: fixed device tables (capacities from the
    // admitted streams), re-captured when a stream is admitted or released
    struct Layout {
        size_t counts_at = 0, gather_at = 0, carry_at = 0, mjobs_at = 0, mitems_at = 0, mnext_at = 0, bytes = 0;
        int cap_gather = 0, cap_carry = 0, cap_mjobs = 0, cap_mitems = 0;
        bool has_mix = false;
        int mix_grid = 0;
        int* mix_err = nullptr;
        std::vector<std::string> keys;  // work-list kernel groups
        std::vector<ppf::PlanView> gview;
        std::vector<ppf::KernelEntry> gentry;
        std::vector<size_t> gjobs_at, gitems_at;
        std::vector<int> cap_gjobs, cap_gitems, ggrid;
    } lay;
    bool graph_dirty = true;
    bool graph_ok = false;      // every admitted stream can run in the graph
    int mix_grid = 0;
    unsigned char* tab_dev = nullptr;
    unsigned char* tab_host[2] = {nullptr, nullptr};
    size_t tab_cap = 0;
    cudaEvent_t tab_free[2] = {nullptr, nullptr};
    int tab_idx = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_launches = 0;
    int64_t graph_ticks = 0;
};

namespace {

ppf_status_t grow_stage(ppf_server_s* s, size_t need)
{
    if (need <= s->stage_cap) return PPF_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return from_cuda(e);
    size_t cap = s->stage_cap ? s->stage_cap : (1 << 20);
    while (cap < need) cap *= 2;
    for (int i = 0; i < 2; ++i) {
        if (s->host_stage[i]) cudaFreeHost(s->host_stage[i]);
        if (s->dev_stage[i]) cudaFree(s->dev_stage[i]);
        s->host_stage[i] = nullptr;
        s->dev_stage[i] = nullptr;
    }
    s->stage_cap = 0;
    for (int i = 0; i < 2; ++i) {
        e = cudaHostAlloc(reinterpret_cast<void**>(&s->host_stage[i]), cap, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->dev_stage[i]), cap);
        if (e != cudaSuccess) return from_cuda(e);
    }
    s->stage_cap = cap;
    return PPF_OK;
}

void add_copy(std::vector<CopySeg>& segs, const void* src, void* dst, int64_t bytes)
{
    const unsigned char* s = static_cast<const unsigned char*>(src);
    unsigned char* d = static_cast<unsigned char*>(dst);
    for (int64_t off = 0; off < bytes; off += kSeg)
        segs.push_back({s + off, d + off, std::min(kSeg, bytes - off)});
}


std::string group_key(const ppf_server_s::Slot& sl)
{
    char key[160];
    std::snprintf(key, sizeof(key), "%d:%d:%d:%s", sl.view.N, sl.view.T, sl.view.dtype, sl.entry.name);
    return key;
}

int segs_for(int64_t bytes) { return (int)((bytes + kSeg - 1) / kSeg); }

// Fixed table layout for the admitted streams; false when a stream has no
// work-list form (the general kernel), which keeps the tick out of a graph.
bool build_layout(ppf_server_s* s)
{
    ppf_server_s::Layout L;
    L.mix_grid = s->mix_grid;
    std::map<std::string, int> gi;
    for (auto& sl : s->slots) {
        if (!sl.used) continue;
        const int64_t N = sl.view.N, T = sl.view.T, B = sl.bps;
        L.cap_gather += 4 * (segs_for((T + 1) * N * B) + segs_for(sl.max_chunk * B) + 2);
        L.cap_carry += segs_for((T + 1) * N * B) + 1;
        if (sl.mix) {
            L.has_mix = true;
            L.cap_mjobs += 8;
            if (!L.mix_err) L.mix_err = sl.view.err;
            continue;
        }
        if (!sl.entry.launch_work) return false;
        const std::string k = group_key(sl);
        auto it = gi.find(k);
        if (it == gi.end()) {
            gi[k] = (int)L.keys.size();
            L.keys.push_back(k);
            L.gview.push_back(sl.view);
            L.gentry.push_back(sl.entry);
            L.cap_gjobs.push_back(8);
            const int units = std::max(1, sl.view.grid_cap / sl.entry.cluster);
            L.ggrid.push_back(units * sl.entry.cluster);
        } else {
            L.cap_gjobs[it->second] += 8;
        }
    }
    L.cap_mitems = L.cap_mjobs + (ppf::kMixItemsPerCta + 4) * L.mix_grid;
    for (size_t g = 0; g < L.keys.size(); ++g) {
        const int units = L.ggrid[g] / L.gentry[g].cluster;
        L.cap_gitems.push_back(L.cap_gjobs[g] + 4 * units + 8);
    }
    size_t off = 0;
    auto place = [&](size_t n) {
        off = (off + 15) / 16 * 16;
        const size_t at = off;
        off += n;
        return at;
    };
    L.counts_at = place(sizeof(int) * (3 + L.keys.size()));
    L.gather_at = place(sizeof(CopySeg) * L.cap_gather);
    L.carry_at = place(sizeof(CopySeg) * L.cap_carry);
    L.mjobs_at = place(sizeof(ppf::MixJob) * L.cap_mjobs);
    L.mitems_at = place(sizeof(ppf::MixItem) * L.cap_mitems);
    L.mnext_at = place(sizeof(int) * 4);
    for (size_t g = 0; g < L.keys.size(); ++g) {
        L.gjobs_at.push_back(place(sizeof(ppf::PpfJob) * L.cap_gjobs[g]));
        L.gitems_at.push_back(place(sizeof(ppf::PpfItem) * L.cap_gitems[g]));
    }
    L.bytes = off + 16;
    s->lay = L;
    return true;
}

// The tick's kernels on s->cap_stream, reading every table (and count) from
// s->tab_dev: gather copy, then the mixed kernel and one work-list launch per
// kernel group on the lanes (forked and joined), then the carry copy.
cudaError_t enqueue_graph_tick(ppf_server_s* s, cudaStream_t st, int* launches)
{
    const ppf_server_s::Layout& L = s->lay;
    unsigned char* d = s->tab_dev;
    const int* counts = reinterpret_cast<const int*>(d + L.counts_at);
    const int cgrid = 4 * s->sms;
    int n = 0;
    batched_copy<<<cgrid, 256, 0, st>>>(reinterpret_cast<const CopySeg*>(d + L.gather_at), 0, counts + 0);
    ppf::note_launch();
    ++n;
    cudaError_t e = cudaGetLastError();
    const int nwork = (L.has_mix ? 1 : 0) + (int)L.keys.size();
    const int nl = std::min(ppf_server_s::kLanes, std::max(1, nwork));
    if (e == cudaSuccess) e = cudaEventRecord(s->fork_ev, st);
    for (int l = 0; l < nl && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(s->lane[l], s->fork_ev, 0);
    int w = 0;
    if (L.has_mix && e == cudaSuccess) {
        ppf::MixWork mw{};
        mw.jobs = reinterpret_cast<const ppf::MixJob*>(d + L.mjobs_at);
        mw.items = reinterpret_cast<const ppf::MixItem*>(d + L.mitems_at);
        mw.n_items_dev = counts + 2 + (int)L.keys.size();
        mw.next = reinterpret_cast<int*>(d + L.mnext_at);
        e = ppf::mix_launch(mw, L.mix_grid, L.mix_err, s->lane[w++ % nl]);
        ++n;
    }
    for (size_t g = 0; g < L.keys.size() && e == cudaSuccess; ++g) {
        ppf::PpfWork pw{};
        pw.jobs = reinterpret_cast<const ppf::PpfJob*>(d + L.gjobs_at[g]);
        pw.items = reinterpret_cast<const ppf::PpfItem*>(d + L.gitems_at[g]);
        pw.n_items = 0;
        pw.n_items_dev = counts + 2 + g;
        e = L.gentry[g].launch_work(L.gview[g], pw, L.ggrid[g], s->lane[w++ % nl]);
        ++n;
    }
    for (int l = 0; l < nl && e == cudaSuccess; ++l) {
        e = cudaEventRecord(s->join_ev[l], s->lane[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->join_ev[l], 0);
    }
    if (e == cudaSuccess) {
        batched_copy<<<cgrid, 256, 0, st>>>(reinterpret_cast<const CopySeg*>(d + L.carry_at), 0, counts + 1);
        ppf::note_launch();
        ++n;
        e = cudaGetLastError();
    }
    *launches = n;
    return e;
}

// Rebuild the layout and re-capture the graph (device synchronised first:
// no tick in flight reads the old tables).
ppf_status_t recapture(ppf_server_s* s)
{
    s->graph_dirty = false;
    s->graph_ok = false;
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    if (!build_layout(s)) return PPF_OK;  // a stream on the general kernel: direct launches
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return from_cuda(e);
    if (s->lay.bytes > s->tab_cap) {
        if (s->tab_dev) cudaFree(s->tab_dev);
        s->tab_dev = nullptr;
        for (int i = 0; i < 2; ++i) {
            if (s->tab_host[i]) cudaFreeHost(s->tab_host[i]);
            s->tab_host[i] = nullptr;
        }
        s->tab_cap = 0;
        size_t cap = 1 << 16;
        while (cap < s->lay.bytes) cap *= 2;
        e = cudaMalloc(reinterpret_cast<void**>(&s->tab_dev), cap);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i)
            e = cudaHostAlloc(reinterpret_cast<void**>(&s->tab_host[i]), cap, cudaHostAllocDefault);
        if (e != cudaSuccess) return from_cuda(e);
        s->tab_cap = cap;
    }
    if (!s->cap_stream) {
        e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return from_cuda(e);
    }
    e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return from_cuda(e);
    int n = 0;
    const cudaError_t le = enqueue_graph_tick(s, s->cap_stream, &n);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return from_cuda(le != cudaSuccess ? le : e);
    }
    e = cudaGraphInstantiate(&s->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return from_cuda(e);
    s->graph_launches = n;
    s->graph_ok = true;
    return PPF_OK;
}
}  // namespace

extern "C" {

ppf_status_t ppf_server_destroy(ppf_server_t s);

ppf_status_t ppf_server_create(ppf_server_t* out, int max_streams, size_t memory_budget_bytes)
{
    if (!out || max_streams < 1 || max_streams > 65536) return PPF_ERR_INVALID_ARG;
    *out = nullptr;
    ppf_server_s* s = new (std::nothrow) ppf_server_s();
    if (!s) return PPF_ERR_OUT_OF_MEMORY;
    s->slots.resize(max_streams);
    s->budget = memory_budget_bytes;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->stage_free[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->tab_free[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = ppf::mix_prepare(dev, &s->mix_grid);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming);
    for (int i = 0; i < ppf_server_s::kLanes && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&s->lane[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->join_ev[i], cudaEventDisableTiming);
    }
    // staging sized up front (64 KiB per stream, 4..64 MiB) so a busy tick
    // does not stall on a reallocation
    if (e == cudaSuccess) {
        const size_t want = std::min<size_t>(64u << 20, std::max<size_t>(4u << 20, (size_t)max_streams << 16));
        const ppf_status_t ps = grow_stage(s, want);
        if (ps != PPF_OK) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        ppf_server_destroy(s);
        return from_cuda(e);
    }
    *out = s;
    return PPF_OK;
}

ppf_status_t ppf_server_admit(ppf_server_t s, ppf_plan_t plan, int64_t max_chunk_samples, int* slot_out)
{
    if (!s || !plan || !slot_out || max_chunk_samples < 1) return PPF_ERR_INVALID_ARG;
    *slot_out = -1;
    ppf::PlanView v;
    ppf::KernelEntry e;
    int bps = 0;
    if (!ppf::plan_info(plan, &v, &e, &bps)) return PPF_ERR_INVALID_ARG;
    int free_slot = -1;
    for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].used) {
            free_slot = (int)i;
            break;
        }
    if (free_slot < 0) return PPF_ERR_BUSY;
    // Two buffers, each able to hold four boundary regions (history plus a
    // prefix, at most 2*T*N samples each) or the history plus four chunks.
    const int64_t cap = (8 * (int64_t)v.T * v.N + 4 * max_chunk_samples + 2 * v.N);
    const size_t bytes = 2 * (size_t)cap * bps;
    size_t free_b = 0, total_b = 0;
    cudaError_t ce = cudaMemGetInfo(&free_b, &total_b);
    if (ce != cudaSuccess) return from_cuda(ce);
    if (s->reserved + bytes > s->budget || bytes + (64u << 20) > free_b) return PPF_ERR_OUT_OF_MEMORY;
    ppf_server_s::Slot& sl = s->slots[free_slot];
    for (int i = 0; i < 2; ++i) {
        ce = cudaMalloc(reinterpret_cast<void**>(&sl.buf[i]), (size_t)cap * bps);
        if (ce != cudaSuccess) {
            if (sl.buf[0]) cudaFree(sl.buf[0]);
            sl.buf[0] = sl.buf[1] = nullptr;
            return from_cuda(ce);
        }
    }
    sl.used = true;
    sl.plan = plan;
    sl.view = v;
    sl.entry = e;
    sl.bps = bps;
    sl.cap = cap;
    sl.cur = 0;
    sl.held = sl.base = sl.pushed = sl.emitted = 0;
    sl.max_chunk = max_chunk_samples;
    sl.bytes = bytes;
    sl.queue.clear();
    sl.done.clear();
    sl.mix = ppf::plan_mixable(plan) && ppf::mix_shape(v.N, v.T) >= 0;
    s->reserved += bytes;
    s->graph_dirty = true;
    *slot_out = free_slot;
    return PPF_OK;
}

ppf_status_t ppf_server_release(ppf_server_t s, int slot)
{
    if (!s || slot < 0 || slot >= (int)s->slots.size() || !s->slots[slot].used) return PPF_ERR_INVALID_ARG;
    ppf_server_s::Slot& sl = s->slots[slot];
    if (!sl.queue.empty()) return PPF_ERR_BUSY;
    cudaError_t e = cudaDeviceSynchronize();
    for (int i = 0; i < 2; ++i)
        if (sl.buf[i]) cudaFree(sl.buf[i]);
    s->reserved -= sl.bytes;
    sl = ppf_server_s::Slot();
    s->graph_dirty = true;
    return from_cuda(e);
}

ppf_status_t ppf_server_submit(ppf_server_t s, int slot, const void* d_chunk, int64_t n_samples, void* d_out,
                               int64_t out_capacity_spectra)
{
    if (!s || slot < 0 || slot >= (int)s->slots.size() || !s->slots[slot].used) return PPF_ERR_INVALID_ARG;
    ppf_server_s::Slot& sl = s->slots[slot];
    if (n_samples < 0 || n_samples > sl.max_chunk || (n_samples > 0 && !d_chunk) || out_capacity_spectra < 0)
        return PPF_ERR_INVALID_ARG;
    int64_t queued = 0;
    for (auto& q : sl.queue) queued += q.n;
    if (sl.queue.size() >= 4) return PPF_ERR_BUSY;  // at most four chunks between ticks: tick first
    // spectra this submission completes
    const int64_t N = sl.view.N, T = sl.view.T;
    const int64_t before = std::max<int64_t>(0, (sl.pushed + queued) / N - T + 1);
    const int64_t after = std::max<int64_t>(0, (sl.pushed + queued + n_samples) / N - T + 1);
    if (after - before > out_capacity_spectra) return PPF_ERR_INVALID_ARG;
    if (after > before && (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15u))) return PPF_ERR_MISALIGNED;
    sl.queue.push_back({d_chunk, n_samples, d_out, out_capacity_spectra});
    return PPF_OK;
}

ppf_status_t ppf_server_submit_many(ppf_server_t s, int n, const int* slots, const void* const* chunks,
                                    const int64_t* n_samples, void* const* outs, const int64_t* caps, int* statuses)
{
    if (!s || n < 0 || (n > 0 && (!slots || !chunks || !n_samples || !outs || !caps))) return PPF_ERR_INVALID_ARG;
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        const ppf_status_t st = ppf_server_submit(s, slots[i], chunks[i], n_samples[i], outs[i], caps[i]);
        if (statuses) statuses[i] = (int)st;
        bad += st != PPF_OK;
    }
    return bad ? PPF_ERR_BUSY : PPF_OK;
}

ppf_status_t ppf_server_tick(ppf_server_t s, void* stream, int* n_done)
{
    if (!s) return PPF_ERR_INVALID_ARG;
    if (n_done) *n_done = 0;
    if (cudaPeekAtLastError() != cudaSuccess) return PPF_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // 1. host bookkeeping: gather copies, PPF jobs, carry copies
    std::vector<CopySeg> gather, carry;
    struct G {
        ppf::PlanView view;
        ppf::KernelEntry entry;
        std::vector<ppf::PpfJob> jobs;
    };
    std::map<std::string, G> groups;
    std::vector<std::string> order;
    struct Single {
        ppf::PlanView view;
        ppf::KernelEntry entry;
        const void* in;
        float2* out;
        int64_t S;
    };
    std::vector<Single> singles;
    std::vector<ppf::MixJob> mjobs;
    std::vector<ppf::MixJobInfo> minfo;
    int processed = 0;
    auto add_job = [&](ppf_server_s::Slot& sl, const void* in, float2* out, int64_t count) {
        if (sl.mix) {
            ppf::MixJob mj{};
            mj.x = in;
            mj.Y = out;
            mj.h = sl.view.h;
            mj.tw = sl.view.tw;
            mj.S = count;
            mj.shape = ppf::mix_shape(sl.view.N, sl.view.T);
            mjobs.push_back(mj);
            minfo.push_back({sl.view.N, sl.view.T, count});
            return;
        }
        if (sl.entry.launch_work) {
            char key[160];
            std::snprintf(key, sizeof(key), "%d:%d:%d:%s", sl.view.N, sl.view.T, sl.view.dtype, sl.entry.name);
            auto it = groups.find(key);
            if (it == groups.end()) {
                groups[key] = G{sl.view, sl.entry, {}};
                order.push_back(key);
                it = groups.find(key);
            }
            ppf::PpfJob j{};
            j.x = in;
            j.Y = out;
            j.h = sl.view.h;
            j.S = count;
            it->second.jobs.push_back(j);
        } else {
            singles.push_back({sl.view, sl.entry, in, out, count});
        }
    };
    for (auto& sl : s->slots) {
        if (!sl.used || sl.queue.empty()) continue;
        const int64_t N = sl.view.N, T = sl.view.T, B = sl.bps;
        unsigned char* H = sl.buf[sl.cur];      // persistent history, starts at stream sample base
        unsigned char* O = sl.buf[sl.cur ^ 1];  // scratch for boundary regions during the tick
        sl.done.assign(sl.queue.size(), 0);
        // The history (stream samples [emitted*N, pushed)) as (pointer, length).
        // It starts at H[0]; afterwards it is the tail of a chunk or the tail
        // of a boundary region.  A region is extended in place when the
        // history is its tail, and a new region is started in O otherwise, so
        // every copy of the tick reads only chunks or H and no copy reads
        // what another copy of the same launch writes.
        const unsigned char* hist = H;
        int64_t hist_len = sl.held;
        unsigned char* tail_end = H + sl.held * B;  // end of the region holding the history
        int64_t o_off = 0;                          // samples of O used by regions this tick
        for (size_t qi = 0; qi < sl.queue.size(); ++qi) {
            const auto& q = sl.queue[qi];
            const int64_t P = sl.pushed, n = q.n, total = P + n;
            if (n == 0) {
                ++processed;
                continue;
            }
            const int64_t e = sl.emitted;
            const int64_t complete = std::max<int64_t>(e, total / N - T + 1);
            const unsigned char* chunk = static_cast<const unsigned char*>(q.chunk);
            const int64_t r0 = (P + N - 1) / N;              // first row starting in the chunk
            const int64_t s1 = std::max(e, r0);              // spectra read in place: [s1, complete)
            const int64_t bnd_end = std::min(s1, complete);  // spectra needing the history: [e, bnd_end)
            const unsigned char* main_in = chunk + (s1 * N - P) * B;
            const bool in_place = complete > e && complete * N >= P &&
                                  (complete <= s1 || (reinterpret_cast<uintptr_t>(main_in) & 15u) == 0);
            // samples of the chunk the boundary region needs: the prefix that
            // completes spectra [e, bnd_end), or the whole chunk otherwise
            const int64_t prefix = in_place ? (bnd_end > e ? std::min(total, (bnd_end - 1 + T) * N) - P : 0) : n;
            const unsigned char* region = nullptr;
            if (prefix > 0) {
                if (hist + hist_len * B == tail_end) {
                    // the history is the tail of the current region: extend it
                    add_copy(gather, chunk, tail_end, prefix * B);
                    region = hist;
                    tail_end += prefix * B;
                    if (tail_end > O && tail_end <= O + sl.cap * B) o_off = (tail_end - O) / B;
                } else {
                    // the history is the tail of a chunk: new region in O (16-byte aligned)
                    const int64_t align = 16 / B;
                    o_off = (o_off + align - 1) / align * align;
                    unsigned char* r = O + o_off * B;
                    if (hist_len > 0) add_copy(gather, hist, r, hist_len * B);
                    add_copy(gather, chunk, r + hist_len * B, prefix * B);
                    o_off += hist_len + prefix;
                    region = r;
                    tail_end = r + (hist_len + prefix) * B;
                }
            }
            float2* out = static_cast<float2*>(q.out);
            if (in_place) {
                if (bnd_end > e) add_job(sl, region, out, bnd_end - e);
                if (complete > s1) add_job(sl, main_in, out + (s1 - e) * N, complete - s1);
                hist = chunk + (complete * N - P) * B;
            } else {
                if (complete > e) add_job(sl, region, out, complete - e);
                hist = region + (complete - e) * N * B;
            }
            hist_len = total - complete * N;
            sl.done[qi] = complete - e;
            sl.emitted = complete;
            sl.pushed = total;
            ++processed;
        }
        // carry the history into a buffer the next tick can extend
        if (hist == H) {
            // unchanged start: nothing to move
        } else if (hist >= H && hist < H + sl.cap * B) {
            if (hist_len > 0) add_copy(carry, hist, O, hist_len * B);
            sl.cur ^= 1;
        } else {
            if (hist_len > 0) add_copy(carry, hist, H, hist_len * B);
        }
        sl.base = sl.emitted * N;
        sl.held = hist_len;
        sl.queue.clear();
    }
    if (processed == 0) return PPF_OK;

    // 2. item lists: the mixed kernel's per-CTA segments; per kernel group,
    //    pieces of about a quarter of a unit's share, largest first
    std::vector<ppf::MixItem> mitems;
    if (!mjobs.empty()) ppf::mix_items(minfo.data(), (int)minfo.size(), s->mix_grid, mitems);
    auto group_items = [&](const G& g, std::vector<ppf::PpfItem>& items) {
        const int RB = g.entry.rows_per_block;
        const int units = std::max(1, g.view.grid_cap / g.entry.cluster);
        int64_t total = 0;
        for (auto& j : g.jobs) total += (j.S + RB - 1) / RB;
        // long enough that the T-1 halo rows and the pipeline fill stay small against the work
        const int64_t min_len = std::max<int64_t>(8, (4 * (int64_t)g.view.T + RB - 1) / RB);
        const int64_t target = std::max<int64_t>(min_len, (total + 4 * units - 1) / (4 * units));
        for (size_t ji = 0; ji < g.jobs.size(); ++ji) {
            const int64_t nblk = (g.jobs[ji].S + RB - 1) / RB;
            const int64_t pieces = std::max<int64_t>(1, (nblk + target / 2) / target);
            for (int64_t k = 0; k < pieces; ++k) {
                ppf::PpfItem it{};
                it.job = (int)ji;
                it.blo = nblk * k / pieces;
                it.bhi = nblk * (k + 1) / pieces;
                if (it.bhi > it.blo) items.push_back(it);
            }
        }
        // round-robin over units then balances like LPT
        std::stable_sort(items.begin(), items.end(), [](const ppf::PpfItem& x, const ppf::PpfItem& y) {
            return (x.bhi - x.blo) > (y.bhi - y.blo);
        });
    };

    // 3. the tick as a replay of the captured graph: upload the tables into
    //    the fixed device area, launch the graph
    if (s->graph_dirty) {
        const ppf_status_t ps = recapture(s);
        if (ps != PPF_OK) return ps;
    }
    if (s->graph_ok && singles.empty()) {
        const ppf_server_s::Layout& L = s->lay;
        bool fits = (int)gather.size() <= L.cap_gather && (int)carry.size() <= L.cap_carry &&
                    (int)mjobs.size() <= L.cap_mjobs && (int)mitems.size() <= L.cap_mitems &&
                    (mjobs.empty() || L.has_mix);
        std::vector<std::vector<ppf::PpfItem>> gitems(L.keys.size());
        std::vector<const G*> gsrc(L.keys.size(), nullptr);
        for (auto& kv : groups) {
            const auto pos = std::find(L.keys.begin(), L.keys.end(), kv.first);
            if (pos == L.keys.end()) {
                fits = false;
                break;
            }
            const size_t gi = (size_t)(pos - L.keys.begin());
            gsrc[gi] = &kv.second;
            group_items(kv.second, gitems[gi]);
            if ((int)kv.second.jobs.size() > L.cap_gjobs[gi] || (int)gitems[gi].size() > L.cap_gitems[gi]) fits = false;
        }
        if (fits) {
            const int k = s->tab_idx;
            s->tab_idx ^= 1;
            cudaError_t e = cudaEventSynchronize(s->tab_free[k]);
            if (e != cudaSuccess) return from_cuda(e);
            unsigned char* h = s->tab_host[k];
            unsigned char* d = s->tab_dev;
            std::vector<int> counts(3 + L.keys.size());
            counts[0] = (int)gather.size();
            counts[1] = (int)carry.size();
            for (size_t g = 0; g < L.keys.size(); ++g) counts[2 + g] = (int)gitems[g].size();
            counts[2 + L.keys.size()] = (int)mitems.size();
            const int zero4[4] = {0, 0, 0, 0};
            auto stage = [&](size_t at, const void* src, size_t n) {
                if (n == 0 || e != cudaSuccess) return;
                std::memcpy(h + at, src, n);
                e = cudaMemcpyAsync(d + at, h + at, n, cudaMemcpyHostToDevice, st);
            };
            stage(L.counts_at, counts.data(), sizeof(int) * counts.size());
            stage(L.gather_at, gather.data(), sizeof(CopySeg) * gather.size());
            stage(L.carry_at, carry.data(), sizeof(CopySeg) * carry.size());
            if (L.has_mix) {
                stage(L.mjobs_at, mjobs.data(), sizeof(ppf::MixJob) * mjobs.size());
                stage(L.mitems_at, mitems.data(), sizeof(ppf::MixItem) * mitems.size());
                stage(L.mnext_at, zero4, sizeof(zero4));  // the item counter starts from zero
            }
            for (size_t g = 0; g < L.keys.size(); ++g) {
                if (!gsrc[g]) continue;
                stage(L.gjobs_at[g], gsrc[g]->jobs.data(), sizeof(ppf::PpfJob) * gsrc[g]->jobs.size());
                stage(L.gitems_at[g], gitems[g].data(), sizeof(ppf::PpfItem) * gitems[g].size());
            }
            if (e == cudaSuccess) e = cudaEventRecord(s->tab_free[k], st);
            if (e == cudaSuccess) e = cudaGraphLaunch(s->exec, st);
            if (e != cudaSuccess) return from_cuda(e);
            s->last_launches = s->graph_launches;
            ++s->ticks;
            ++s->graph_ticks;
            if (n_done) *n_done = processed;
            return PPF_OK;
        }
    }

    // 4. direct launches (a stream on the general kernel, or tables beyond
    //    the graph's capacities)
    struct Tab {
        size_t jobs_at, items_at;
        std::vector<ppf::PpfItem> items;
        int grid;
    };
    std::vector<Tab> tabs(order.size());
    size_t off = 0;
    auto place = [&](size_t n, size_t align) {
        off = (off + align - 1) / align * align;
        const size_t at = off;
        off += n;
        return at;
    };
    const size_t gather_at = place(sizeof(CopySeg) * gather.size(), 16);
    const size_t carry_at = place(sizeof(CopySeg) * carry.size(), 16);
    const size_t mjobs_at = place(sizeof(ppf::MixJob) * mjobs.size(), 16);
    const size_t mitems_at = place(sizeof(ppf::MixItem) * mitems.size(), 16);
    const size_t mnext_at = place(sizeof(int) * 4, 16);
    for (size_t gi = 0; gi < order.size(); ++gi) {
        G& g = groups[order[gi]];
        Tab& tb = tabs[gi];
        group_items(g, tb.items);
        const int units = std::max(1, g.view.grid_cap / g.entry.cluster);
        tb.grid = std::min<int>(units, (int)tb.items.size()) * g.entry.cluster;
        tb.jobs_at = place(sizeof(ppf::PpfJob) * g.jobs.size(), 16);
        tb.items_at = place(sizeof(ppf::PpfItem) * tb.items.size(), 16);
    }
    ppf_status_t ps = grow_stage(s, off + 256);
    if (ps != PPF_OK) return ps;

    // 3. fill the staging slot (after the tick that last used it has uploaded it)
    const int k = s->stage_idx;
    s->stage_idx ^= 1;
    cudaError_t e = cudaEventSynchronize(s->stage_free[k]);
    if (e != cudaSuccess) return from_cuda(e);
    unsigned char* hs = s->host_stage[k];
    unsigned char* ds = s->dev_stage[k];
    std::memcpy(hs + gather_at, gather.data(), sizeof(CopySeg) * gather.size());
    std::memcpy(hs + carry_at, carry.data(), sizeof(CopySeg) * carry.size());
    std::memcpy(hs + mjobs_at, mjobs.data(), sizeof(ppf::MixJob) * mjobs.size());
    std::memcpy(hs + mitems_at, mitems.data(), sizeof(ppf::MixItem) * mitems.size());
    std::memset(hs + mnext_at, 0, sizeof(int) * 4);  // the item counter starts from zero
    std::vector<ppf::PpfWork> works(order.size());
    for (size_t gi = 0; gi < order.size(); ++gi) {
        G& g = groups[order[gi]];
        Tab& tb = tabs[gi];
        std::memcpy(hs + tb.jobs_at, g.jobs.data(), sizeof(ppf::PpfJob) * g.jobs.size());
        std::memcpy(hs + tb.items_at, tb.items.data(), sizeof(ppf::PpfItem) * tb.items.size());
        works[gi].jobs = reinterpret_cast<const ppf::PpfJob*>(ds + tb.jobs_at);
        works[gi].items = reinterpret_cast<const ppf::PpfItem*>(ds + tb.items_at);
        works[gi].n_items = (int)tb.items.size();
    }
    e = cudaMemcpyAsync(ds, hs, off, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->stage_free[k], st);
    if (e != cudaSuccess) return from_cuda(e);

    // 4. launches: gather, PPF groups, general-kernel jobs, carry
    int launches = 0;
    const int cgrid = std::max(1, std::min<int>((int)gather.size(), 4 * s->sms));
    if (!gather.empty()) {
        batched_copy<<<cgrid, 256, 0, st>>>(reinterpret_cast<const CopySeg*>(ds + gather_at), (int)gather.size(),
                                            nullptr);
        ppf::note_launch();
        ++launches;
    }
    // PPF groups run concurrently on the lanes, forked from and joined back
    // into the caller's stream, so one group's tail overlaps the next's start
    const bool mix = !mitems.empty();
    const int nwork = (int)order.size() + (int)singles.size() + (mix ? 1 : 0);
    const int nl = std::min(ppf_server_s::kLanes, std::max(1, nwork));
    if (e == cudaSuccess) e = cudaEventRecord(s->fork_ev, st);
    for (int l = 0; l < nl && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(s->lane[l], s->fork_ev, 0);
    int w = 0;
    if (mix && e == cudaSuccess) {
        ppf::MixWork mw{};
        mw.jobs = reinterpret_cast<const ppf::MixJob*>(ds + mjobs_at);
        mw.items = reinterpret_cast<const ppf::MixItem*>(ds + mitems_at);
        mw.n_items = (int)mitems.size();
        mw.next = reinterpret_cast<int*>(ds + mnext_at);
        int* err = nullptr;
        for (auto& sl : s->slots)
            if (sl.used && sl.mix) {
                err = sl.view.err;
                break;
            }
        e = ppf::mix_launch(mw, s->mix_grid, err, s->lane[w++ % nl]);
        ++launches;
    }
    for (size_t gi = 0; gi < order.size() && e == cudaSuccess; ++gi, ++w) {
        G& g = groups[order[gi]];
        e = g.entry.launch_work(g.view, works[gi], tabs[gi].grid, s->lane[w % nl]);
        ++launches;
    }
    // jobs on the general kernel (no work-list form): one launch each, on one lane
    for (auto& sg : singles) {
        if (e != cudaSuccess) break;
        e = sg.entry.launch(sg.view, sg.in, sg.out, sg.S, s->lane[0]);
        ++launches;
    }
    for (int l = 0; l < nl && e == cudaSuccess; ++l) {
        e = cudaEventRecord(s->join_ev[l], s->lane[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->join_ev[l], 0);
    }
    if (e == cudaSuccess && !carry.empty()) {
        const int kgrid = std::max(1, std::min<int>((int)carry.size(), 4 * s->sms));
        batched_copy<<<kgrid, 256, 0, st>>>(reinterpret_cast<const CopySeg*>(ds + carry_at), (int)carry.size(),
                                            nullptr);
        ppf::note_launch();
        ++launches;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return from_cuda(e);
    s->last_launches = launches;
    ++s->ticks;
    if (n_done) *n_done = processed;
    return PPF_OK;
}

ppf_status_t ppf_server_position(ppf_server_t s, int slot, int64_t* samples_in, int64_t* spectra_out)
{
    if (!s || slot < 0 || slot >= (int)s->slots.size() || !s->slots[slot].used) return PPF_ERR_INVALID_ARG;
    if (samples_in) *samples_in = s->slots[slot].pushed;
    if (spectra_out) *spectra_out = s->slots[slot].emitted;
    return PPF_OK;
}

ppf_status_t ppf_server_info(ppf_server_t s, size_t* reserved_bytes, int* streams, int* last_tick_launches)
{
    if (!s) return PPF_ERR_INVALID_ARG;
    int n = 0;
    for (auto& sl : s->slots) n += sl.used ? 1 : 0;
    if (reserved_bytes) *reserved_bytes = s->reserved;
    if (streams) *streams = n;
    if (last_tick_launches) *last_tick_launches = s->last_launches;
    return PPF_OK;
}

int64_t ppf_server_graph_ticks(ppf_server_t s) { return s ? s->graph_ticks : -1; }

ppf_status_t ppf_server_destroy(ppf_server_t s)
{
    if (!s) return PPF_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    for (auto& sl : s->slots)
        for (int i = 0; i < 2; ++i)
            if (sl.buf[i]) cudaFree(sl.buf[i]);
    for (int i = 0; i < 2; ++i) {
        if (s->host_stage[i]) cudaFreeHost(s->host_stage[i]);
        if (s->dev_stage[i]) cudaFree(s->dev_stage[i]);
        if (s->stage_free[i]) cudaEventDestroy(s->stage_free[i]);
    }
    for (int i = 0; i < ppf_server_s::kLanes; ++i) {
        if (s->lane[i]) cudaStreamDestroy(s->lane[i]);
        if (s->join_ev[i]) cudaEventDestroy(s->join_ev[i]);
    }
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->tab_dev) cudaFree(s->tab_dev);
    for (int i = 0; i < 2; ++i) {
        if (s->tab_host[i]) cudaFreeHost(s->tab_host[i]);
        if (s->tab_free[i]) cudaEventDestroy(s->tab_free[i]);
    }
    delete s;
    return from_cuda(e);
}

}  // extern "C"
