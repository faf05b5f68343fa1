// C ABI of the GB300 polyphase filter bank: plans, execution, streams.
// The operations are specified in include/ppf.h (Section 2 Eq. 1 and the DFT
// stage of arXiv 1411.3656); this file validates arguments, owns device
// memory for coefficients, twiddles and stream history, and picks a kernel.
#include "ppf.h"
#include "ppf_launch.h"

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

namespace ppf {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

KernelEntry select_fast_entry(int N, int T, int dtype, int variant, int out_f16);  // ppf_select.cu
KernelEntry fir_only_entry(int N, int T, int dtype);                                // ppf_fir.cu

}  // namespace ppf

using ppf::KernelEntry;
using ppf::PlanView;

struct ppf_plan_s {
    PlanView view;           // launch parameters (device pointers inside)
    PlanView fir_view;       // FIR-only view (PPF_FLAG_FIR_ONLY)
    KernelEntry entry;       // kernel ppf_execute launches
    KernelEntry fir_entry;   // FIR-only kernel (or the general kernel in FIR-only mode)
    ppf_dtype_t dtype = PPF_IN_C32;
    unsigned flags = 0;
    int device = 0;
    void* d_h = nullptr;
    float2* d_tw = nullptr;
    int* h_err = nullptr;    // mapped host word a kernel sets when a bounded wait gives up
    // staging for ppf_execute_host (allocated on first use): kHostSlots
    // slots of input and output, one stream per stage (upload, kernel,
    // download) and per slot the events that hand a slice between stages
    static constexpr int kHostSlots = 3;
    std::mutex host_mu;
    void* d_stage_in[kHostSlots] = {};
    float2* d_stage_out[kHostSlots] = {};
    int64_t stage_rows = 0;  // spectra per slice the staging buffers hold
    cudaStream_t copy_st[3] = {};               // upload, kernel, download
    cudaEvent_t ev_in[kHostSlots] = {};         // slice uploaded into the slot
    cudaEvent_t ev_k[kHostSlots] = {};          // slot's slice transformed (input slot free)
    cudaEvent_t ev_out[kHostSlots] = {};        // slot's spectra downloaded (output slot free)
};

struct ppf_stream_s {
    ppf_plan_t plan = nullptr;
    void* d_buf[2] = {nullptr, nullptr};  // history + newest samples, ping-pong
    int64_t cap = 0;                      // capacity of each buffer in samples
    int cur = 0;                          // buffer holding the live samples
    int64_t held = 0;                     // samples currently held
    int64_t base = 0;                     // stream index of d_buf[cur][0]
    int64_t pushed = 0;                   // total samples pushed
    int64_t emitted = 0;                  // total spectra emitted
    cudaStream_t last = nullptr;          // CUDA stream of the last push
    bool has_last = false;                // a push (or restore) has enqueued work on `last`
    cudaEvent_t order_ev = nullptr;       // orders a push after the previous one on another stream
};

namespace {
int sample_bytes(ppf_dtype_t d);
}

namespace ppf {
// Plan internals for the batch builder (ppf_batch.cu).
bool plan_info(ppf_plan_t plan, PlanView* view, KernelEntry* entry, int* bps)
{
    if (!plan || (plan->flags & PPF_FLAG_FIR_ONLY)) return false;
    *view = plan->view;
    *entry = plan->entry;
    *bps = sample_bytes(plan->dtype);
    return true;
}

// A plan the mixed-shape kernel may run: complex64 in and out, its tuned
// default kernel (no forced variant or general kernel).
bool plan_mixable(ppf_plan_t plan)
{
    return plan && plan->dtype == PPF_IN_C32 &&
           !(plan->flags & (PPF_FLAG_FIR_ONLY | PPF_FLAG_GENERIC | PPF_FLAG_OUT_F16 | 0xFF00u));
}

int plan_device(ppf_plan_t plan) { return plan ? plan->device : 0; }
}  // namespace ppf

namespace {

int sample_bytes(ppf_dtype_t d)
{
    switch (d) {
    case PPF_IN_C32: return 8;
    case PPF_IN_C16: return 4;
    case PPF_IN_CI8: return 2;
    default: return 0;
    }
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
    return a0 < b0 + nb && b0 < a0 + na;
}

ppf_status_t from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return PPF_OK;
    if (e == cudaErrorMemoryAllocation) return PPF_ERR_OUT_OF_MEMORY;
    return PPF_ERR_CUDA;
}

// Errors left by earlier asynchronous work (without clearing them).
bool pending_cuda_error() { return cudaPeekAtLastError() != cudaSuccess; }

void free_plan_memory(ppf_plan_s* p)
{
    if (p->d_h) cudaFree(p->d_h);
    if (p->d_tw) cudaFree(p->d_tw);
    if (p->h_err) cudaFreeHost(p->h_err);
    for (int i = 0; i < ppf_plan_s::kHostSlots; ++i) {
        if (p->d_stage_in[i]) cudaFree(p->d_stage_in[i]);
        if (p->d_stage_out[i]) cudaFree(p->d_stage_out[i]);
        if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
        if (p->ev_k[i]) cudaEventDestroy(p->ev_k[i]);
        if (p->ev_out[i]) cudaEventDestroy(p->ev_out[i]);
    }
    for (int i = 0; i < 3; ++i)
        if (p->copy_st[i]) cudaStreamDestroy(p->copy_st[i]);
}

}  // namespace

extern "C" {

const char* ppf_status_string(ppf_status_t s)
{
    switch (s) {
    case PPF_OK: return "PPF_OK";
    case PPF_ERR_INVALID_ARG: return "PPF_ERR_INVALID_ARG";
    case PPF_ERR_UNSUPPORTED: return "PPF_ERR_UNSUPPORTED";
    case PPF_ERR_MISALIGNED: return "PPF_ERR_MISALIGNED";
    case PPF_ERR_OUT_OF_MEMORY: return "PPF_ERR_OUT_OF_MEMORY";
    case PPF_ERR_CUDA: return "PPF_ERR_CUDA";
    case PPF_ERR_TIMEOUT: return "PPF_ERR_TIMEOUT";
    case PPF_ERR_BUSY: return "PPF_ERR_BUSY";
    default: return "PPF_ERR_UNKNOWN";
    }
}

int64_t ppf_launch_count(void) { return ppf::g_launches.load(); }

const char* ppf_plan_kernel_name(ppf_plan_t plan)
{
    if (!plan) return nullptr;
    return plan->flags & PPF_FLAG_FIR_ONLY ? plan->fir_entry.name : plan->entry.name;
}

ppf_status_t ppf_plan_create(ppf_plan_t* out, int N, int T, const float* h_host,
                             ppf_dtype_t in_dtype, unsigned flags)
{
    if (!out || !h_host) return PPF_ERR_INVALID_ARG;
    *out = nullptr;
    const int bps = sample_bytes(in_dtype);
    if (bps == 0) return PPF_ERR_UNSUPPORTED;
    if (!is_pow2(N) || N < 4 || N > 4096 || T < 1 || T > 64) return PPF_ERR_UNSUPPORTED;
    if (flags & ~(PPF_FLAG_FIR_ONLY | PPF_FLAG_GENERIC | PPF_FLAG_OUT_F16 | 0xFF00u)) return PPF_ERR_INVALID_ARG;
    if ((flags & PPF_FLAG_FIR_ONLY) && (flags & PPF_FLAG_OUT_F16)) return PPF_ERR_UNSUPPORTED;
    const int variant = (int)((flags >> 8) & 0xFFu) - 1;  // -1: tuned default
    if (variant >= 0 && variant >= ppf_variant_count(N, T, in_dtype)) return PPF_ERR_UNSUPPORTED;

    ppf_plan_s* p = new (std::nothrow) ppf_plan_s();
    if (!p) return PPF_ERR_OUT_OF_MEMORY;
    p->dtype = in_dtype;
    p->flags = flags;
    cudaError_t e = cudaGetDevice(&p->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return from_cuda(e);
    }

    // Coefficients: FP32 for complex64 input, FP16 for the reduced types.
    const size_t nh = (size_t)N * T;
    if (in_dtype == PPF_IN_C32) {
        e = cudaMalloc(&p->d_h, nh * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(p->d_h, h_host, nh * sizeof(float), cudaMemcpyHostToDevice);
    } else {
        std::vector<__half> h16(nh);
        for (size_t i = 0; i < nh; ++i) h16[i] = __float2half_rn(h_host[i]);
        e = cudaMalloc(&p->d_h, nh * sizeof(__half));
        if (e == cudaSuccess) e = cudaMemcpy(p->d_h, h16.data(), nh * sizeof(__half), cudaMemcpyHostToDevice);
    }
    // Twiddles W_N^m = exp(-2*pi*i*m/N), evaluated in FP64 and rounded to FP32.
    if (e == cudaSuccess) {
        std::vector<float2> tw(N);
        const double two_pi = 6.283185307179586476925286766559;
        for (int m = 0; m < N; ++m) {
            const double a = two_pi * (double)m / (double)N;
            tw[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
        }
        e = cudaMalloc(&p->d_tw, N * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemcpy(p->d_tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
    }
    int* d_err = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&p->h_err, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *p->h_err = 0;
        e = cudaHostGetDevicePointer((void**)&d_err, p->h_err, 0);
    }
    if (e != cudaSuccess) {
        free_plan_memory(p);
        delete p;
        return from_cuda(e);
    }

    PlanView v;
    v.N = N;
    v.T = T;
    v.dtype = (int)in_dtype;
    v.h = p->d_h;
    v.tw = p->d_tw;
    v.sms = sms;
    v.err = d_err;
    v.out_f16 = (flags & PPF_FLAG_OUT_F16) ? 1 : 0;
    p->view = v;
    p->fir_view = v;
    p->fir_view.fir_only = 1;

    // FIR-only mode: the FIR-only kernel where it has a tile shape, else the
    // general kernel's FIR-only form
    p->fir_entry = ppf::fir_only_entry(N, T, (int)in_dtype);
    if (!p->fir_entry.launch) p->fir_entry = ppf::generic_entry(N, (int)in_dtype);
    const int out_f16 = (flags & PPF_FLAG_OUT_F16) ? 1 : 0;
    const ppf::KernelEntry general = ppf::generic_entry(N, (int)in_dtype, out_f16);
    p->entry = (flags & PPF_FLAG_GENERIC) ? general : ppf::select_fast_entry(N, T, (int)in_dtype, variant, out_f16);
    if (!p->entry.launch) p->entry = general;
    if (!p->entry.launch || !p->fir_entry.launch) {
        free_plan_memory(p);
        delete p;
        return PPF_ERR_UNSUPPORTED;
    }
    e = p->entry.prepare(p->view);
    if (e == cudaSuccess) e = p->fir_entry.prepare(p->fir_view);
    if (e != cudaSuccess) {
        free_plan_memory(p);
        delete p;
        return from_cuda(e);
    }
    *out = p;
    return PPF_OK;
}

ppf_status_t ppf_plan_destroy(ppf_plan_t plan)
{
    if (!plan) return PPF_ERR_INVALID_ARG;
    free_plan_memory(plan);
    delete plan;
    return PPF_OK;
}

ppf_status_t ppf_execute(ppf_plan_t plan, const void* d_in, void* d_out, int64_t n_spectra,
                         void* stream)
{
    if (!plan || n_spectra < 0) return PPF_ERR_INVALID_ARG;
    if (n_spectra == 0) return PPF_OK;
    if (!d_in || !d_out) return PPF_ERR_INVALID_ARG;
    const PlanView& v = plan->view;
    if (!aligned16(d_in) || !aligned16(d_out)) return PPF_ERR_MISALIGNED;
    const size_t in_bytes = (size_t)(n_spectra + v.T - 1) * v.N * sample_bytes(plan->dtype);
    const size_t out_bytes = (size_t)n_spectra * v.N * (v.out_f16 ? 4 : sizeof(float2));
    if (overlaps(d_in, in_bytes, d_out, out_bytes)) return PPF_ERR_MISALIGNED;
    if (pending_cuda_error()) return PPF_ERR_CUDA;
    if (*(volatile int*)plan->h_err) return PPF_ERR_TIMEOUT;
    cudaError_t e;
    if (plan->flags & PPF_FLAG_FIR_ONLY)
        e = plan->fir_entry.launch(plan->fir_view, d_in, static_cast<float2*>(d_out), n_spectra,
                                   static_cast<cudaStream_t>(stream));
    else
        e = plan->entry.launch(v, d_in, static_cast<float2*>(d_out), n_spectra,
                               static_cast<cudaStream_t>(stream));
    return from_cuda(e);
}

ppf_status_t ppf_execute_host(ppf_plan_t plan, const void* h_in, void* h_out, int64_t n_spectra,
                              void* stream)
{
    if (!plan || n_spectra < 0) return PPF_ERR_INVALID_ARG;
    if (plan->view.out_f16) return PPF_ERR_UNSUPPORTED;
    if (n_spectra == 0) return PPF_OK;
    if (!h_in || !h_out) return PPF_ERR_INVALID_ARG;
    if (pending_cuda_error()) return PPF_ERR_CUDA;
    std::lock_guard<std::mutex> lock(plan->host_mu);
    const PlanView& v = plan->view;
    const int bps = sample_bytes(plan->dtype);
    const int64_t N = v.N, T = v.T;
    // Slices of about 16 Mi samples (shorter pipeline fill and drain per call
    // than 32 Mi, measured faster over the 20-cell sweep) in a three-stage
    // pipeline: the upload
    // stream copies slice s into slot s mod 3 once the kernel of slice s - 3
    // has read that slot, the kernel stream transforms it once it has landed
    // and the download of slice s - 3 has emptied the output slot, and the
    // download stream copies the spectra back; uploads and downloads of
    // different slices run at the same time (the link is full duplex).
    constexpr int NS = ppf_plan_s::kHostSlots;
    int64_t rows = (int64_t)((16ll << 20) / N);
    if (rows < 1) rows = 1;
    cudaError_t e = cudaSuccess;
    if (plan->stage_rows < rows) {
        for (int i = 0; i < NS; ++i) {
            if (plan->d_stage_in[i]) cudaFree(plan->d_stage_in[i]);
            if (plan->d_stage_out[i]) cudaFree(plan->d_stage_out[i]);
            plan->d_stage_in[i] = nullptr;
            plan->d_stage_out[i] = nullptr;
        }
        plan->stage_rows = 0;
        for (int i = 0; i < NS && e == cudaSuccess; ++i) {
            e = cudaMalloc(&plan->d_stage_in[i], (size_t)(rows + T - 1) * N * bps);
            if (e == cudaSuccess) e = cudaMalloc((void**)&plan->d_stage_out[i], (size_t)rows * N * sizeof(float2));
            if (e == cudaSuccess && !plan->ev_in[i]) e = cudaEventCreateWithFlags(&plan->ev_in[i], cudaEventDisableTiming);
            if (e == cudaSuccess && !plan->ev_k[i]) e = cudaEventCreateWithFlags(&plan->ev_k[i], cudaEventDisableTiming);
            if (e == cudaSuccess && !plan->ev_out[i])
                e = cudaEventCreateWithFlags(&plan->ev_out[i], cudaEventDisableTiming);
        }
        for (int i = 0; i < 3 && e == cudaSuccess; ++i)
            if (!plan->copy_st[i]) e = cudaStreamCreateWithFlags(&plan->copy_st[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) return from_cuda(e);
        plan->stage_rows = rows;
    }
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    cudaStream_t up = plan->copy_st[0], kst = plan->copy_st[1], down = plan->copy_st[2];
    cudaEvent_t start_ev;
    e = cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return from_cuda(e);
    // Work already queued on the caller's stream comes first.
    e = cudaEventRecord(start_ev, user);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(plan->copy_st[i], start_ev, 0);
    const char* src = static_cast<const char*>(h_in);
    char* dst = static_cast<char*>(h_out);
    int64_t slice = 0;
    for (int64_t s0 = 0; s0 < n_spectra && e == cudaSuccess; s0 += rows, ++slice) {
        const int k = (int)(slice % NS);
        const bool reuse = slice >= NS;
        const int64_t n = n_spectra - s0 < rows ? n_spectra - s0 : rows;
        // upload: the slot's previous slice has been read by its kernel
        if (reuse) e = cudaStreamWaitEvent(up, plan->ev_k[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(plan->d_stage_in[k], src + (size_t)s0 * N * bps, (size_t)(n + T - 1) * N * bps,
                                cudaMemcpyHostToDevice, up);
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_in[k], up);
        // kernel: the slice has landed and the slot's previous spectra are downloaded
        if (e == cudaSuccess) e = cudaStreamWaitEvent(kst, plan->ev_in[k], 0);
        if (e == cudaSuccess && reuse) e = cudaStreamWaitEvent(kst, plan->ev_out[k], 0);
        if (e == cudaSuccess) e = plan->entry.launch(v, plan->d_stage_in[k], plan->d_stage_out[k], n, kst);
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_k[k], kst);
        // download
        if (e == cudaSuccess) e = cudaStreamWaitEvent(down, plan->ev_k[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst + (size_t)s0 * N * sizeof(float2), plan->d_stage_out[k],
                                (size_t)n * N * sizeof(float2), cudaMemcpyDeviceToHost, down);
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_out[k], down);
    }
    for (int i = 0; i < 3; ++i) {
        cudaError_t e2 = cudaStreamSynchronize(plan->copy_st[i]);
        if (e == cudaSuccess) e = e2;
    }
    cudaEventDestroy(start_ev);
    return from_cuda(e);
}

ppf_status_t ppf_stream_open(ppf_plan_t plan, ppf_stream_t* out)
{
    if (!plan || !out) return PPF_ERR_INVALID_ARG;
    *out = nullptr;
    if (plan->view.out_f16) return PPF_ERR_UNSUPPORTED;
    ppf_stream_s* s = new (std::nothrow) ppf_stream_s();
    if (!s) return PPF_ERR_OUT_OF_MEMORY;
    s->plan = plan;
    *out = s;
    return PPF_OK;
}

ppf_status_t ppf_stream_position(ppf_stream_t s, int64_t* samples_in, int64_t* spectra_out)
{
    if (!s) return PPF_ERR_INVALID_ARG;
    if (samples_in) *samples_in = s->pushed;
    if (spectra_out) *spectra_out = s->emitted;
    return PPF_OK;
}

ppf_status_t ppf_stream_push(ppf_stream_t s, const void* d_chunk, int64_t n_samples, void* d_out,
                             int64_t out_capacity_spectra, int64_t* n_spectra_out, void* stream)
{
    if (!s || n_samples < 0 || out_capacity_spectra < 0) return PPF_ERR_INVALID_ARG;
    if (n_samples > 0 && !d_chunk) return PPF_ERR_INVALID_ARG;
    if (n_spectra_out) *n_spectra_out = 0;
    ppf_plan_t plan = s->plan;
    const int64_t N = plan->view.N, T = plan->view.T;
    const int bps = sample_bytes(plan->dtype);
    const int64_t total = s->pushed + n_samples;
    const int64_t complete = total / N - T + 1 > 0 ? total / N - T + 1 : 0;
    const int64_t fresh = complete - s->emitted;
    if (fresh > out_capacity_spectra) return PPF_ERR_INVALID_ARG;
    if (fresh > 0 && !d_out) return PPF_ERR_INVALID_ARG;
    if (fresh > 0 && !aligned16(d_out)) return PPF_ERR_MISALIGNED;
    if (pending_cuda_error()) return PPF_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;

    // Pushes of one stream object may come on different CUDA streams: this
    // push's copies, kernel and frees are ordered after everything the
    // previous push enqueued on its own stream.
    if (s->has_last && st != s->last) {
        if (!s->order_ev) e = cudaEventCreateWithFlags(&s->order_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(s->order_ev, s->last);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->order_ev, 0);
        if (e != cudaSuccess) return from_cuda(e);
    }

    // Grow the two buffers so they hold the history plus this chunk.
    const int64_t need = s->held + n_samples;
    if (need > s->cap) {
        int64_t cap = s->cap ? s->cap : (T + 1) * N;
        while (cap < need) cap *= 2;
        void* nb[2] = {nullptr, nullptr};
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMallocAsync(&nb[i], (size_t)cap * bps, st);
        if (e == cudaSuccess && s->held > 0)
            e = cudaMemcpyAsync(nb[0], s->d_buf[s->cur], (size_t)s->held * bps, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            for (int i = 0; i < 2; ++i)
                if (nb[i]) cudaFreeAsync(nb[i], st);
            return from_cuda(e);
        }
        for (int i = 0; i < 2; ++i)
            if (s->d_buf[i]) cudaFreeAsync(s->d_buf[i], st);
        s->d_buf[0] = nb[0];
        s->d_buf[1] = nb[1];
        s->cur = 0;
        s->cap = cap;
    }
    char* buf = static_cast<char*>(s->d_buf[s->cur]);
    if (n_samples > 0)
        e = cudaMemcpyAsync(buf + (size_t)s->held * bps, d_chunk, (size_t)n_samples * bps,
                            cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
    s->held += n_samples;
    s->pushed = total;
    s->last = st;
    s->has_last = true;
    if (fresh > 0) {
        // The live buffer always starts at the first row of spectrum s->emitted.
        e = plan->entry.launch(plan->view, buf, static_cast<float2*>(d_out), fresh, st);
        if (e != cudaSuccess) return from_cuda(e);
        s->emitted = complete;
        const int64_t drop = s->emitted * N - s->base;
        const int64_t keep = s->held - drop;
        char* other = static_cast<char*>(s->d_buf[s->cur ^ 1]);
        if (keep > 0)
            e = cudaMemcpyAsync(other, buf + (size_t)drop * bps, (size_t)keep * bps, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return from_cuda(e);
        s->cur ^= 1;
        s->base += drop;
        s->held = keep;
    }
    if (n_spectra_out) *n_spectra_out = fresh;
    return PPF_OK;
}

// Saved stream state: this header, then the held samples in the plan's
// storage type.  The held samples are the stream's samples from the first row
// of spectrum `emitted` on (held = pushed - emitted*N < T*N).
namespace {
struct StreamStateHeader {
    char magic[4];  // "PPFS"
    int32_t version;
    int32_t N, T, dtype, pad;
    int64_t pushed, emitted, held;
};
constexpr int32_t kStreamStateVersion = 1;
}  // namespace

ppf_status_t ppf_stream_state_bytes(ppf_stream_t s, size_t* bytes)
{
    if (!s || !bytes) return PPF_ERR_INVALID_ARG;
    *bytes = sizeof(StreamStateHeader) + (size_t)s->held * sample_bytes(s->plan->dtype);
    return PPF_OK;
}

ppf_status_t ppf_stream_save(ppf_stream_t s, void* h_state, size_t capacity_bytes)
{
    if (!s || !h_state) return PPF_ERR_INVALID_ARG;
    const int bps = sample_bytes(s->plan->dtype);
    const size_t need = sizeof(StreamStateHeader) + (size_t)s->held * bps;
    if (capacity_bytes < need) return PPF_ERR_INVALID_ARG;
    if (pending_cuda_error()) return PPF_ERR_CUDA;
    // the pushes enqueued so far must have written the history (every push
    // is ordered after the one before, so the last push's stream covers all)
    cudaError_t e = s->has_last ? cudaStreamSynchronize(s->last) : cudaSuccess;
    if (e != cudaSuccess) return from_cuda(e);
    StreamStateHeader hd{};
    std::memcpy(hd.magic, "PPFS", 4);
    hd.version = kStreamStateVersion;
    hd.N = s->plan->view.N;
    hd.T = s->plan->view.T;
    hd.dtype = (int32_t)s->plan->dtype;
    hd.pushed = s->pushed;
    hd.emitted = s->emitted;
    hd.held = s->held;
    std::memcpy(h_state, &hd, sizeof(hd));
    if (s->held > 0)
        e = cudaMemcpy(static_cast<char*>(h_state) + sizeof(hd), s->d_buf[s->cur], (size_t)s->held * bps,
                       cudaMemcpyDeviceToHost);
    return from_cuda(e);
}

ppf_status_t ppf_stream_restore(ppf_plan_t plan, const void* h_state, size_t bytes, ppf_stream_t* out,
                                void* stream)
{
    if (!plan || !h_state || !out) return PPF_ERR_INVALID_ARG;
    *out = nullptr;
    if (plan->view.out_f16) return PPF_ERR_UNSUPPORTED;
    if (bytes < sizeof(StreamStateHeader)) return PPF_ERR_INVALID_ARG;
    StreamStateHeader hd;
    std::memcpy(&hd, h_state, sizeof(hd));
    const int64_t N = plan->view.N, T = plan->view.T;
    const int bps = sample_bytes(plan->dtype);
    // the state must be one a stream of this plan's N, T and dtype can be in
    if (std::memcmp(hd.magic, "PPFS", 4) != 0 || hd.version != kStreamStateVersion || hd.N != N || hd.T != T ||
        hd.dtype != (int32_t)plan->dtype || hd.pushed < 0)
        return PPF_ERR_INVALID_ARG;
    const int64_t complete = hd.pushed / N - T + 1 > 0 ? hd.pushed / N - T + 1 : 0;
    if (hd.emitted != complete || hd.held != hd.pushed - hd.emitted * N || hd.held < 0 || hd.held >= T * N)
        return PPF_ERR_INVALID_ARG;
    if (bytes < sizeof(hd) + (size_t)hd.held * bps) return PPF_ERR_INVALID_ARG;
    if (pending_cuda_error()) return PPF_ERR_CUDA;
    ppf_stream_s* s = new (std::nothrow) ppf_stream_s();
    if (!s) return PPF_ERR_OUT_OF_MEMORY;
    s->plan = plan;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t cap = (T + 1) * N;
    while (cap < hd.held) cap *= 2;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMallocAsync(&s->d_buf[i], (size_t)cap * bps, st);
    if (e == cudaSuccess && hd.held > 0)
        e = cudaMemcpyAsync(s->d_buf[0], static_cast<const char*>(h_state) + sizeof(hd), (size_t)hd.held * bps,
                            cudaMemcpyHostToDevice, st);
    // the caller's buffer may be reused once this returns
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        for (int i = 0; i < 2; ++i)
            if (s->d_buf[i]) cudaFreeAsync(s->d_buf[i], st);
        cudaStreamSynchronize(st);
        delete s;
        return from_cuda(e);
    }
    s->cap = cap;
    s->cur = 0;
    s->held = hd.held;
    s->pushed = hd.pushed;
    s->emitted = hd.emitted;
    s->base = hd.emitted * N;
    s->last = st;
    s->has_last = true;
    *out = s;
    return PPF_OK;
}

ppf_status_t ppf_stream_close(ppf_stream_t s)
{
    if (!s) return PPF_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2; ++i)
        if (s->d_buf[i]) {
            cudaError_t e2 = cudaFreeAsync(s->d_buf[i], s->last);
            if (e == cudaSuccess) e = e2;
        }
    cudaError_t e2 = s->last ? cudaStreamSynchronize(s->last) : cudaDeviceSynchronize();
    if (e == cudaSuccess) e = e2;
    if (s->order_ev) cudaEventDestroy(s->order_ev);
    delete s;
    return from_cuda(e);
}

}  // extern "C"
