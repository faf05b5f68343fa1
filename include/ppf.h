/*
 * ppf.h -- C ABI of the GB300-native polyphase filter bank (PPF).
 *
 * Method: Adamek, Novotny, Armour, "The Implementation of a Real-Time
 * Polyphase Filter" (arXiv 1411.3656).  A PPF applies a T-tap FIR filter
 * (Section 2, Eq. 1; Algorithm 1) to each of N frequency channels of a
 * complex sample stream and then takes an N-point DFT of every filtered
 * spectrum (Section 2: the channels are the DFT bins; Section 3: a standard
 * forward FFT).  Concretely, for output spectrum s, channel c and bin k:
 *
 *     y[s][c] = sum_{t=0}^{T-1} h[t*N + c] * x[(s+t)*N + c]
 *     Y[s][k] = sum_{c=0}^{N-1} y[s][c] * exp(-2*pi*i*k*c/N)
 *
 * h[c] weights the oldest of the T input rows a spectrum reads and
 * h[(T-1)*N + c] the newest; this is Eq. 1 with b_i = h[(T-1-i)*N + c].  The
 * DFT is forward, unnormalised, in natural bin order (k = 0..N-1).
 *
 * Everything runs in hand-written sm_103a CUDA kernels.  There is no CPU
 * fallback: without a usable GPU every compute entry point returns
 * PPF_ERR_CUDA.
 *
 * Conventions shared by all entry points:
 *   - Sizes: N is a power of two, 4 <= N <= 4096; 1 <= T <= 64, for every
 *     input type.  Anything else is PPF_ERR_UNSUPPORTED.
 *   - Samples: PPF_IN_C32 = float2 (I, Q) 8 bytes; PPF_IN_C16 = two IEEE
 *     half values (I, Q) 4 bytes; PPF_IN_CI8 = two signed 8-bit integers
 *     (I, Q) 2 bytes, used unscaled.  Output is float2 (complex64), or FP16
 *     (I, Q) pairs with PPF_FLAG_OUT_F16.
 *   - Arithmetic: FIR and FFT accumulate in FP32.  h is FP32 for C32 input
 *     and is rounded to FP16 for C16 / CI8 input.
 *   - Device buffers belong to the caller, must be 16-byte aligned
 *     (PPF_ERR_MISALIGNED otherwise) and must not overlap.
 *   - Work is enqueued on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream) and the call returns without
 *     waiting.  Argument errors are reported synchronously and enqueue
 *     nothing.  Errors of earlier asynchronous work surface as PPF_ERR_CUDA.
 *   - A plan is immutable after creation and may be used from several host
 *     threads and CUDA streams at once (its kernels keep no state in device
 *     memory between launches).  A stream object is not thread-safe.
 */
#ifndef PPF_H_
#define PPF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ppf_plan_s* ppf_plan_t;
typedef struct ppf_stream_s* ppf_stream_t;

typedef enum {
    PPF_OK = 0,
    PPF_ERR_INVALID_ARG = 1,   /* null pointer, negative count, too-small capacity */
    PPF_ERR_UNSUPPORTED = 2,   /* N, T or dtype outside the supported set */
    PPF_ERR_MISALIGNED = 3,    /* device buffer not 16-byte aligned, or overlapping */
    PPF_ERR_OUT_OF_MEMORY = 4, /* a device or host allocation failed */
    PPF_ERR_CUDA = 5,          /* a CUDA runtime error (this call or earlier async work) */
    PPF_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    PPF_ERR_BUSY = 7           /* the object is in use (e.g. close with pending work) */
} ppf_status_t;

typedef enum {
    PPF_IN_C32 = 0,            /* float2 (I, Q) */
    PPF_IN_C16 = 1,            /* half2 (I, Q) */
    PPF_IN_CI8 = 2             /* int8 (I, Q) */
} ppf_dtype_t;

/* Plan flags. */
#define PPF_FLAG_NONE 0u
#define PPF_FLAG_FIR_ONLY 1u   /* write the FIR output y instead of Y (the first of the paper's two
                                  passes, Section 3; a FIR-only kernel for complex64 N >= 128,
                                  T in {4, 8, 16, 32}, else the general kernel's FIR-only form) */
#define PPF_FLAG_GENERIC 2u    /* always use the general kernel (runtime T, any size) */
/* Output bins as FP16 (I, Q) pairs (4 bytes per bin, rounded to nearest)
 * instead of complex64: a quarter less HBM traffic for complex64 input, 40%
 * less for int8 I/Q.  Bins beyond +-65504 become +-inf; the arithmetic stays
 * FP32.  Supported by ppf_execute and ppf_batch_*; ppf_execute_host,
 * ppf_stream_open and ppf_server_admit return PPF_ERR_UNSUPPORTED for such a
 * plan, and so does ppf_plan_create together with PPF_FLAG_FIR_ONLY. */
#define PPF_FLAG_OUT_F16 4u
/* Force specialised kernel variant i (0-based) of ppf_variant_count(N, T, dtype)
 * instead of the tuned default; used by the autotuner. */
#define PPF_FLAG_VARIANT(i) ((((unsigned)(i) + 1u) & 0xFFu) << 8)

/*
 * ppf_plan_create -- build a plan for N channels and T taps (Section 2, Eq. 1).
 *   out      [out] receives the plan handle (owned by the caller; release it
 *            with ppf_plan_destroy).
 *   N, T     channels (power of two, 4..4096) and taps (1..64).
 *   h_host   host array of N*T float coefficients, h[t*N + c] = tap t of
 *            channel c.  Copied to the device; the caller keeps ownership.
 *   in_dtype storage type of the input samples.
 *   flags    PPF_FLAG_* bits.
 * Allocates device memory for the coefficients and the FFT twiddle factors
 * (computed in FP64 on the host, stored in FP32).  Synchronises the current
 * device.  Returns PPF_ERR_UNSUPPORTED for unsupported sizes,
 * PPF_ERR_INVALID_ARG for null pointers, PPF_ERR_OUT_OF_MEMORY or
 * PPF_ERR_CUDA on device failure (nothing is leaked).
 */
ppf_status_t ppf_plan_create(ppf_plan_t* out, int N, int T, const float* h_host,
                             ppf_dtype_t in_dtype, unsigned flags);

/* Release a plan's device memory.  The caller must ensure no work using the
 * plan is still running.  A NULL plan is PPF_ERR_INVALID_ARG. */
ppf_status_t ppf_plan_destroy(ppf_plan_t plan);

/*
 * ppf_execute -- the whole PPF on a device-resident batch (streaming mode,
 * the paper's M_c, Section 3).
 *   d_in       device input, (n_spectra + T - 1) * N samples of the plan's
 *              dtype, one contiguous stream (sample n = r*N + c is row r,
 *              channel c).  Read only.
 *   d_out      device output, n_spectra * N bins, row-major [s][k]: complex64,
 *              or FP16 (I, Q) pairs for a plan made with PPF_FLAG_OUT_F16.
 *   n_spectra  number of output spectra S >= 0 (0 enqueues nothing).
 *   stream     cudaStream_t as void*.
 * One launch of the fused FIR+FFT kernel: each input sample is read from
 * device memory once and filtered spectra never leave the chip.
 */
ppf_status_t ppf_execute(ppf_plan_t plan, const void* d_in, void* d_out,
                         int64_t n_spectra, void* stream);

/*
 * ppf_execute_host -- the whole PPF on host buffers (the paper's single mode,
 * M_b, Section 3, Table 2): copies host->device, runs the fused kernel and
 * copies the spectra back, in slices of about 16 Mi samples through a
 * three-stage pipeline (upload, kernel, download on their own streams, three
 * staging slots), so the upload of one slice, the kernel of another and the
 * download of a third run at the same time.  Blocks until the result is in
 * h_out.
 *   h_in   host input, (n_spectra + T - 1) * N samples (pinned memory gives
 *          full link bandwidth; pageable memory works but is slower).
 *   h_out  host output, n_spectra * N complex64.
 * Device staging buffers are allocated on the first call and cached in the
 * plan (released by ppf_plan_destroy); calls on one plan are serialised.
 */
ppf_status_t ppf_execute_host(ppf_plan_t plan, const void* h_in, void* h_out,
                              int64_t n_spectra, void* stream);

/*
 * ppf_stream_open -- a continuous stream on top of a plan.  The stream owns a
 * device buffer holding the FIR history: the last (T-1)*N samples plus the
 * fewer-than-N samples of an incomplete row (Section 2: each output needs the
 * newest sample and T-1 past samples of its channel).
 */
ppf_status_t ppf_stream_open(ppf_plan_t plan, ppf_stream_t* out);

/*
 * ppf_stream_push -- feed n_samples new samples (device pointer, plan dtype,
 * any count, not necessarily a multiple of N) and emit every spectrum whose
 * window is now complete.  After pushes totalling L samples the stream has
 * emitted max(0, floor(L/N) - T + 1) spectra in total, identical to
 * ppf_execute on the concatenation of all pushes.
 *   d_out                 device output, row-major complex64 spectra.
 *   out_capacity_spectra  rows available in d_out; if fewer than the spectra
 *                         this push completes, PPF_ERR_INVALID_ARG and the
 *                         stream is unchanged.
 *   n_spectra_out [out]   spectra written by this push.
 * Ordered on `stream`; the history update is enqueued on the same stream.
 * Successive pushes of one stream object may use different CUDA streams: a
 * push made on another stream than the previous one first makes its stream
 * wait (an event) for the work the previous push enqueued.
 */
ppf_status_t ppf_stream_push(ppf_stream_t s, const void* d_chunk, int64_t n_samples,
                             void* d_out, int64_t out_capacity_spectra,
                             int64_t* n_spectra_out, void* stream);

/*
 * Checkpoint and resume of a stream.  A stream's whole state is its position
 * (samples pushed, spectra emitted) and the samples it holds: the T-1 rows
 * the next spectrum shares with the last one emitted plus the incomplete
 * newest row (Section 2: every output needs the newest sample and T-1 past
 * samples of its channel) -- fewer than T*N samples.
 *
 * ppf_stream_state_bytes -- bytes ppf_stream_save writes for the stream now:
 *   a 48-byte header (magic "PPFS", version, N, T, dtype, pushed, emitted,
 *   held) followed by the held samples in the plan's storage type.
 * ppf_stream_save -- wait for the stream's pushes, then write its state into
 *   the caller's host buffer h_state (capacity_bytes; PPF_ERR_INVALID_ARG if
 *   smaller than ppf_stream_state_bytes).  The stream itself is unchanged
 *   and may go on.
 * ppf_stream_restore -- open a new stream on `plan` (same N, T and dtype as
 *   the saved stream, else PPF_ERR_INVALID_ARG; any coefficients) from a
 *   saved state; the history is uploaded on `stream` and the call returns
 *   once it is on the device.  Pushes to the new stream continue exactly
 *   where the saved one stopped: the spectra are those of an uninterrupted
 *   stream.  A truncated or inconsistent state is PPF_ERR_INVALID_ARG.  The
 *   caller owns h_state; close the new stream with ppf_stream_close.
 */
ppf_status_t ppf_stream_state_bytes(ppf_stream_t s, size_t* bytes);
ppf_status_t ppf_stream_save(ppf_stream_t s, void* h_state, size_t capacity_bytes);
ppf_status_t ppf_stream_restore(ppf_plan_t plan, const void* h_state, size_t bytes, ppf_stream_t* out,
                                void* stream);

/*
 * ppf_execute_noalloc -- the whole PPF with no plan and no device allocation.
 * The paper has no counterpart; this is for callers that cannot allocate
 * device memory when they need a filter bank: plug-ins whose host framework
 * owns all device memory and forbids cudaMalloc/cudaFree, and real-time
 * threads that must not block on the allocator (cudaMalloc and cudaFree can
 * synchronise the whole device).
 *   N, T, dtype  as for ppf_plan_create; N at most 4096 (the scratch limit:
 *                larger N returns PPF_ERR_UNSUPPORTED).
 *   d_h          device array of N*T float coefficients, h[t*N + c] (FP32 for
 *                every input type).  Read only.
 *   d_in, d_out, n_spectra, stream  as for ppf_execute.  d_h must not overlap
 *                d_out either (PPF_ERR_MISALIGNED).
 * Runs the general fused kernel.  Its FFT twiddle table is scratch kept in one
 * library-wide static device array of 4096 complex values (32 KiB per GPU
 * that loads the library, held until exit), rewritten by every call on the
 * call's stream.  Calls that overlap on the GPU (different streams, or the
 * same stream from several threads without ordering) share that array and
 * race.  The first call on each device runs a one-time set-up (symbol
 * address, kernel attributes); make that first call before any stream capture
 * begins.  A set-up that fails returns PPF_ERR_CUDA and is tried again by the
 * next call; only a successful one is kept.  Allocates nothing, frees
 * nothing, calls no allocating library.
 */
ppf_status_t ppf_execute_noalloc(int N, int T, ppf_dtype_t dtype, const float* d_h, const void* d_in,
                                 void* d_out, int64_t n_spectra, void* stream);

/*
 * Batches: many independent streams (each with its own plan, so its own N, T,
 * dtype and coefficients) in as few launches as possible.  This is the
 * method's data-parallel form over streams (Section 3 processes one stream;
 * independent streams simply run side by side).  Every complex64 job whose
 * (N, T) has a tile shape in the mixed-shape kernel (128 <= N <= 2048 and
 * N*T <= 16384, complex64 output, the plan's tuned default) joins ONE
 * persistent launch over a device work list of (job, spectrum band) items of
 * any N and T and about equal measured cost, which the CTAs take largest
 * first, each CTA asking for the next item when it has finished one.  Other
 * jobs whose plans use the same specialised kernel share one persistent
 * launch over their work list; jobs on the general kernel launch one by one.
 */
typedef struct ppf_batch_s* ppf_batch_t;

typedef struct {
    ppf_plan_t plan;     /* the job's plan (not owned; must outlive the batch) */
    const void* d_in;    /* device input, (n_spectra + T - 1) * N samples, 16-byte aligned */
    void* d_out;         /* device output, n_spectra * N bins (complex64, or FP16 pairs with
                            PPF_FLAG_OUT_F16), 16-byte aligned */
    int64_t n_spectra;   /* spectra of this job, >= 0 */
} ppf_job_t;

#define PPF_BATCH_GRAPH 1u   /* capture the launches into a CUDA graph on the first execute, replay after */
#define PPF_BATCH_PER_KERNEL 2u  /* no mixed-shape launch: one persistent launch per specialised kernel */

/*
 * ppf_batch_create -- group `jobs` by kernel, split them into spectrum bands
 * and upload the work lists (device memory owned by the batch).  The jobs'
 * pointers are fixed for the batch's lifetime; their contents may change
 * between executions.  Synchronises the device.  Errors: PPF_ERR_INVALID_ARG
 * (null, negative count, bad job), PPF_ERR_MISALIGNED, PPF_ERR_OUT_OF_MEMORY,
 * PPF_ERR_CUDA.
 */
ppf_status_t ppf_batch_create(ppf_batch_t* out, const ppf_job_t* jobs, int n_jobs, unsigned flags);

/* Enqueue every job of the batch on `stream` (cudaStream_t as void*), as a
 * CUDA graph launch when the batch was created with PPF_BATCH_GRAPH.  An
 * execution first zeroes the batch's device item counter: two executions of
 * one batch must not overlap on the GPU (order them on one stream). */
ppf_status_t ppf_batch_execute(ppf_batch_t batch, void* stream);

/* Kernel launches one execution enqueues (1 for a captured graph counts its
 * kernels), or -1 for a NULL batch. */
int ppf_batch_launches(ppf_batch_t batch);

/* Release the batch's device memory and graph.  Synchronises the device. */
ppf_status_t ppf_batch_destroy(ppf_batch_t batch);

/*
 * Serving: many continuous streams (each a stream of Section 3's real-time
 * workload, with its own plan) share the GPU.  Streams are admitted while
 * device memory allows; chunks are queued as they arrive and each tick runs
 * everything queued so far as one set of launches (continuous batching):
 * one batched copy of the new chunks behind each stream's FIR history, one
 * persistent PPF launch per specialised kernel, one batched history carry.
 * Results are identical to ppf_stream_push on each stream alone.  A server is
 * not thread-safe; all ticks of a server must be ordered on one CUDA stream.
 */
typedef struct ppf_server_s* ppf_server_t;

/* max_streams slots; memory_budget_bytes caps the device memory streams may
 * reserve (admission also needs that much free device memory). */
ppf_status_t ppf_server_create(ppf_server_t* out, int max_streams, size_t memory_budget_bytes);

/*
 * ppf_server_admit -- reserve a slot for a stream with `plan` whose chunks hold
 * at most max_chunk_samples samples: two device buffers of
 * 8*T*N + 4*max_chunk_samples + 2*N samples (history and boundary regions
 * for up to four chunks queued between ticks).
 * *slot_out receives the slot.  PPF_ERR_OUT_OF_MEMORY when the budget or the
 * free device memory is exhausted, PPF_ERR_BUSY when every slot is taken.
 */
ppf_status_t ppf_server_admit(ppf_server_t s, ppf_plan_t plan, int64_t max_chunk_samples, int* slot_out);

/* Free a slot (no chunk may be queued: PPF_ERR_BUSY).  Synchronises the device. */
ppf_status_t ppf_server_release(ppf_server_t s, int slot);

/*
 * ppf_server_submit -- queue n_samples (<= max_chunk_samples) new samples of
 * the slot's stream at d_chunk (device, read during the next tick; keep it
 * valid until the tick's work completes).  The spectra this chunk completes
 * are written to d_out (capacity out_capacity_spectra rows, 16-byte aligned)
 * by the next tick.  Spectra whose windows lie inside the chunk are read from
 * d_chunk in place when it is 16-byte aligned at their first row.
 * PPF_ERR_INVALID_ARG if the capacity is too small, PPF_ERR_BUSY if four
 * chunks are already queued for the slot (tick first).
 */
ppf_status_t ppf_server_submit(ppf_server_t s, int slot, const void* d_chunk, int64_t n_samples, void* d_out,
                               int64_t out_capacity_spectra);

/* Submit n chunks at once (arrays of n entries, meanings as in
 * ppf_server_submit); statuses[i] (may be NULL) gets each one's status.
 * Returns PPF_OK when all were queued, else PPF_ERR_BUSY (see statuses). */
ppf_status_t ppf_server_submit_many(ppf_server_t s, int n, const int* slots, const void* const* chunks,
                                    const int64_t* n_samples, void* const* outs, const int64_t* caps, int* statuses);

/* Run one tick on `stream`: every queued chunk of every slot.  *n_done gets the
 * number of chunks processed (may be NULL).  Returns after enqueuing. */
ppf_status_t ppf_server_tick(ppf_server_t s, void* stream, int* n_done);

/* Samples submitted and spectra produced (through the last tick) of a slot. */
ppf_status_t ppf_server_position(ppf_server_t s, int slot, int64_t* samples_in, int64_t* spectra_out);

/* Device bytes reserved, admitted streams, launches of the last tick (any may be NULL). */
ppf_status_t ppf_server_info(ppf_server_t s, size_t* reserved_bytes, int* streams, int* last_tick_launches);

/* Ticks of the server that ran as a replay of its captured CUDA graph (the
 * gather copy, the mixed-shape kernel, one work-list launch per other kernel
 * group and the carry copy, all reading their tables from a fixed device
 * area); the graph is captured on the first tick after an admit or release.
 * A stream on the general kernel, or a tick whose tables exceed the capacity
 * planned from the admitted streams, runs as direct launches instead.
 * -1 for a NULL server. */
int64_t ppf_server_graph_ticks(ppf_server_t s);

/* Release every slot and the staging buffers.  Synchronises the device. */
ppf_status_t ppf_server_destroy(ppf_server_t s);

/* Total samples pushed and spectra emitted so far (either pointer may be NULL). */
ppf_status_t ppf_stream_position(ppf_stream_t s, int64_t* samples_in, int64_t* spectra_out);

/* Release the stream's device history.  Synchronises the stream's last CUDA
 * stream first, so no pushed work is pending when the memory is freed. */
ppf_status_t ppf_stream_close(ppf_stream_t s);

/* Static, human-readable name of a status code. */
const char* ppf_status_string(ppf_status_t status);

/* Which kernel ppf_execute launches for this plan, as a static string (e.g.
 * "fused_ring" or "generic"); NULL for a NULL plan.  For tests and reports. */
const char* ppf_plan_kernel_name(ppf_plan_t plan);

/*
 * ppf_variant_count -- number of compiled variants of the specialised kernels
 * (thread count, spectra per block, ring depth, cluster size) for (N, T,
 * dtype); 0 when only the general kernel covers the size.  Pure host query.
 * ppf_variant_name -- static description of variant i, NULL if out of range.
 * These are the tile shapes the autotuner times on the device; the fastest
 * becomes the default the library picks.
 */
int ppf_variant_count(int N, int T, ppf_dtype_t dtype);
const char* ppf_variant_name(int N, int T, ppf_dtype_t dtype, int i);

/* Kernel launches this library has issued since load (for reports). */
int64_t ppf_launch_count(void);

/*
 * ppf_check_timeout -- failure-detection self-check (no paper counterpart).
 * One warp on the device waits on an mbarrier that nothing completes, through
 * the same bounded wait every PPF kernel uses for its copies and exchanges,
 * with a limit of limit_us microseconds (1..1000000) instead of the kernels'
 * 2 s; the wait gives up and raises the mapped error word.  Synchronises
 * `stream` (cudaStream_t as void*).  Returns PPF_ERR_TIMEOUT when the wait ran
 * out and was reported (the expected result), PPF_OK if it was not reported,
 * PPF_ERR_INVALID_ARG for a limit out of range, PPF_ERR_CUDA on a CUDA error.
 * The device stays usable afterwards.
 */
ppf_status_t ppf_check_timeout(unsigned limit_us, void* stream);

/*
 * ppf_fma_peak -- FP32 throughput probe for the roofline of FMA-bound tiles
 * (no paper counterpart; measurement infrastructure).  Enqueues on `stream`
 * (cudaStream_t as void*) one launch of `blocks` (1..65535) CTAs of 512
 * threads, each thread running 8 independent chains of `iters` (1..2^24)
 * packed FP32 FMAs (fma.rn.f32x2), and stores in *lane_fmas the number of
 * scalar FMA lanes the launch executes; the caller times the launch (CUDA
 * events on the same stream) and divides.  Reads and writes no memory.
 * Errors: PPF_ERR_INVALID_ARG, PPF_ERR_CUDA (launch failure).
 */
ppf_status_t ppf_fma_peak(int blocks, int iters, void* stream, double* lane_fmas);

/*
 * ppf_check_violations -- out-of-bounds accesses counted by the checked
 * build of this library (compiled with -DPPF_CHECKED: every instrumented
 * shared-memory and global access of the kernels first tests its index
 * against its buffer, counts a violation and skips the access instead of
 * making it).  Synchronises the device, returns the count since the last
 * reset (reset != 0 clears it), -1 in the normal build (no checks compiled),
 * -2 if the device could not be read.  The paper has no counterpart: this is
 * test infrastructure standing in for a memory checker.
 */
int64_t ppf_check_violations(int reset);

/* Window of the prototype low-pass filter (Section 2). */
typedef enum {
    PPF_WINDOW_HAMMING = 0,    /* 0.54 - 0.46 cos(2 pi n / (L-1)) */
    PPF_WINDOW_KAISER = 1      /* I0(beta sqrt(1 - (2n/(L-1) - 1)^2)) / I0(beta) */
} ppf_window_t;

/*
 * ppf_design_coeffs -- windowed-sinc prototype filter for an N-channel,
 * T-tap bank (Section 2: a truncated sinc shaped by a window; the paper names
 * a Kaiser window and gives no parameter, so beta is the caller's).  Host
 * only, no device work; needs no GPU.
 *   N, T      channels (>= 1) and taps per channel (>= 1); L = N*T.
 *   window    PPF_WINDOW_HAMMING or PPF_WINDOW_KAISER.
 *   beta      Kaiser shape parameter (>= 0; ignored for Hamming).
 *   h_out     caller-owned host array of N*T floats, written as
 *             h[n] = sinc((n - (L-1)/2) / N) * w[n], sinc(x) = sin(pi x)/(pi x),
 *             computed in FP64 and rounded to FP32; no normalisation.  The
 *             layout is the one ppf_plan_create takes (h[t*N + c], t = n / N).
 * I0 is evaluated by its power series.  Returns PPF_ERR_INVALID_ARG for a
 * NULL h_out, N < 1, T < 1, an unknown window or a negative or non-finite
 * beta.
 */
ppf_status_t ppf_design_coeffs(int N, int T, ppf_window_t window, double beta, float* h_out);

#ifdef __cplusplus
}
#endif

#endif /* PPF_H_ */
