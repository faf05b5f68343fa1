// Inline-PTX wrappers for sm_103a: mbarriers, TMA bulk copies, cluster
// barriers and distributed shared memory.  Every wait is bounded in time.
#pragma once

#include <cstdint>

namespace ppf {

// Give up a wait after this many nanoseconds of %globaltimer (2 s): the
// kernel then records PPF_ERR_TIMEOUT and returns instead of hanging.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the async proxy and the cluster.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar`; false if kWaitLimitNs passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// L2 policy: evict-first (the input stream is read exactly once).
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 1-D bulk copy global -> this CTA's shared memory, completion on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                            uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// 1-D bulk prefetch global -> L2 (no completion, no shared memory): pulls a
// ring chunk the CTA will copy later into L2 ahead of time, so that more of
// the stream is in flight than the ring holds.  src 16-byte aligned, bytes a
// multiple of 16, the whole range inside the caller's input buffer.
__device__ __forceinline__ void l2_prefetch_1d(const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------- clusters
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_arrive_release()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait_acquire()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_shared_rank(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Asynchronous store of 16 bytes into a peer CTA's shared memory (16-byte
// aligned address); completion is counted (16 bytes of complete_tx) on the
// peer's mbarrier `rbar`.  No fence is needed: the receiver observes the data
// through that mbarrier.
__device__ __forceinline__ void st_async_f4(uint32_t addr, float4 v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rbar)
                 : "memory");
}

// Arrive once on an mbarrier of a peer CTA (cluster shared-memory address),
// with release semantics at cluster scope: the shared-memory reads
// this CTA made before (ordered by a CTA barrier) happen before anything a
// peer does after observing the phase with mbar_wait_cluster_bounded.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t rbar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rbar) : "memory");
}

// Bounded wait with acquire semantics at cluster scope (pairs with mbar_arrive_cluster).
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity,
                                                          uint64_t limit_ns = kWaitLimitNs)
{
    auto try_wait = [&] {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (try_wait()) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 1;; ++i) {
        if (try_wait()) return true;
        if ((i & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// ---------------------------------------------------------------- named barriers
// CTA barriers over a subset of warps (barrier `id` in 1..15, `count` threads,
// a multiple of 32).  The non-.aligned forms count every thread's arrival on
// its own, so a warp need not be converged when it gets there.  arrive marks
// arrival without waiting (a producer); sync waits for the barrier to
// complete (a consumer); the memory accesses a thread made before arriving
// are performed before the threads that complete the wait go on.
__device__ __forceinline__ void nbar_sync(int id, int count)
{
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int count)
{
    asm volatile("barrier.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// barrier.sync over `count` threads that also returns the OR of `v` over them.
__device__ __forceinline__ bool nbar_sync_or(int id, int count, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "barrier.red.or.pred o, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// ---------------------------------------------------------------- register split
// Move registers between the warpgroups of a CTA (sm_90a and later "a"
// targets): every thread of a warpgroup executes the same instruction; `dec`
// hands registers back to the CTA's pool, `inc` waits until the pool holds
// enough.  The pool is what the CTA was launched with (threads x registers a
// thread at launch), so the counts a kernel asks for must add up to at most
// that: the host checks the launch register count before the first launch.
template <int R>
__device__ __forceinline__ void regs_inc()
{
    static_assert(R >= 24 && R <= 256 && R % 8 == 0, "register count");
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(R));
}
template <int R>
__device__ __forceinline__ void regs_dec()
{
    static_assert(R >= 24 && R <= 256 && R % 8 == 0, "register count");
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(R));
}

}  // namespace ppf
