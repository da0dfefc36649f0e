// lbm_bulk.cuh -- bulk asynchronous copies from global into shared memory
// (the TMA engine's non-tensor form, cp.async.bulk), completed on an
// mbarrier's transaction count, in inline PTX for sm_100-class GPUs. Every
// wait is bounded in time: a caller that gets `false` back sets a status bit
// and stops issuing work instead of spinning on.
#pragma once
#include <cstdint>

namespace tlv {

__device__ __forceinline__ unsigned cta_smem(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Barrier with one expected arrival per phase: the issuing lane's
// arrive.expect_tx, after which the phase completes when the copies' bytes
// have all landed.
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cta_smem(bar)) : "memory");
}

// Makes barrier initialisation visible to the copy engine.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies (async proxy) into the same bytes.
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cta_smem(bar)), "r"(bytes)
                 : "memory");
}

// dst (shared) and src (global) 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     cta_smem(dst)),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(cta_smem(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(cta_smem(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits (acquire) for the phase of the given parity; false once limit_ns
// has passed without it completing.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long limit_ns = 1000000000ull)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

} // namespace tlv
