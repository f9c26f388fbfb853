// Inline-PTX wrappers shared by the tensor-core kernels (glynn_tc.cu,
// mlp_tc.cu): mbarriers, TMA tile loads into shared memory, and the 5th-
// generation tensor-core instructions (tcgen05) with their shared-memory and
// instruction descriptors.  Internal to the library.
//
// Waits are bounded: mbar_wait gives up after `max_polls` unsuccessful
// try_wait polls and returns false, so a kernel whose producer or consumer has
// stopped records an error and returns instead of spinning.  A kernel that
// gives up must still let its own asynchronous work finish before it exits
// (TMA loads write its shared memory, MMAs its tensor memory): it waits, with
// kCleanupPolls, for the loads it issued and for a final tcgen05.commit.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace pcv {
namespace tcx {

// Clean-up waits on work that is already in flight (a TMA load or MMA
// completes in microseconds); far beyond any legitimate latency.
constexpr long long kCleanupPolls = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the phase of parity `parity` to complete; false after max_polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_polls)
{
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < max_polls; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];\n" ::"l"(map) : "memory");
}

// Tiled TMA load of one box into shared memory, completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int u)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(u), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout written by TMA: rows of 128 B, 8-row atoms 1024 B apart.  The start
// address sits in the low bits in 16-byte units, so a descriptor plus j
// addresses the tile 16 j bytes further on.
__device__ __forceinline__ uint64_t sdesc_sw128(const void* p)
{
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr & 0x3FFFF) >> 4;                 // start address
    d |= (uint64_t)(16 >> 4) << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version of tcgen05
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major) and an
// FP32 accumulator, M = m (64 or 128), N = n (a multiple of 16, <= 256).
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n)
{
    uint32_t d = 0;
    d |= 1u << 4;                               // accumulator: FP32
    d |= 1u << 7;                               // A: BF16
    d |= 1u << 10;                              // B: BF16
    d |= (uint32_t)(n >> 3) << 17;              // N / 8
    d |= (uint32_t)(m >> 4) << 24;              // M / 16
    return d;
}

// D[tmem] (+)= A[ad] . B[bd]^T, one CTA, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` when every tcgen05 operation this thread issued so far is complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst_smem)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Issued-load bookkeeping of a ring of `slots` barriers filled in order
// 0, 1, 2, ...: after `issued` loads, wait (with the clean-up bound) for the
// last load that went to each slot.  Loads a consumer already waited for
// complete at once.
__device__ __forceinline__ bool wait_issued(uint64_t* bars, int slots, uint32_t issued)
{
    bool ok = true;
    for (int s = 0; s < slots; ++s) {
        if (issued <= (uint32_t)s) break;
        const uint32_t last = (uint32_t)s + ((issued - 1 - (uint32_t)s) / (uint32_t)slots) * (uint32_t)slots;
        ok = mbar_wait(&bars[s], (last / (uint32_t)slots) & 1u, kCleanupPolls) && ok;
    }
    return ok;
}

}  // namespace tcx
}  // namespace pcv
