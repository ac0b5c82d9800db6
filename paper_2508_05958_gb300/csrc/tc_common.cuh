// Device helpers shared by the tensor-core kernels (tcgen05, sm_103a): shared-memory
// matrix descriptors, bounded mbarrier waits, bulk and tensor copies, MMA issue and
// commit, and the three-way BF16 split.
#pragma once

#include <cuda_bf16.h>

#include "htlr_internal.h"

namespace htlr {
namespace tcc {

constexpr int kSplits = 3;
// Default limit of a bounded device wait, in SM clock cycles: about 2 s at 2 GHz.  The
// kernels take their limit from the launch arguments (htlr_options.tc_wait_cycles); the
// waits of the clean-up after an abort, which must see copies and MMAs already in flight
// land, always use this one.
constexpr long long kWaitCycles = 4000000000ll;
// Limits below this many cycles poll with the non-blocking mbarrier.test_wait, so that
// they hold to within a few polls; longer ones let mbarrier.try_wait suspend the thread
// between polls.
constexpr long long kPollBelow = 1ll << 20;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture; no swizzle
    return d;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

// One poll of the phase with the given parity: true once it has completed.  `suspend`
// lets the hardware hold the thread for a while before answering (try_wait); otherwise
// the answer is immediate (test_wait).
__device__ __forceinline__ bool mbar_poll(uint64_t *b, uint32_t parity, bool suspend)
{
    uint32_t done;
    if (suspend)
        asm volatile(
            "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
            " selp.b32 %0, 1, 0, P1;\n}"
            : "=r"(done)
            : "r"(smem_u32(b)), "r"(parity)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred P1;\n mbarrier.test_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
            " selp.b32 %0, 1, 0, P1;\n}"
            : "=r"(done)
            : "r"(smem_u32(b)), "r"(parity)
            : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity; false after `limit` SM cycles, or at
// once when *abort_flag (may be null) is set by another role of the CTA.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity,
                                          long long limit = kWaitCycles,
                                          volatile int *abort_flag = nullptr)
{
    const bool suspend = limit >= kPollBelow;
    const long long t0 = clock64();
    while (true) {
        if (mbar_poll(b, parity, suspend)) return true;
        if ((abort_flag && *abort_flag) || clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 5-D tiled tensor load (TMA) into shared memory, completion on an mbarrier.  Box
// coordinates outside the tensor read zeros.
__device__ __forceinline__ void tensor_load_5d(void *dst, const void *tmap, int c0, int c1, int c2,
                                               int c3, int c4, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Split x into three BF16 terms; returns term `split` (0, 1, 2) as raw bits.
__device__ __forceinline__ uint16_t bf16_split(double x, int split)
{
    const __nv_bfloat16 a1 = __float2bfloat16_rn((float)x);
    if (split == 0) return __bfloat16_as_ushort(a1);
    const double r1 = x - (double)__bfloat162float(a1);
    const __nv_bfloat16 a2 = __float2bfloat16_rn((float)r1);
    if (split == 1) return __bfloat16_as_ushort(a2);
    const double r2 = r1 - (double)__bfloat162float(a2);
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)r2));
}

}  // namespace tcc

}  // namespace htlr
