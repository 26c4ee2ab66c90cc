// stage.cuh -- copy a volume's daughter table from global into shared memory
// with the bulk-copy engine (cp.async.bulk, completion on an mbarrier).
//
// Every wait is bounded: after kWaitLimit polls the block records
// ST_TMA_TIMEOUT in the volume's status word, waits (bounded again) for its
// own copy, and reports failure so the kernel returns without using the
// table.  No cluster is involved (a CTA is its own cluster of one).
#pragma once
#include <cstdint>
#include "geo_internal.h"

namespace geonav {

constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint32_t kChunk = 32768;   // bytes per bulk copy instruction

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
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

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Stage up to two segments (sizes multiple of 16, all addresses 16-byte
// aligned) into shared memory with one barrier.  Must be called by all threads
// of the block.  Returns false (for every thread) on timeout.
__device__ __forceinline__ bool stage_tables(void* dst0, const void* src0, uint32_t bytes0, void* dst1,
                                             const void* src1, uint32_t bytes1, uint64_t* bar,
                                             unsigned int* status) {
    if (bytes0 + bytes1 == 0) return true;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes0 + bytes1);
        for (uint32_t off = 0; off < bytes0; off += kChunk) {
            const uint32_t len = (bytes0 - off) < kChunk ? (bytes0 - off) : kChunk;
            bulk_g2s(static_cast<char*>(dst0) + off, static_cast<const char*>(src0) + off, len, bar);
        }
        for (uint32_t off = 0; off < bytes1; off += kChunk) {
            const uint32_t len = (bytes1 - off) < kChunk ? (bytes1 - off) : kChunk;
            bulk_g2s(static_cast<char*>(dst1) + off, static_cast<const char*>(src1) + off, len, bar);
        }
    }
    uint32_t it = 0;
    bool done = false;
    while (!(done = mbar_try_wait(bar, 0)) && ++it < kWaitLimit) {
    }
    if (!done) {
        atomicOr(status, ST_TMA_TIMEOUT);
        // do not leave while the copy may still write this block's memory
        for (uint32_t k = 0; k < kWaitLimit && !mbar_try_wait(bar, 0); ++k) {
        }
    }
    return __syncthreads_and(done ? 1 : 0) != 0;
}

__device__ __forceinline__ bool stage_table(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                            unsigned int* status) {
    return stage_tables(dst, src, bytes, nullptr, nullptr, 0, bar, status);
}

}  // namespace geonav
