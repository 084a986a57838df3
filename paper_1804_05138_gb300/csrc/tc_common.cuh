// tc_common.cuh -- inline-PTX building blocks shared by the tcgen05 kernels (mbarriers, TMA,
// UMMA descriptors, tensor-memory MMA, TF32 rounding) and the host-side tensor-map encoder.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace rq {
namespace tc {

constexpr unsigned long long kTcWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned cnt)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps until the phase completes or about
// kTcSuspendNs pass, so a waiting warp costs no issue slots.
constexpr unsigned kTcSuspendNs = 100000;
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(kTcSuspendNs)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of parity `parity`; gives up after kTcWaitNs, or as soon as another
// role of the block has recorded a failure in *fail (when fail is not null).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, const volatile int* fail)
{
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_test(b, parity)) return true;
        if (fail != nullptr && *fail) return false;
        if (globaltimer_ns() - t0 > kTcWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}
// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t umma_desc(const void* base)
{
    const uint64_t addr = su32(base);
    return ((addr >> 4) & 0x3FFFull) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}
// Instruction descriptor: D FP32, A and B TF32, both K-major, N >> 3, M >> 4.
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// Instruction descriptor: D FP32, A and B BF16, both K-major, N >> 3, M >> 4.
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// A (M x K BF16, lane m = row m, two consecutive K elements per 32-bit column, the lower index in
// the low half) in tensor memory, B in shared memory; K = 16 per instruction.
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(
            tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
// A (M x K, lane m = row m, one TF32 element per 32-bit column) in tensor memory, B in shared memory.
__device__ __forceinline__ void mma_tf32_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(
            tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
// A (M x K) and B (N x K) both in shared memory (descriptors), TF32, K = 8 per instruction.
__device__ __forceinline__ void mma_tf32_ss(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
// TF32 rounding of a finite FP32 value to its top 19 bits (10 explicit mantissa bits), ties away
// from zero, by integer arithmetic on the bit pattern: adding half a TF32 ulp (bit 12) carries
// into the kept bits (and the exponent) exactly when the dropped 13 bits are at least half.
__device__ __forceinline__ float tf32_rn(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Bulk tensor store (shared -> global) of one 2-D box; completion tracked by bulk groups.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x), "r"(y),
                 "r"(su32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until all committed bulk stores have finished reading their shared-memory source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// wait until all committed bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, unsigned cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst_smem)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, unsigned cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

}  // namespace tc

// 2-D FP32 tensor map: `inner` contiguous elements per line, `outer` lines ld elements apart, box
// box_inner x box_outer, 128-byte swizzle (box_inner = 32) or none.  False if the driver's
// encoder is unavailable or rejects the map.
bool tc_encode_2d(CUtensorMap* map, const float* base, long long inner, long long outer, long long ld, int box_inner,
                  int box_outer, bool swizzle128);
// The same for FP32 (elem_bytes 4) or BF16 (elem_bytes 2) elements; ld in elements.
bool tc_encode_2d_typed(CUtensorMap* map, const void* base, int elem_bytes, long long inner, long long outer,
                        long long ld, int box_inner, int box_outer, bool swizzle128);
bool tc_encoder_available();

}  // namespace rq
