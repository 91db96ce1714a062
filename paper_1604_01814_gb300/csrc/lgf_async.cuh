// Bulk asynchronous copies (the TMA engine's 1-D form, cp.async.bulk) into
// shared memory, completed on an mbarrier, with a bounded wait.
//
// Every wait has a time limit.  When it runs out the waiting thread sets a
// bit of the context's device error word (the host reports LGF_ETIMEOUT, see
// lgf_device_status), waits once more with the same limit so that no copy is
// left writing into the CTA's shared memory, and the caller returns without
// using the staged data.  Nothing traps, so the context stays usable.
#pragma once
#include <cstdint>

namespace lgf {
namespace async {

constexpr long long kWaitCycles = 2000000000LL;   // about one second at the maximum SM clock
constexpr int kErrWait = 1;                       // error-word bit: a bulk-copy wait ran out

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One thread: an mbarrier expecting one arrival, made visible to the async proxy.
__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The single arrival, announcing `bytes` of copies to complete before the
// phase ends.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst_smem)),
                 "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` for at most `limit` SM cycles; on timeout
// set `code` in *err, wait once more with the same limit, and return false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, long long limit = kWaitCycles,
                                          int code = kErrWait)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > limit) {
            if (err) atomicOr(err, code);
            const long long t1 = clock64();
            while (!mbar_try(bar, parity))
                if (clock64() - t1 > limit) break;
            return false;
        }
    return true;
}

}  // namespace async
}  // namespace lgf
