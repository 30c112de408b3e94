// lbm_mbar.cuh -- PTX wrappers for transaction-counted mbarriers and bulk
// asynchronous copies (sm_90 and later), with the bounded wait every kernel of
// this library uses: a wait gives up after a fixed number of try_wait rounds and
// reports failure instead of spinning for ever.
#pragma once

#include <cstdint>

namespace lbm {

// ---- PTX wrappers (sm_90+ bulk asynchronous copies and transaction mbarriers)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// Value written to the status word when a copy would not be 16-byte aligned; the
// copy is then skipped (its wait runs out and the block leaves instead of faulting).
constexpr int kStatusMisaligned = 100;

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                          int* status) {
    if (((dst | bytes) & 15u) != 0u || (reinterpret_cast<uintptr_t>(src) & 15u) != 0u || bytes == 0u) {
        atomicExch(status, kStatusMisaligned);
        return;
    }
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
constexpr int kWaitLimit = 1 << 21;   // try_wait rounds before a wait is declared lost
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kWaitLimit) {
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace lbm
