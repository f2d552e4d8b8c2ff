// blink_sync.cuh -- bounded waits on shared-memory mbarriers.
//
// Every wait of the library's kernels on an asynchronous copy or MMA gives
// up after a time limit of the global timer, so a transfer that never lands
// turns into an error status the host reads instead of a hung GPU.
#pragma once

#include <cstdint>

namespace blink {

// Default limit: 1 s (the transfers and MMAs waited for take microseconds).
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Polls the barrier until its phase `parity` completes or `limit_ns` pass
// (try_wait may suspend the thread for a while on each poll).  Limit 0: one
// non-blocking test.  Returns whether the phase completed.
__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kWaitNs) {
    if (limit_ns == 0) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        return ok != 0;
    }
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 >= limit_ns) return false;
    }
}

}  // namespace blink
