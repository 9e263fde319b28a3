// Bounded grid-wide barrier for cooperative launches, on a monotonically increasing arrival counter.
//
// Device state: two 32-bit words on separate 128-byte lines, zeroed once at allocation:
//   count  arrivals of all launches so far (never reset; wraps modulo 2^32)
//   base   the value of count when the current launch started (written by the previous launch)
// A launch that passes nbar barriers with G CTAs reads base at entry; its i-th barrier (i = 1 .. nbar)
// completes when count reaches base + i G. Arrival is a fire-and-forget release add; waiting is an acquire
// poll of count alone, so no CTA ever resets shared state while others poll it. Every CTA arrives at every
// barrier even after a wait of its own gave up (ST_TIMEOUT), so count always ends at base + nbar G, and the
// launch's last step (gb_finish, CTA 0 after its last barrier) stores that as the next launch's base.
#pragma once

#include "eda_internal.cuh"

namespace eda {

struct GridBarWords {
    unsigned* count;   // 128-byte aligned
    unsigned* base;    // count + 32 (its own line)
    long long spin;    // polls before a wait gives up
};

__device__ __forceinline__ unsigned gb_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void gb_red_release(unsigned* p) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

// The launch's base (every thread may call it; stable for the whole launch).
__device__ __forceinline__ unsigned gb_base(const GridBarWords& w) { return *reinterpret_cast<volatile unsigned*>(w.base); }

// Barrier number i (1-based) of the launch. Returns false when this CTA's wait gave up.
__device__ __forceinline__ bool gb_sync(const GridBarWords& w, unsigned base, unsigned i, int* status) {
    __shared__ int gb_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        gb_red_release(w.count);
        const unsigned target = base + i * gridDim.x;
        long long it = 0;
        while ((int)(gb_ld_acquire(w.count) - target) < 0) {
            if (++it > w.spin) {
                atomicOr(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
        gb_ok = ok;
    }
    __syncthreads();
    return gb_ok != 0;
}

// After the launch's last barrier (nbar in all): CTA 0 publishes the next launch's base.
__device__ __forceinline__ void gb_finish(const GridBarWords& w, unsigned base, unsigned nbar) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<volatile unsigned*>(w.base) = base + nbar * gridDim.x;
}

}  // namespace eda
