// Grid-level helpers shared by the cooperative fuse-regime solvers of
// libvfunc: a bounded two-level grid barrier and warp-aggregated slot
// reservation.
#pragma once

#include <cuda/atomic>

#include "vf_internal.h"

namespace vf {

constexpr unsigned kGroup = 8;  // blocks per barrier group

using dev_atomic = cuda::atomic_ref<unsigned int, cuda::thread_scope_device>;

// Bounded two-level grid barrier for cooperative launches (groups of kGroup
// blocks, then the group leaders). The last block to arrive runs `last(…)`
// while every other block is waiting, then releases them. A wait gives up
// after ~2^22 polls: it records kErrTimeout in *err and every block returns
// false, so a caller leaves its kernel instead of spinning.
template <class Last>
__device__ __forceinline__ bool bar2(Bar2* bar, unsigned nblocks, uint32_t* err, Last last) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        s_ok = 1;
        dev_atomic gen(bar->gen);
        const unsigned g0 = gen.load(cuda::memory_order_acquire);
        __threadfence();
        const unsigned grp = blockIdx.x / kGroup;
        const unsigned gsize = min(kGroup, nblocks - grp * kGroup);
        const unsigned ngroups = (nblocks + kGroup - 1) / kGroup;
        bool released = false;
        dev_atomic gc(bar->grp[grp]);
        if (gc.fetch_add(1u, cuda::memory_order_acq_rel) == gsize - 1) {
            gc.store(0u, cuda::memory_order_relaxed);
            dev_atomic cc(bar->count);
            if (cc.fetch_add(1u, cuda::memory_order_acq_rel) == ngroups - 1) {
                cc.store(0u, cuda::memory_order_relaxed);
                last();
                gen.fetch_add(1u, cuda::memory_order_release);
                released = true;
            }
        }
        if (!released) {
            dev_atomic e(*err);
            uint32_t polls = 0;
            while (gen.load(cuda::memory_order_acquire) == g0) {
                if (++polls > (1u << 22) || (e.load(cuda::memory_order_relaxed) & kErrTimeout)) {
                    atomicOr(err, kErrTimeout);
                    break;
                }
                if (polls > 4096) __nanosleep(64);
            }
        }
        if (dev_atomic(*err).load(cuda::memory_order_relaxed) & (kErrTimeout | kErrFrontier)) s_ok = 0;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ uint32_t lane_id32() { return threadIdx.x & 31u; }

// Warp-aggregated reservation of `want` slots; returns this lane's first slot.
// Every lane of the warp must call it.
__device__ __forceinline__ uint32_t warp_reserve(uint32_t* ctr, uint32_t want) {
    const unsigned lane = lane_id32();
    uint32_t incl = want;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= unsigned(d)) incl += y;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + incl - want;
}

}  // namespace vf
