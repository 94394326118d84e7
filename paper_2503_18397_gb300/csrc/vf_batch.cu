// Batched construction kernels of libvfunc (sm_103a): hashing, shard
// histograms and the radix scatter for many independent structures at once.
// The keys of all structures form one index space; each item of the
// descriptor table owns the range [key_off, key_off + n) of it, and each
// (structure, shard) pair owns one histogram / cursor slot.
#include "vf_internal.h"

namespace vf {

constexpr int kBT = 256;
constexpr int kItemCache = 4096;  // key offsets of up to 4096 structures cached in shared memory

// Item owning global key g: largest i with key_off[i] <= g.
__device__ __forceinline__ uint32_t find_item(const uint64_t* off, uint32_t count, uint64_t g) {
    uint32_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t batch_value(const void* values, int b, uint64_t i) {
    uint32_t v;
    if (b <= 8) v = __ldg(static_cast<const uint8_t*>(values) + i);
    else if (b <= 16) v = __ldg(static_cast<const uint16_t*>(values) + i);
    else v = __ldg(static_cast<const uint32_t*>(values) + i);
    return b == 32 ? v : (v & ((1u << b) - 1u));
}

// Loads the items' key offsets into shared memory when they fit.
__device__ __forceinline__ const uint64_t* cache_offsets(const BatchItem* items, uint32_t count, uint64_t* s_off) {
    if (count <= kItemCache) {
        for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) s_off[i] = items[i].key_off;
        __syncthreads();
        return s_off;
    }
    return nullptr;
}

__device__ __forceinline__ uint32_t item_of(const BatchItem* items, const uint64_t* s_off, const uint64_t* g_off,
                                            uint32_t count, uint64_t g) {
    return find_item(s_off ? s_off : g_off, count, g);
}

// Per-(structure, shard) key counts. Lanes of a warp that hit the same slot
// add once (match + popcount).
__global__ void __launch_bounds__(kBT) k_batch_hist(const BatchItem* __restrict__ items,
                                                    const uint64_t* __restrict__ key_off, uint32_t count,
                                                    uint64_t total, uint32_t* __restrict__ hist) {
    __shared__ uint64_t s_off[kItemCache];
    const uint64_t* so = cache_offsets(items, count, s_off);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t warp0 = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u);
    const unsigned lane = threadIdx.x & 31u;
    for (uint64_t g0 = warp0; g0 < total; g0 += stride) {
        const uint64_t g = g0 + lane;
        uint32_t slot = 0xFFFFFFFFu;
        if (g < total) {
            const uint32_t it = item_of(items, so, key_off, count, g);
            const BatchItem& d = items[it];
            const Sig s = sig_u64(__ldg(d.keys + (g - d.key_off)), d.kh, d.kl);
            slot = d.hist_off + uint32_t(shard_of(s, d.h));
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, slot);
        if (slot != 0xFFFFFFFFu && lane == unsigned(__ffs(peers) - 1)) atomicAdd(hist + slot, uint32_t(__popc(peers)));
    }
}

// Radix scatter into the concatenated bucketed arrays: cursor[slot] starts at
// the slot's first position and advances by the number of lanes writing there.
__global__ void __launch_bounds__(kBT) k_batch_scatter(const BatchItem* __restrict__ items,
                                                       const uint64_t* __restrict__ key_off, uint32_t count,
                                                       uint64_t total, unsigned long long* __restrict__ cursor,
                                                       uint64_t* __restrict__ loc_out, uint32_t* __restrict__ val_out) {
    __shared__ uint64_t s_off[kItemCache];
    const uint64_t* so = cache_offsets(items, count, s_off);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t warp0 = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u);
    const unsigned lane = threadIdx.x & 31u;
    for (uint64_t g0 = warp0; g0 < total; g0 += stride) {
        const uint64_t g = g0 + lane;
        uint32_t slot = 0xFFFFFFFFu;
        uint64_t local = 0;
        uint32_t value = 0;
        if (g < total) {
            const uint32_t it = item_of(items, so, key_off, count, g);
            const BatchItem& d = items[it];
            const uint64_t j = g - d.key_off;
            const Sig s = sig_u64(__ldg(d.keys + j), d.kh, d.kl);
            slot = d.hist_off + uint32_t(shard_of(s, d.h));
            local = local_of(s, d.h);
            value = d.vals ? batch_value(d.vals, d.b, j) : 0u;
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, slot);
        const unsigned leader = unsigned(__ffs(peers) - 1);
        unsigned long long base = 0;
        if (slot != 0xFFFFFFFFu && lane == leader) base = atomicAdd(cursor + slot, (unsigned long long)__popc(peers));
        base = __shfl_sync(0xFFFFFFFFu, base, int(leader));
        if (slot != 0xFFFFFFFFu) {
            const uint64_t pos = base + __popc(peers & ((1u << lane) - 1u));
            loc_out[pos] = local;
            val_out[pos] = value;
        }
    }
}

static unsigned batch_grid(uint64_t total) {
    uint64_t blocks = (total + kBT - 1) / kBT;
    const uint64_t cap = uint64_t(num_sms()) * 8;
    if (blocks > cap) blocks = cap;
    return unsigned(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_batch_hist(const BatchItem* items, const uint64_t* key_off, uint32_t count, uint64_t total,
                              uint32_t* hist, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    k_batch_hist<<<batch_grid(total), kBT, 0, st>>>(items, key_off, count, total, hist);
    return cudaGetLastError();
}

cudaError_t launch_batch_scatter(const BatchItem* items, const uint64_t* key_off, uint32_t count, uint64_t total,
                                 unsigned long long* cursor, uint64_t* loc, uint32_t* val, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    k_batch_scatter<<<batch_grid(total), kBT, 0, st>>>(items, key_off, count, total, cursor, loc, val);
    return cudaGetLastError();
}

}  // namespace vf
