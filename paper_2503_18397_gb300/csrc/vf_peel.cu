// Fuse-regime solver of libvfunc (sm_103a): peeling in synchronous rounds and
// reverse-round assignment for shards whose vertex state lives in global
// memory (L2-resident per round).
//
// Peeling (Sec. 4.3 visit, round-synchronous): a frontier entry is a vertex of
// degree one together with its only edge, read exactly from the compare-and-
// swap that brought the vertex's packed word (bits 0..4 degree, bits 5..31 XOR
// of shard-local edge indices) to degree one. Later changes to that word can
// only remove that very edge, which claims it, so a round needs no re-read of
// the word: it claims the edge with one bit, removes it from the other two
// vertices with compare-and-swap, and pushes every vertex that reaches degree
// one. Each peeled edge writes a 16-byte assignment record {peeled vertex,
// other vertex, other vertex, value}; round r's records are contiguous.
//
// Assignment runs the rounds in reverse: an edge peeled in round r has its
// other two vertices either never peeled (value 0) or peeled in a later round,
// and no two edges of a round share their peeled vertex.
//
// Rounds are separated by a two-level grid barrier (groups of 8 blocks, then
// the group leaders) whose waits are bounded: after ~2^22 polls a wait records
// kErrTimeout and every block leaves the kernel.
#include <cuda/atomic>

#include "vf_grid.cuh"
#include "vf_internal.h"

namespace vf {

constexpr int kPT = 1024;          // threads per block (one block per SM)
constexpr int kStartCache = 2048;  // shard starts cached in shared memory

__device__ __forceinline__ unsigned long long shard_start(const FuseSolveArgs& a, const unsigned long long* sst,
                                                          uint32_t s) {
    return a.S < kStartCache ? sst[s] : __ldg(a.start + s);
}

__global__ void __launch_bounds__(kPT, 1) k_peel2(FuseSolveArgs a) {
    __shared__ unsigned long long sst[kStartCache];
    if (a.S < kStartCache)
        for (uint32_t i = threadIdx.x; i <= a.S; i += blockDim.x) sst[i] = __ldg(a.start + i);
    const unsigned nblocks = gridDim.x;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t warp0 = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u);
    const unsigned lane = lane_id32();
    const uint32_t cells = uint32_t(a.g.cells);
    const uint64_t V = uint64_t(a.S) * cells;
    __syncthreads();

    // Round 0 frontier: every vertex of degree one, with its edge.
    for (uint64_t v0 = warp0; v0 < V; v0 += nthreads) {
        const uint64_t v = v0 + lane;
        uint32_t w = v < V ? __ldcg(a.W + v) : 0u;
        const bool one = (w & 31u) == 1u;
        const uint32_t slot = warp_reserve(&a.ctr[0], one ? 1u : 0u);
        if (one) {
            if (slot < a.front_cap) {
                const uint32_t s = uint32_t(v) / cells;
                a.front[0][slot] = make_uint2(uint32_t(v), uint32_t(shard_start(a, sst, s) + (w >> 5)));
            } else {
                atomicOr(a.err, kErrFrontier);
            }
        }
    }
    if (!bar2(a.bar, nblocks, a.err, [&] {
            a.ctr[1] = 0;
            a.ctr[3] = 0;
        }))
        return;

    for (uint32_t r = 0;; r++) {
        const uint32_t cur = r & 1u, nxt = cur ^ 1u;
        const uint32_t sz = dev_atomic(a.ctr[cur]).load(cuda::memory_order_relaxed);
        if (sz == 0) break;
        const uint2* F = a.front[cur];
        uint2* G = a.front[nxt];
        for (uint64_t i0 = warp0; i0 < sz; i0 += nthreads) {
            const uint64_t i = i0 + lane;
            bool peel = false;
            uint4 rec = make_uint4(0, 0, 0, 0);
            uint32_t other3 = 0;
            uint2 push[3] = {make_uint2(0, 0), make_uint2(0, 0), make_uint2(0, 0)};
            uint32_t np = 0;
            const int kk = a.g.k == 4 ? 4 : 3;
            if (i < sz) {
                const uint2 fe = __ldcg(F + i);
                const uint32_t v = fe.x, e = fe.y;
                const uint64_t local = __ldg(a.loc + e);
                const uint32_t value = a.val ? __ldg(a.val + e) : 0u;
                const uint32_t bit = 1u << (e & 31u);
                if (!(atomicOr(a.claimed + (e >> 5), bit) & bit)) {
                    peel = true;
                    const uint32_t s = v / cells;
                    const uint32_t base = s * cells;
                    const unsigned long long st0 = shard_start(a, sst, s);
                    const uint32_t el = uint32_t(e - st0);
                    uint64_t vv[4];
                    edge_of(a.g, local, vv);
                    const uint32_t lv = v - base;
                    uint32_t side = 0;
                    for (int k = 0; k < kk; k++)
                        if (uint32_t(vv[k]) == lv) side = uint32_t(k);
                    uint32_t other[3] = {0, 0, 0};
                    int o = 0;
                    for (int k = 0; k < kk; k++)
                        if (uint32_t(k) != side) other[o++] = base + uint32_t(vv[k]);
                    for (int k = 0; k < kk - 1; k++) {
                        uint32_t* wp = a.W + other[k];
                        uint32_t old = __ldcg(wp);
                        for (;;) {
                            const uint32_t nw = ((old ^ (el << 5)) & ~31u) | ((old & 31u) - 1u);
                            const uint32_t got = atomicCAS(wp, old, nw);
                            if (got == old) {
                                if ((nw & 31u) == 1u) push[np++] = make_uint2(other[k], uint32_t(st0 + (nw >> 5)));
                                break;
                            }
                            old = got;
                        }
                    }
                    rec = make_uint4(v, other[0], other[1], a.val ? value : fingerprint_slice(local, a.g.b, a.g.fpb, a.g.fps));
                    other3 = other[2];
                }
            }
            const uint32_t slot = warp_reserve(&a.ctr[2], peel ? 1u : 0u);
            if (peel) {
                a.rec[slot] = rec;
                if (a.rec3) a.rec3[slot] = other3;
            }
            const uint32_t fs = warp_reserve(&a.ctr[nxt], np);
            if (np) {
                if (fs + np <= a.front_cap) {
                    for (uint32_t k = 0; k < np; k++) G[fs + k] = push[k];
                } else {
                    atomicOr(a.err, kErrFrontier);
                }
            }
        }
        if (!bar2(a.bar, nblocks, a.err, [&] {
                const uint32_t nr = r + 1;
                if (nr < a.round_cap) a.round_off[nr] = a.ctr[2];
                else atomicOr(a.err, kErrFrontier);
                a.ctr[cur] = 0;
                a.ctr[3] = nr;
            }))
            return;
    }
}

__global__ void __launch_bounds__(kPT, 1) k_assign2(FuseSolveArgs a) {
    const unsigned nblocks = gridDim.x;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
    const int b = a.g.b;
    for (uint32_t r = a.rounds; r-- > 0;) {
        const uint32_t lo = __ldg(a.round_off + r), hi = __ldg(a.round_off + r + 1);
        for (uint64_t i = lo + tid; i < hi; i += nthreads) {
            const uint4 rec = __ldg(a.rec + i);
            uint32_t x =
                rec.w ^ cell_get_cg(a.data, b, a.cell_base + rec.y) ^ cell_get_cg(a.data, b, a.cell_base + rec.z);
            if (a.rec3) x ^= cell_get_cg(a.data, b, a.cell_base + __ldg(a.rec3 + i));
            cell_put_zero(a.data, b, a.cell_base + rec.x, x);
        }
        if (r > 0 && !bar2(a.bar, nblocks, a.err, [] {})) return;
    }
}

// Blocks for a cooperative launch: one per SM at most, fewer for small graphs
// (a round's frontier is a thin wave, so fewer blocks mean a cheaper barrier).
static unsigned fuse_grid(const void* fn, uint64_t vertices) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPT, 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t cap = uint64_t(num_sms());
    uint64_t want = (vertices + (uint64_t(1) << 16) - 1) >> 16;
    if (want < 1) want = 1;
    return unsigned(want < cap ? want : cap);
}

cudaError_t launch_peel(FuseSolveArgs a, cudaStream_t st) {
    void* args[] = {&a};
    const unsigned grid = fuse_grid(reinterpret_cast<const void*>(k_peel2), uint64_t(a.S) * a.g.cells);
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_peel2), dim3(grid), dim3(kPT), args, 0, st);
}

cudaError_t launch_assign(FuseSolveArgs a, cudaStream_t st) {
    if (a.rounds == 0) return cudaSuccess;
    void* args[] = {&a};
    const unsigned grid = fuse_grid(reinterpret_cast<const void*>(k_assign2), uint64_t(a.S) * a.g.cells);
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_assign2), dim3(grid), dim3(kPT), args, 0,
                                       st);
}

}  // namespace vf
