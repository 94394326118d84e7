// Asynchronous fuse-regime solver of libvfunc (sm_103a): worklist peeling and
// dataflow assignment, with no grid-wide barrier between peeling steps.
//
// Vertex word (32 bits): bits 0..4 degree, bits 5..31 the SUM modulo 2^27 of
// the shard-local indices of the incident edges (a shard holds fewer than 2^27
// edges). It plays the part of the XOR trick of Sec. 4.3: at degree one the sum
// is the one remaining edge index. Removing an edge is a single fetch-and-add,
// so a peeling step needs no read-modify-write retry loop.
//
// Peeling (the visit of Sec. 4.3 with many stacks at once): a lane follows one
// chain: after peeling an edge it continues with a vertex that the edge brought
// to degree one. A second such vertex goes to a free lane of the same warp
// (a fork, by shuffle) or, when the warp has none, to a global queue. Lanes
// of a warp with no work at all reserve queue slots and take the item once it
// is written.
//
// Order: every item takes a record slot from its shard's counter together
// with its claim, before it removes the edge from the other two vertices. A
// vertex that an edge f still touches can only be peeled (by some edge g of
// the same shard) after f's removal from it, hence after f's slot was taken:
// g's slot is larger. So each shard's records in decreasing slot order are a
// reverse peeling order, the order in which assignment must run (each peeled
// vertex is assigned after the vertices its value depends on). Items whose
// claim failed leave an empty slot. One counter per shard (each on its own
// line) instead of one for all: the counter is taken by every warp step, and
// doubling the traffic on a single shared one cost 12% of the peel.
// Why "before" holds on the hardware and not only in program order: the slot
// fetch-and-add is issued by one lane of each group of the warp's lanes with
// the same shard, and the whole warp then executes a warp-synchronous shuffle
// of the returned values (every lane's slot comes from its group's) before
// reaching the removals. The shuffle cannot execute before those values have
// returned, a warp issues its instructions in order, and a fetch-and-add
// returns only once it has been performed at L2; so the slot is taken, at L2,
// before either removal of the step is even issued, and a later peel of a
// vertex the removal freed takes its slot from the same counter afterwards.
// The compiler barrier keeps the compiler from moving the removals above the
// shuffle.
//
// Assignment is a dataflow in decreasing slot order per shard: once final, a
// vertex's value word (64 bits, in the queue's memory) holds its value with bit
// 32 set (vertices no edge was peeled from are final from the start, value 0);
// an edge waits (bounded) until its two other vertices are final. An edge only
// waits on edges of its shard with larger slots, which were handed out before
// it, so the earliest unfinished edge can always proceed.
#include <atomic>

#include <cuda/atomic>

#include "vf_internal.h"

namespace vf {

constexpr int kFT = 256;
constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kFinal = 1ull << 32;
constexpr uint32_t kHole = 0xFFFFFFFFu;     // record of an item whose claim failed
constexpr uint32_t kIdleLimit = 1u << 23;  // polls of ~1 us: a wait gives up after ~8 s
constexpr unsigned kNapMax = 512;          // ns, peeling (idle lanes; 256 -> 512 ns: -0.7%)
constexpr unsigned kAssignNapMin = 16;     // ns, assignment: first back-off
constexpr unsigned kAssignNapMax = 16;     // ns, assignment: longest back-off (measured: 256 -> 16 ns
                                           // took the assignment from 12.5 to 10.9 ms at 10^8 keys)
constexpr uint32_t kWavePrefetch = 5;      // segments ahead of a peeling step whose vertex words are prefetched
constexpr uint32_t kSigPrefetch = 3;       // and whose edges' signatures are (2: same, 5: +0.7%; none: +6%)

using dev_atomic32 = cuda::atomic_ref<unsigned int, cuda::thread_scope_device>;
using dev_atomic64 = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;

__device__ __forceinline__ unsigned lane32() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanes_below() { return (1u << lane32()) - 1u; }

__device__ __forceinline__ uint32_t flow_shard_of_edge(const unsigned long long* __restrict__ start, uint32_t S,
                                                       uint64_t e) {
    uint32_t lo = 0, hi = S;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// One slot each for the lanes in `mask` (non-empty), from a 64-bit counter.
__device__ __forceinline__ unsigned long long reserve64(unsigned long long* ctr, unsigned mask, bool me) {
    const int lead = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (int(lane32()) == lead) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, lead);
    return me ? base + __popc(mask & lanes_below()) : 0ull;
}

// Position of the r-th (from 0) set bit of m; m has more than r set bits.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t r) {
    uint32_t pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const uint32_t low = (1u << w) - 1u;
        const uint32_t c = __popc(m & low);
        if (r >= c) {
            r -= c;
            m >>= w;
            pos += w;
        } else {
            m &= low;
        }
    }
    return pos;
}

__device__ __forceinline__ unsigned long long* ctr64(const FlowArgs& a, uint32_t word) {
    return reinterpret_cast<unsigned long long*>(a.ctr + word);
}

// Incidence: degree += 1 and sum += shard-local edge index, per vertex. Edges
// whose bit is set in `drop` (duplicate filter keys) are left out.
__global__ void __launch_bounds__(kFT) k_incidence32(const uint64_t* __restrict__ loc, uint64_t n,
                                                     const unsigned long long* __restrict__ start, uint32_t S, Geom g,
                                                     uint32_t* __restrict__ W, uint32_t* err,
                                                     const uint32_t* __restrict__ drop) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < n; e += stride) {
        if (drop && ((__ldg(drop + (e >> 5)) >> (e & 31u)) & 1u)) continue;
        const uint32_t s = flow_shard_of_edge(start, S, e);
        const uint32_t inc = 1u + (uint32_t(e - __ldg(start + s)) << 5);
        uint64_t v[4];
        edge_of(g, __ldg(loc + e), v);
        const uint64_t base = uint64_t(s) * g.cells;
        const int kk = g.k == 4 ? 4 : 3;
        uint32_t old[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (k < kk) old[k] = atomicAdd(W + base + v[k], inc);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if ((old[k] & 31u) == 31u) atomicOr(err, kErrDegOverflow);
    }
}

// The same incidence over segment-ordered edges, owner-computes: a block owns
// one segment t of one shard at a time and accumulates, in shared memory, every
// contribution that lands in it: vertex j of the edges of bin t - j for j < k
// (edges start in a segment and reach the next k - 1). It then stores the
// segment's vertex words, so no global atomic is needed and the words need no
// zeroing before. An edge is read by k blocks. seg_ends[i]: one past the last
// edge of bin i (bins in (shard, segment) order, one segment each, l = T - k + 1
// bins a shard). A segment larger than shared memory holds (2^15 words) is owned
// in chunks of 2^15 cells by as many blocks, each reading the segment's bins and
// keeping the contributions that land in its chunk (the neighbouring chunks'
// blocks read the same bins at about the same time, so L2 serves the repeats).
// XOR: the round solver's words (degree, XOR of the indices) instead of the
// worklist solver's (degree, sum of the indices).
constexpr int kIncSegThreads = 1024;
constexpr uint32_t kIncSegLgChunk = 15;  // cells a block owns at once: 128 KB of shared memory
constexpr uint32_t kIncSegLgMax = 18;    // larger segments: at most 8 chunks, each reading the bins
constexpr uint32_t kIncSegUnroll = 8;    // edges a thread loads before using any
constexpr uint32_t kSegBins = 2048;  // segment groups per shard in the segment order (below)

template <bool XOR>
__global__ void __launch_bounds__(kIncSegThreads) k_incidence_seg(const uint64_t* __restrict__ loc,
                                                                  const unsigned long long* __restrict__ start,
                                                                  uint32_t S, uint32_t nb, Geom g,
                                                                  const unsigned long long* __restrict__ seg_ends,
                                                                  uint32_t* __restrict__ W, uint32_t* err,
                                                                  const uint32_t* __restrict__ drop) {
    extern __shared__ uint32_t sw[];
    const uint32_t lgc = g.lg_seg < kIncSegLgChunk ? g.lg_seg : kIncSegLgChunk;
    const uint32_t chunk = 1u << lgc, nch = 1u << (g.lg_seg - lgc);
    const uint32_t K = g.k == 4 ? 4u : 3u;
    const uint32_t T = nb + K - 1;  // segments of a shard
    const uint64_t tasks = uint64_t(S) * T * nch;
    for (uint64_t task = blockIdx.x; task < tasks; task += gridDim.x) {
        const uint32_t ch = uint32_t(task % nch);
        const uint32_t sh = uint32_t(task / nch / T);
        const uint32_t t = uint32_t(task / nch % T);
        const uint64_t st0 = __ldg(start + sh);
        for (uint32_t i = threadIdx.x; i < chunk; i += blockDim.x) sw[i] = 0;
        __syncthreads();
        bool wrap = false;
#pragma unroll 1
        for (uint32_t k = 0; k < K; k++) {  // vertex k of the edges of bin t - k
            if (t < k || t - k >= nb) continue;
            const uint64_t bin = uint64_t(sh) * nb + (t - k);
            const uint64_t lo = bin ? __ldg(seg_ends + bin - 1) : 0ull, hi = __ldg(seg_ends + bin);
            const uint64_t choff = uint64_t(ch) << lgc;  // the chunk's first cell within the segment
            const uint64_t step = uint64_t(kIncSegUnroll) * blockDim.x;
            for (uint64_t e0 = lo + threadIdx.x; e0 < hi; e0 += step) {
                // all of a thread's signature (and drop-word) loads are issued
                // before any is used: one load in flight per thread left the
                // block bound by the load latency, not by bandwidth
                uint64_t sg[kIncSegUnroll];
                uint32_t dw[kIncSegUnroll];
#pragma unroll
                for (uint32_t u = 0; u < kIncSegUnroll; u++) {
                    const uint64_t e = e0 + uint64_t(u) * blockDim.x;
                    sg[u] = e < hi ? __ldg(loc + e) : 0ull;
                    dw[u] = (drop && e < hi) ? __ldg(drop + (e >> 5)) : 0u;
                }
#pragma unroll
                for (uint32_t u = 0; u < kIncSegUnroll; u++) {
                    const uint64_t e = e0 + uint64_t(u) * blockDim.x;
                    if (e >= hi || ((dw[u] >> (e & 31u)) & 1u)) continue;
                    const uint32_t el = uint32_t(e - st0);
                    // vertex k of a bin t - k edge lies in segment t (for k = 0 this is
                    // checked: a misplaced edge gives an offset beyond the segment)
                    const uint64_t r = fuse_vertex_in_segment(g, sg[u], k, t) - choff;
                    if (r >= chunk) {
                        // another chunk of the segment (or, if the segment has one chunk,
                        // impossible for segment-ordered edges)
                        if (nch == 1) wrap = true;
                    } else if (XOR) {
                        wrap |= (atomicAdd(sw + r, 1u) & 31u) == 31u;
                        atomicXor(sw + r, el << 5);
                    } else {
                        wrap |= (atomicAdd(sw + r, 1u + (el << 5)) & 31u) == 31u;
                    }
                }
            }
        }
        if (wrap) atomicOr(err, kErrDegOverflow);
        __syncthreads();
        uint32_t* out = W + uint64_t(sh) * g.cells + (uint64_t(t) << g.lg_seg) + (uint64_t(ch) << lgc);
        for (uint32_t i = threadIdx.x; i < chunk; i += blockDim.x) out[i] = sw[i];
        __syncthreads();
    }
}

bool incidence_seg_fits(const Geom& g) {
    if (g.regime != kRegimeFuse || (g.k != 3 && g.k != 4) || g.lg_seg > kIncSegLgMax || g.lg_seg < 5) return false;
    const uint32_t l = uint32_t(g.span >> g.lg_seg);
    return l >= 1 && l <= kSegBins;  // one segment per bin of the segment order
}

cudaError_t launch_incidence_seg(const uint64_t* loc, uint64_t n, const unsigned long long* start, uint32_t S,
                                 const Geom& g, const unsigned long long* seg_ends, uint32_t* W, uint32_t* err,
                                 const uint32_t* drop, bool xor_words, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (!incidence_seg_fits(g)) return cudaErrorInvalidValue;
    const uint32_t nb = uint32_t(g.span >> g.lg_seg);
    const uint32_t lgc = g.lg_seg < kIncSegLgChunk ? g.lg_seg : kIncSegLgChunk;
    const size_t smem = (size_t(1) << lgc) * 4;
    static std::atomic<uint64_t> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(attr_done.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_incidence_seg<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(size_t(1) << 17));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_incidence_seg<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(size_t(1) << 17));
        if (e != cudaSuccess) return e;
        attr_done.fetch_or(bit);
    }
    const uint64_t tasks = uint64_t(S) * (nb + (g.k == 4 ? 3 : 2)) << (g.lg_seg - lgc);
    const unsigned grid = unsigned(std::min<uint64_t>(tasks, uint64_t(num_sms())));
    if (xor_words)
        k_incidence_seg<true><<<grid, kIncSegThreads, smem, st>>>(loc, start, S, nb, g, seg_ends, W, err, drop);
    else
        k_incidence_seg<false><<<grid, kIncSegThreads, smem, st>>>(loc, start, S, nb, g, seg_ends, W, err, drop);
    return cudaGetLastError();
}

// Initial items: every vertex of degree one with its edge, for the shards
// [s_lo, s_hi) of one peeling batch. A block takes chunks of kSeedPer * kFT
// vertices and reserves the chunk's queue slots with one atomic.
constexpr int kSeedPer = 16;

__global__ void __launch_bounds__(kFT) k_flow_seed(FlowArgs a, uint32_t s_lo, uint32_t s_hi) {
    __shared__ uint32_t s_warp[kFT / 32];
    __shared__ unsigned long long s_base;
    const uint32_t cells = uint32_t(a.g.cells);
    const uint64_t V = uint64_t(s_hi) * cells;
    const uint64_t chunk = uint64_t(kFT) * kSeedPer;
    const unsigned warp = threadIdx.x >> 5;
    for (uint64_t c0 = uint64_t(s_lo) * cells + blockIdx.x * chunk; c0 < V; c0 += uint64_t(gridDim.x) * chunk) {
        uint32_t w[kSeedPer], cnt = 0;
#pragma unroll
        for (int j = 0; j < kSeedPer; j++) {
            const uint64_t v = c0 + uint64_t(j) * kFT + threadIdx.x;
            w[j] = v < V ? a.W[v] : 0u;
            cnt += (w[j] & 31u) == 1u;
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane32() >= unsigned(d)) incl += y;
        }
        if (lane32() == 31) s_warp[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t total = 0;
            for (int i = 0; i < kFT / 32; i++) {
                const uint32_t t = s_warp[i];
                s_warp[i] = total;
                total += t;
            }
            s_base = total ? atomicAdd(ctr64(a, kFlowSlots), (unsigned long long)total << 32) >> 32 : 0ull;
        }
        __syncthreads();
        unsigned long long slot = s_base + s_warp[warp] + incl - cnt;
#pragma unroll
        for (int j = 0; j < kSeedPer; j++) {
            if ((w[j] & 31u) == 1u) {
                const uint64_t v = c0 + uint64_t(j) * kFT + threadIdx.x;
                a.queue[slot++] = (v << 32) | (__ldg(a.start + uint32_t(v / cells)) + (w[j] >> 5));
            }
        }
        __syncthreads();
    }
}

// Between peeling batches: consumers of the next batch start at the tail (the
// lanes that reserved slots beyond it have left).
__global__ void k_rebase_head(FlowArgs a) {
    *ctr64(a, kFlowHead) = *ctr64(a, kFlowSlots) >> 32;
}

// Peeled edges = set claim bits.
__global__ void __launch_bounds__(kFT) k_count_claims(FlowArgs a, uint64_t words) {
    uint32_t c = 0;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < words; i += uint64_t(gridDim.x) * blockDim.x)
        c += __popc(__ldg(a.claimed + i));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, d);
    if (lane32() == 0 && c) atomicAdd(a.ctr + kFlowPeeled, c);
}

// Worklist peeling; one chain per lane at a time. An iteration has two memory
// phases per warp: first every request that does not depend on this
// iteration's results (queue slots for idle lanes, polls of reserved slots,
// the item's signature, its claim, its record slot, the queue slot of an item
// produced in the previous iteration), then the removals of the claimed edges.
// The record and queue-tail counters share one 64-bit word (record slots in
// the low half, queue slots in the high half), so one fetch-and-add takes both.
// Termination: chains start from queue items (tail counter) or forks. The done
// counter holds chain ends minus forks, added once per iteration by lane 0 (so
// a fork is subtracted before its chain's end is added); done == tail means no
// chain is running. Reading done, then tail, and finding them equal means none
// ran when done was read, so none can start again.
// K: vertices per edge (3, or 4 for a 4-uniform fuse graph), fixed at compile time.
template <int K>
__global__ void __launch_bounds__(kFT) k_flow_peel(FlowArgs a) {
    const unsigned lane = lane32();
    const uint32_t cells = uint32_t(a.g.cells);
    unsigned long long* head = ctr64(a, kFlowHead);
    unsigned long long* slots = ctr64(a, kFlowSlots);
    unsigned long long* done = ctr64(a, kFlowDone);
    bool have = false;                   // holds an item (v, e)
    unsigned long long slot = ~0ull;     // reserved queue slot, not yet filled
    bool pend = false;                   // produced item (pu, pe) waiting for a queue slot
    uint32_t v = 0, e = 0, pu = 0, pe = 0;
    uint32_t idle = 0;
    uint32_t dacc = 0;  // lane 0: ended chains not yet added to done
    unsigned nap = 32;
    for (;;) {
        const unsigned mhave = __ballot_sync(0xFFFFFFFFu, have);
        const bool need = !have && slot == ~0ull && mhave == 0;  // only an idle warp takes queue slots
        const unsigned mneed = __ballot_sync(0xFFFFFFFFu, need);
        const unsigned mpend = __ballot_sync(0xFFFFFFFFu, pend);
        // ---- phase 1: independent requests, all in flight together
        unsigned long long hb = 0, rt = 0;  // rt: queue slots (high half)
        uint32_t rbase = 0, rgrp = 0, rsh = 0;  // record slots: a counter per shard
        if (mneed && int(lane) == __ffs(mneed) - 1) hb = atomicAdd(head, (unsigned long long)__popc(mneed));
        if (mpend && int(lane) == __ffs(mpend) - 1) rt = atomicAdd(slots, (unsigned long long)__popc(mpend) << 32);
        if (have) {  // one fetch-and-add per shard among the warp's items
            rsh = v / cells;
            rgrp = __match_any_sync(mhave, rsh);
            if (int(lane) == __ffs(rgrp) - 1) rbase = atomicAdd(a.rc + rsh * kRcStride, uint32_t(__popc(rgrp)));
        }
        unsigned long long it = kEmpty;
        if (!have && slot < a.queue_cap) it = dev_atomic64(a.queue[slot]).load(cuda::memory_order_relaxed);
        uint64_t local = 0;
        uint32_t value = 0, cold = 0;
        const uint32_t bit = 1u << (e & 31u);
        if (have) {
            local = __ldg(a.loc + e);
            if (a.val) value = __ldg(a.val + e);
            cold = atomicOr(a.claimed + (e >> 5), bit);
        }
        if (mneed) {
            hb = __shfl_sync(0xFFFFFFFFu, hb, __ffs(mneed) - 1);
            if (need) slot = hb + __popc(mneed & lanes_below());
        }
        if (mpend) rt = __shfl_sync(0xFFFFFFFFu, rt, __ffs(mpend) - 1);
        if (mhave) {
            const uint32_t b0 = __shfl_sync(0xFFFFFFFFu, rbase, have ? __ffs(rgrp) - 1 : int(lane));
            if (have) rbase = b0 + __popc(rgrp & lanes_below());
        }
        if (mpend) {
            if (pend) {
                const unsigned long long qs = (rt >> 32) + __popc(mpend & lanes_below());
                if (qs < a.queue_cap)
                    dev_atomic64(a.queue[qs]).store((unsigned long long)pu << 32 | pe, cuda::memory_order_relaxed);
                else
                    atomicOr(a.err, kErrFrontier);
                pend = false;
            }
        }
        bool got = false;
        if (!have && it != kEmpty) {
            got = true;
            slot = ~0ull;
        }
        // ---- phase 2: removals of the claimed edges
        bool retire = false;
        if (mhave) {
            asm volatile("" ::: "memory");  // the record slot is taken before the removals below
            const bool peeled = have && !(cold & bit);
            bool next = false;
            uint32_t nv = 0, ne = 0;
            if (have) {
                const uint64_t rs = uint64_t(rsh) * cells + rbase;
                if (peeled) {
                    atomicOr(a.pv + (v >> 5), 1u << (v & 31u));
                    const uint32_t s = rsh;  // v / cells, taken in phase 1
                    const uint32_t base = s * cells;
                    const unsigned long long st0 = __ldg(a.start + s);
                    const uint32_t dec = 1u + (uint32_t(e - st0) << 5);
                    uint64_t vv[4];
                    edge_of(a.g, local, vv);
                    const uint32_t lv = v - base;
                    constexpr bool four = K == 4;
                    // the vertices other than v, in edge order (two, or three for k = 4)
                    const uint32_t c0 = uint32_t(vv[0]), c1 = uint32_t(vv[1]), c2 = uint32_t(vv[2]);
                    const uint32_t c3 = four ? uint32_t(vv[3]) : 0u;
                    const uint32_t o0 = base + (c0 == lv ? c1 : c0);
                    const uint32_t o1 = base + (c0 == lv || c1 == lv ? c2 : c1);
                    const uint32_t o2 = base + (c0 == lv || c1 == lv || c2 == lv ? c3 : c2);
                    // the removals first; the prefetches below go out while they are in flight
                    const uint32_t a0 = atomicAdd(a.W + o0, 0u - dec);
                    const uint32_t a1 = atomicAdd(a.W + o1, 0u - dec);
                    const uint32_t a2 = four ? atomicAdd(a.W + o2, 0u - dec) : 0u;
                    if (a.g.regime == kRegimeFuse) {
                        // the waves sweep the segments: warm L2 with a line of vertex
                        // words kWavePrefetch segments ahead, in either direction
                        const uint32_t sv = lv >> a.g.lg_seg, T = cells >> a.g.lg_seg;
                        const uint32_t off = uint32_t(mix64(e) & ((1ull << a.g.lg_seg) - 1)) & ~31u;
                        if (sv + kWavePrefetch < T)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.W + base + ((sv + kWavePrefetch) << a.g.lg_seg) + off));
                        if (sv >= kWavePrefetch)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.W + base + ((sv - kWavePrefetch) << a.g.lg_seg) + off));
                    }
                    if (a.g.regime == kRegimeFuse && a.epsg) {
                        // and a line of the signatures of the edges that start about
                        // kSigPrefetch segments ahead, in either direction (edges are
                        // in segment order, about epsg per segment; a multiply-shift
                        // spreads the line over the segment without a division)
                        const uint32_t rel = uint32_t(e - st0), ns = uint32_t(__ldg(a.start + s + 1) - st0);
                        const uint32_t jit = uint32_t((uint64_t(uint32_t(mix64(e ^ 0x9E3779B9u) >> 32)) * a.epsg) >> 32);
                        const uint32_t far = kSigPrefetch * a.epsg;
                        if (rel + far + jit < ns)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.loc + st0 + rel + far + jit));
                        if (rel + jit >= far && rel + jit - far < ns)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.loc + st0 + rel + jit - far));
                    }
                    const uint32_t w0 = a0 - dec;
                    const uint32_t w1 = a1 - dec;
                    if ((w0 & 31u) == 1u) {
                        next = true;
                        nv = o0;
                        ne = uint32_t(st0 + (w0 >> 5));
                    }
                    if ((w1 & 31u) == 1u) {
                        if (!next) {
                            next = true;
                            nv = o1;
                            ne = uint32_t(st0 + (w1 >> 5));
                        } else {
                            pend = true;
                            pu = o1;
                            pe = uint32_t(st0 + (w1 >> 5));
                        }
                    }
                    if (four && ((a2 - dec) & 31u) == 1u) {
                        const uint32_t e2 = uint32_t(st0 + ((a2 - dec) >> 5));
                        if (!next) {
                            next = true;
                            nv = o2;
                            ne = e2;
                        } else if (!pend) {
                            pend = true;
                            pu = o2;
                            pe = e2;
                        } else {  // a third vertex freed at once (rare): to the queue now
                            const unsigned long long qs = atomicAdd(slots, 1ull << 32) >> 32;
                            if (qs < a.queue_cap)
                                dev_atomic64(a.queue[qs]).store((unsigned long long)o2 << 32 | e2,
                                                                cuda::memory_order_relaxed);
                            else
                                atomicOr(a.err, kErrFrontier);
                        }
                    }
                    if (rbase < cells) {  // a shard has at most one item per vertex
                        a.rec[rs] = make_uint4(v, o0, o1, a.val ? value : fingerprint_slice(local, a.g.b, a.g.fpb, a.g.fps));
                        if (four) a.rec3[rs] = o2;
                    } else {
                        atomicOr(a.err, kErrFrontier);
                    }
                } else {
                    if (rbase < cells) a.rec[rs].x = kHole;
                    else atomicOr(a.err, kErrFrontier);
                }
                if (next) {
                    v = nv;
                    e = ne;
                } else {
                    have = false;
                    retire = true;
                }
            }
        }
        // forks: second vertices go to lanes with neither an item nor a queue slot
        const bool free_lane = !have && slot == ~0ull && !got;
        const unsigned mfree = __ballot_sync(0xFFFFFFFFu, free_lane);
        const unsigned mp = __ballot_sync(0xFFFFFFFFu, pend);
        const uint32_t forks = min(__popc(mfree), __popc(mp));
        if (forks) {
            const uint32_t fr = __popc(mfree & lanes_below());
            const uint32_t src = (free_lane && fr < forks) ? nth_set_bit(mp, fr) : lane;
            const uint32_t xu = __shfl_sync(0xFFFFFFFFu, pu, src), xe = __shfl_sync(0xFFFFFFFFu, pe, src);
            if (free_lane && fr < forks) {
                have = true;
                v = xu;
                e = xe;
            }
            if (pend && uint32_t(__popc(mp & lanes_below())) < forks) pend = false;
        }
        // done += ended chains - forks (a chain that ended had its produced items
        // counted in earlier iterations). Forks are added at once; ended chains
        // wait in lane 0's count until it would go negative or the warp idles, so
        // done never runs ahead of the true count and the exit test below stays
        // exact, while the shared word is taken far less often (each taking costs
        // the whole peel: twice the traffic on it was 4.6% slower).
        const unsigned mret = __ballot_sync(0xFFFFFFFFu, retire);
        if (lane == 0) {
            const long long net = (long long)dacc + (long long)__popc(mret) - (long long)forks;
            if (net < 0) {
                atomicAdd(done, (unsigned long long)net);
                dacc = 0;
            } else {
                dacc = uint32_t(net);
            }
        }
        if (got) {
            v = uint32_t(it >> 32);
            e = uint32_t(it);
            have = true;
        }
        if (__ballot_sync(0xFFFFFFFFu, have || pend) != 0) {
            idle = 0;
            nap = 32;
            continue;
        }
        // nothing in flight in this warp: hand in its ended chains, then leave once
        // every queue item's chain has ended (checked every 8th idle pass: the
        // counters' lines are shared by all)
        if (lane == 0 && dacc) {
            atomicAdd(done, (unsigned long long)dacc);
            dacc = 0;
        }
        unsigned long long f = 0, t = 1;
        uint32_t er = 0;
        if (lane == 0 && (idle & 7u) == 0) {
            f = dev_atomic64(*done).load(cuda::memory_order_acquire);
            t = dev_atomic64(*slots).load(cuda::memory_order_relaxed) >> 32;
            er = dev_atomic32(*a.err).load(cuda::memory_order_relaxed);
        }
        f = __shfl_sync(0xFFFFFFFFu, f, 0);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        er = __shfl_sync(0xFFFFFFFFu, er, 0);
        if (f == t || (er & (kErrTimeout | kErrFrontier))) break;
        if (++idle > kIdleLimit) {
            if (lane == 0) atomicOr(a.err, kErrTimeout);
            break;
        }
        __nanosleep(nap);
        nap = min(nap * 2u, kNapMax);
    }
}

// -------------------------------------------------------------- assignment

// Vertices no edge was peeled from are final with value 0; the others wait.
__global__ void __launch_bounds__(kFT) k_final_init(FlowArgs a) {
    const uint64_t V = uint64_t(a.S) * a.g.cells;
    for (uint64_t v = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v < V; v += uint64_t(gridDim.x) * blockDim.x)
        a.fv[v] = (a.stall || ((__ldg(a.pv + (v >> 5)) >> (v & 31u)) & 1u)) ? 0ull : kFinal;
}

// Dataflow assignment over the record slots, largest slot first within each
// shard. Positions go round robin over the shards in groups of 32 (a warp's
// grab: 32 consecutive records of one shard, whose vertices were peeled close
// together; 2.5% faster than interleaving single records), so every shard's
// dataflow advances at once; a record waits only on larger slots of its own
// shard, which come at smaller positions.
template <int K>
__global__ void __launch_bounds__(kFT) k_flow_assign(FlowArgs a) {
    const int b = a.g.b;
    const uint64_t count = ((a.rmax + 31) & ~uint64_t(31)) * a.S;
    const uint64_t cells = a.g.cells;
    const unsigned lane = lane32();
    const uint32_t vmask = b == 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
    const uint32_t limit = a.assign_limit ? a.assign_limit : kIdleLimit;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(ctr64(a, kFlowNext), 32ull);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= count) break;
        const uint64_t k = base + lane;
        uint4 r = make_uint4(kHole, 0, 0, 0);
        uint32_t r3 = kHole;
        if (k < count) {
            const uint64_t c = k >> 5;  // a warp's 32 positions: consecutive records of one shard
            const uint32_t s = uint32_t(c % a.S);
            const uint64_t j = ((c / a.S) << 5) + (k & 31u);
            const uint32_t taken = __ldg(a.rc + s * kRcStride);
            if (j < taken) {
                const uint64_t rs = s * cells + (taken - 1 - j);
                r = __ldg(a.rec + rs);
                if (K == 4 && r.x != kHole) r3 = __ldg(a.rec3 + rs);  // third other vertex
            }
        }
        bool done = r.x == kHole;
        uint32_t polls = 0;
        unsigned nap = kAssignNapMin;
        bool fail = false;
        for (;;) {
            if (!done) {
                const unsigned long long wy = dev_atomic64(a.fv[r.y]).load(cuda::memory_order_relaxed);
                const unsigned long long wz = dev_atomic64(a.fv[r.z]).load(cuda::memory_order_relaxed);
                const unsigned long long w3 =
                    K == 4 && r3 != kHole ? dev_atomic64(a.fv[r3]).load(cuda::memory_order_relaxed) : kFinal;
                if (wy & wz & w3 & kFinal) {
                    const uint32_t x = (r.w ^ uint32_t(wy) ^ uint32_t(wz) ^ uint32_t(w3)) & vmask;
                    dev_atomic64(a.fv[r.x]).store(kFinal | x, cuda::memory_order_relaxed);
                    cell_put_zero(a.data, b, a.cell_base + r.x, x);
                    done = true;
                }
            }
            if (__all_sync(0xFFFFFFFFu, done)) break;
            if (++polls > limit) fail = true;
            if ((polls & 63u) == 0 && (dev_atomic32(*a.err).load(cuda::memory_order_relaxed) & kErrTimeout)) fail = true;
            if (__any_sync(0xFFFFFFFFu, fail)) {
                fail = true;
                break;
            }
            __nanosleep(nap);
            nap = min(nap * 2u, kAssignNapMax);
        }
        if (fail) {
            if (lane == 0) atomicOr(a.err, kErrTimeout);
            break;
        }
    }
}

// ----------------------------------------------------- segment order (locality)

// Edges of a fuse shard are peeled as two waves that sweep the segments, and
// the first vertex of an edge fixes its segment (v0 = mulhi(local, l*seg)
// grows with the local signature). A counting sort of each shard's edges by
// that segment (groups of 2^sshift segments when a shard has more than
// kSegBins) puts the edges the waves touch at one time next to each other, so
// incidence accumulates into a few segments' vertex words at a time and a
// peeling step's signature, value and claim bit share cache lines with its
// neighbours'. Bins are (shard, segment group); tiles of kTile consecutive
// edges (in one or two shards after the shard scatter) count and scatter
// their bins in shared memory and reserve each bin's range with one global
// atomic.
constexpr int kTile = 4096;
constexpr int kTileThreads = 256;

__device__ __forceinline__ uint32_t seg_bin(uint64_t x, const Geom& g, uint32_t sshift) {
    return uint32_t(mulhi(x, g.span) >> g.lg_seg) >> sshift;
}

// Per tile: its first shard f, the first key of shard f + 1 (relative), and
// whether it spans more than two shards (then it is counted key by key).
__device__ __forceinline__ void tile_shards(const unsigned long long* start, uint32_t S, uint64_t t0, uint32_t m,
                                            uint32_t& f, uint32_t& split, bool& many) {
    f = flow_shard_of_edge(start, S, t0);
    const uint32_t l = flow_shard_of_edge(start, S, t0 + m - 1);
    many = l - f > 1;
    const unsigned long long sp = __ldg(start + f + 1) - t0;
    split = sp < m ? uint32_t(sp) : m;
}

// counts[s * nb + bin] += edges of shard s in segment group bin.
__global__ void __launch_bounds__(kTileThreads) k_seg_count(const uint64_t* __restrict__ loc, uint64_t n,
                                                             const unsigned long long* __restrict__ start, uint32_t S,
                                                             Geom g, uint32_t nb, uint32_t sshift,
                                                             unsigned long long* __restrict__ counts) {
    extern __shared__ __align__(16) uint32_t s_cnt[];  // 2 * nb
    __shared__ uint32_t s_f, s_split;
    __shared__ bool s_many;
    for (uint64_t t0 = uint64_t(blockIdx.x) * kTile; t0 < n; t0 += uint64_t(gridDim.x) * kTile) {
        const uint32_t m = n - t0 < uint64_t(kTile) ? uint32_t(n - t0) : uint32_t(kTile);
        if (threadIdx.x == 0) {
            uint32_t f, sp;
            bool many;
            tile_shards(start, S, t0, m, f, sp, many);
            s_f = f, s_split = sp, s_many = many;
        }
        for (uint32_t i = threadIdx.x; i < 2 * nb; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        const uint32_t f = s_f, split = s_split;
        constexpr int kPer = kTile / kTileThreads;
        uint64_t xs[kPer];  // every load of the tile issued before the first count
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const uint32_t i = threadIdx.x + uint32_t(j) * kTileThreads;
            xs[j] = i < m ? __ldg(loc + t0 + i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const uint32_t i = threadIdx.x + uint32_t(j) * kTileThreads;
            if (i >= m) continue;
            if (s_many) {
                const uint32_t s = flow_shard_of_edge(start, S, t0 + i);
                atomicAdd(counts + uint64_t(s) * nb + seg_bin(xs[j], g, sshift), 1ull);
            } else {
                atomicAdd(&s_cnt[(i >= split ? nb : 0u) + seg_bin(xs[j], g, sshift)], 1u);
            }
        }
        __syncthreads();
        if (!s_many)
            for (uint32_t i = threadIdx.x; i < 2 * nb; i += blockDim.x) {
                const uint32_t c = s_cnt[i];
                const uint32_t s = f + (i >= nb ? 1u : 0u);
                if (c && s < S) atomicAdd(counts + uint64_t(s) * nb + (i >= nb ? i - nb : i), (unsigned long long)c);
            }
        __syncthreads();
    }
}

// Exclusive scan of the bin counts into cursors, starting at each shard's
// first key (one block).
__global__ void __launch_bounds__(1024) k_seg_scan(unsigned long long* __restrict__ counts, uint64_t nbins,
                                                    const unsigned long long* __restrict__ start, uint32_t nb) {
    __shared__ unsigned long long s_part[1024];
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    const uint64_t per = (nbins + T - 1) / T;
    const uint64_t b0 = min(nbins, uint64_t(tid) * per), b1 = min(nbins, b0 + per);
    unsigned long long sum = 0;
    for (uint64_t i = b0; i < b1; i++) sum += counts[i];
    s_part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0;
        for (uint32_t t = 0; t < T; t++) {
            const unsigned long long x = s_part[t];
            s_part[t] = run;
            run += x;
        }
    }
    __syncthreads();
    unsigned long long run = s_part[tid];
    for (uint64_t i = b0; i < b1; i++) {
        const unsigned long long c = counts[i];
        counts[i] = run;  // the shards are contiguous, so the running sum is also each shard's start
        run += c;
    }
}

// Scatter every edge (signature and value) to its bin's next slot.
__global__ void __launch_bounds__(kTileThreads, 3) k_seg_scatter(const uint64_t* __restrict__ loc,
                                                               const uint32_t* __restrict__ val, uint64_t n,
                                                               const unsigned long long* __restrict__ start,
                                                               uint32_t S, Geom g, uint32_t nb, uint32_t sshift,
                                                               unsigned long long* __restrict__ cursor,
                                                               uint64_t* __restrict__ loc_out,
                                                               uint32_t* __restrict__ val_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_base = reinterpret_cast<unsigned long long*>(smem);  // 2 * nb
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_base + 2 * nb);             // 2 * nb
    __shared__ uint32_t s_f, s_split;
    __shared__ bool s_many;
    for (uint64_t t0 = uint64_t(blockIdx.x) * kTile; t0 < n; t0 += uint64_t(gridDim.x) * kTile) {
        const uint32_t m = n - t0 < uint64_t(kTile) ? uint32_t(n - t0) : uint32_t(kTile);
        if (threadIdx.x == 0) {
            uint32_t f, sp;
            bool many;
            tile_shards(start, S, t0, m, f, sp, many);
            s_f = f, s_split = sp, s_many = many;
        }
        for (uint32_t i = threadIdx.x; i < 2 * nb; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        const uint32_t f = s_f, split = s_split;
        constexpr int kPer = kTile / kTileThreads;
        uint64_t xs[kPer];
        uint32_t rk[kPer], bn[kPer];
#pragma unroll
        for (int j = 0; j < kPer; j++) {  // every load of the tile issued before the first rank
            const uint32_t i = threadIdx.x + uint32_t(j) * kTileThreads;
            xs[j] = i < m ? __ldg(loc + t0 + i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const uint32_t i = threadIdx.x + uint32_t(j) * kTileThreads;
            bn[j] = 0xFFFFFFFFu;
            if (i < m) {
                if (s_many) {
                    const uint32_t s = flow_shard_of_edge(start, S, t0 + i);
                    const unsigned long long pos = atomicAdd(cursor + uint64_t(s) * nb + seg_bin(xs[j], g, sshift), 1ull);
                    loc_out[pos] = xs[j];
                    if (val) val_out[pos] = __ldg(val + t0 + i);
                } else {
                    bn[j] = (i >= split ? nb : 0u) + seg_bin(xs[j], g, sshift);
                    rk[j] = atomicAdd(&s_cnt[bn[j]], 1u);
                }
            }
        }
        __syncthreads();
        if (!s_many)
            for (uint32_t i = threadIdx.x; i < 2 * nb; i += blockDim.x) {
                const uint32_t c = s_cnt[i];
                const uint32_t s = f + (i >= nb ? 1u : 0u);
                if (c && s < S) s_base[i] = atomicAdd(cursor + uint64_t(s) * nb + (i >= nb ? i - nb : i),
                                                      (unsigned long long)c);
            }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            if (bn[j] == 0xFFFFFFFFu) continue;
            const unsigned long long pos = s_base[bn[j]] + rk[j];
            loc_out[pos] = xs[j];
            if (val) val_out[pos] = __ldg(val + t0 + threadIdx.x + uint32_t(j) * kTileThreads);
        }
        __syncthreads();
    }
}

// ------------------------------------------------- filter de-duplication

// Duplicate local signatures within a shard (a key given twice, Sec. 4.4)
// are identical edges, which never peel: a build with duplicates always leaves
// them unpeeled. After a failed peel the unpeeled edges are inserted into an
// open-addressing table keyed by (shard, local signature); every edge that
// finds its key already present is marked in `drop` (one copy of each group
// survives, Sec. 4.5) and counted, in total and per shard. With `val` (a
// function) a copy whose value differs from the copy already in the table is
// counted in *nconflict instead: if any copy differs from the first one, that
// copy does, so every key given two values is found. Without `claimed` every
// edge is inserted (duplicate count only).
__global__ void __launch_bounds__(kFT) k_find_dups(const uint64_t* __restrict__ loc, const uint32_t* __restrict__ val,
                                                   uint64_t n, const unsigned long long* __restrict__ start,
                                                   uint32_t S, const uint32_t* __restrict__ claimed,
                                                   unsigned long long* __restrict__ table, uint64_t cap,
                                                   uint32_t* __restrict__ drop, unsigned long long* ndrop,
                                                   unsigned long long* __restrict__ per_shard,
                                                   unsigned long long* nconflict) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < n; e += stride) {
        if (claimed && ((__ldg(claimed + (e >> 5)) >> (e & 31u)) & 1u)) continue;
        const uint64_t local = __ldg(loc + e);
        const uint32_t s = flow_shard_of_edge(start, S, e);
        uint64_t h = mix64(local + (uint64_t(s) + 1) * kGolden) & (cap - 1);
        for (uint64_t probe = 0; probe < cap; probe++) {
            const unsigned long long prev = atomicCAS(table + h, 0ull, (unsigned long long)e + 1);
            if (prev == 0) break;  // first copy
            const uint64_t o = prev - 1;
            if (__ldg(loc + o) == local && flow_shard_of_edge(start, S, o) == s) {
                if (val && __ldg(val + o) != __ldg(val + e)) {
                    atomicAdd(nconflict, 1ull);
                    break;
                }
                if (drop) atomicOr(drop + (e >> 5), 1u << (e & 31u));
                atomicAdd(ndrop, 1ull);
                if (per_shard) atomicAdd(per_shard + s, 1ull);
                break;
            }
            h = (h + 1) & (cap - 1);
        }
    }
}

// ------------------------------------------------------------------ launches

static unsigned grid_for(uint64_t work) {
    uint64_t blocks = (work + kFT - 1) / kFT;
    const uint64_t cap = uint64_t(num_sms()) * 8;
    if (blocks > cap) blocks = cap;
    return unsigned(blocks < 1 ? 1 : blocks);
}

// Worker grids: one block of 8 warps per SM. Fewer, fuller warps take fewer
// turns at the shared queue and record counters, whose queueing sets the
// latency of a peeling step.
static unsigned worker_grid() { return unsigned(num_sms()); }
// Assignment polls without hot counters on its path. Fuse graphs are a deep,
// narrow dataflow with two wave fronts per shard: one block per SM for a single
// shard (more blocks only add pollers: 1.16 -> 1.00 ms at 2^20 keys), two when
// sharded; random hypergraphs (shallow, wide) take four.
static unsigned assign_grid(const Geom& g) {
    return unsigned(num_sms()) * (g.regime == kRegimeFuse ? (g.h == 0 ? 1u : 2u) : 4u);
}

cudaError_t launch_incidence32(const uint64_t* loc, uint64_t n, const unsigned long long* start, uint32_t S,
                               const Geom& g, uint32_t* W, uint32_t* err, const uint32_t* drop, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_incidence32<<<grid_for(n), kFT, 0, st>>>(loc, n, start, S, g, W, err, drop);
    return cudaGetLastError();
}

// Shards per peeling batch: the waves of a batch (two per shard, a few
// segments of 4-byte vertex words each) should stay well inside L2. Larger
// batches overlap more shards' waves but miss L2 once their working set grows
// past a few tens of MB, which lengthens every step of the dependency chain.
constexpr uint32_t kBatchHotMB = 16;

static uint32_t shards_per_batch(const FlowArgs& a) {
    if (a.g.regime != kRegimeFuse) return a.S;  // random hypergraphs peel in a few levels, no wave
    const uint64_t seg = uint64_t(1) << a.g.lg_seg;
    const uint64_t hot = 2 * 4 * seg * 4;  // bytes per shard
    const uint64_t k = (uint64_t(kBatchHotMB) << 20) / hot;
    return uint32_t(k < 1 ? 1 : (k > a.S ? a.S : k));
}

uint32_t flow_batches(const FlowArgs& a) {
    const uint32_t per = shards_per_batch(a);
    return (a.S + per - 1) / per;
}

cudaError_t launch_flow_peel(const FlowArgs& a, cudaStream_t st) {
    const uint32_t per = shards_per_batch(a);
    for (uint32_t s0 = 0; s0 < a.S; s0 += per) {
        const uint32_t s1 = s0 + per < a.S ? s0 + per : a.S;
        if (s0 > 0) k_rebase_head<<<1, 1, 0, st>>>(a);
        k_flow_seed<<<grid_for((uint64_t(s1 - s0) * a.g.cells + kSeedPer - 1) / kSeedPer), kFT, 0, st>>>(a, s0, s1);
        if (a.g.k == 4) k_flow_peel<4><<<worker_grid(), kFT, 0, st>>>(a);
        else k_flow_peel<3><<<worker_grid(), kFT, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t words = (uint64_t(a.claimed_bits) + 31) / 32;
    k_count_claims<<<grid_for(words), kFT, 0, st>>>(a, words);
    return cudaGetLastError();
}

cudaError_t launch_flow_assign(const FlowArgs& a, cudaStream_t st) {
    k_final_init<<<grid_for(uint64_t(a.S) * a.g.cells), kFT, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.nrec == 0 || a.rmax == 0) return e;
    if (a.g.k == 4) k_flow_assign<4><<<assign_grid(a.g), kFT, 0, st>>>(a);
    else k_flow_assign<3><<<assign_grid(a.g), kFT, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_segment_order(const uint64_t* loc, const uint32_t* val, uint64_t n,
                                 const unsigned long long* start, uint32_t S, const Geom& g, unsigned long long* counts,
                                 uint64_t* loc_out, uint32_t* val_out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint32_t l = uint32_t(g.span >> g.lg_seg);
    uint32_t sshift = 0;
    while (((l - 1) >> sshift) + 1 > kSegBins) sshift++;
    const uint32_t nb = ((l - 1) >> sshift) + 1;
    const uint64_t nbins = uint64_t(S) * nb;
    cudaError_t e = cudaMemsetAsync(counts, 0, nbins * 8, st);
    if (e != cudaSuccess) return e;
    uint64_t tiles = (n + kTile - 1) / kTile;
    const uint64_t cap = uint64_t(num_sms()) * 4;
    const unsigned grid = unsigned(tiles < cap ? tiles : cap);
    k_seg_count<<<grid, kTileThreads, size_t(2 * nb) * 4, st>>>(loc, n, start, S, g, nb, sshift, counts);
    k_seg_scan<<<1, 1024, 0, st>>>(counts, nbins, start, nb);
    k_seg_scatter<<<grid, kTileThreads, size_t(2 * nb) * 12, st>>>(loc, val, n, start, S, g, nb, sshift, counts,
                                                                    loc_out, val_out);
    return cudaGetLastError();
}

uint64_t segment_order_bins(const Geom& g, uint32_t S) {
    const uint32_t l = uint32_t(g.span >> g.lg_seg);
    uint32_t sshift = 0;
    while (((l - 1) >> sshift) + 1 > kSegBins) sshift++;
    return uint64_t(S) * (((l - 1) >> sshift) + 1);
}

cudaError_t launch_find_dups(const uint64_t* loc, const uint32_t* val, uint64_t n, const unsigned long long* start,
                             uint32_t S, const uint32_t* claimed, unsigned long long* table, uint64_t cap,
                             uint32_t* drop, unsigned long long* ndrop, unsigned long long* per_shard,
                             unsigned long long* nconflict, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_find_dups<<<grid_for(n), kFT, 0, st>>>(loc, val, n, start, S, claimed, table, cap, drop, ndrop, per_shard,
                                             nconflict);
    return cudaGetLastError();
}

}  // namespace vf
