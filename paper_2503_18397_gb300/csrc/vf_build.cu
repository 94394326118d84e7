// Construction kernels of libvfunc (sm_103a):
//   k_hist_*      signature hash + per-shard histogram (Sec. 4: shard = top h bits)
//   k_scatter_*   bucket (local signature, value) by shard (radix scatter)
//   k_accumulate  fuse regime: degree and XOR-of-edge incidence per vertex (Sec. 4.3)
//   k_peel        fuse regime: round-synchronous peeling with a bounded grid barrier
//   k_assign      fuse regime: reverse-round value assignment
//   k_sigs_*      signatures only (inspection entry point)
#include "vf_internal.h"

namespace vf {

constexpr int kThreads = 256;
constexpr int kSmemBinsMax = 4096;  // shard histograms up to 2^12 bins live in shared memory

// ------------------------------------------------------------ hash + histogram

__global__ void __launch_bounds__(kThreads) k_hist_u64(const uint64_t* __restrict__ keys, uint64_t n, Geom g,
                                                       uint32_t* __restrict__ hist) {
    __shared__ uint32_t sh[kSmemBinsMax];
    const uint32_t S = 1u << g.h;
    const bool in_smem = S <= kSmemBinsMax;
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        uint32_t s0 = uint32_t(shard_of(sig_u64(__ldg(keys + i), g.kh, g.kl), g.h));
        if (in_smem) atomicAdd(&sh[s0], 1u); else atomicAdd(&hist[s0], 1u);
    }
    __syncthreads();
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Byte-string keys: hash once, keep the signature for the scatter pass.
__global__ void __launch_bounds__(kThreads) k_hist_bytes(const uint8_t* __restrict__ buf,
                                                         const uint64_t* __restrict__ offs, uint64_t n, Geom g,
                                                         uint32_t* __restrict__ hist, Sig* __restrict__ sig_out) {
    __shared__ uint32_t sh[kSmemBinsMax];
    const uint32_t S = 1u << g.h;
    const bool in_smem = S <= kSmemBinsMax;
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t total = __ldg(offs + n);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        uint64_t o0 = __ldg(offs + i), o1 = __ldg(offs + i + 1);
        Sig s = sig_bytes(buf, total, o0, o1 - o0, g.kh, g.kl);
        sig_out[i] = s;
        uint32_t b = uint32_t(shard_of(s, g.h));
        if (in_smem) atomicAdd(&sh[b], 1u); else atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// ------------------------------------------------------------- radix scatter

__device__ __forceinline__ uint32_t load_value(const void* values, int b, uint64_t i) {
    uint32_t v;
    if (b <= 8) v = __ldg(reinterpret_cast<const uint8_t*>(values) + i);
    else if (b <= 16) v = __ldg(reinterpret_cast<const uint16_t*>(values) + i);
    else v = __ldg(reinterpret_cast<const uint32_t*>(values) + i);
    return b == 32 ? v : (v & ((1u << b) - 1u));
}

// Each block takes tiles of kThreads*kItems keys, counts the tile's keys per
// shard in shared memory, reserves one contiguous range per (tile, shard) with
// a single global atomic, and writes each key into its range.
// cursor[s] starts at shard_start[s]. sig_in (byte keys) replaces hashing.
constexpr int kItems = 4;

__global__ void __launch_bounds__(kThreads) k_scatter(const uint64_t* __restrict__ keys,
                                                      const Sig* __restrict__ sig_in, const void* __restrict__ values,
                                                      uint64_t n, Geom g, unsigned long long* __restrict__ cursor,
                                                      uint64_t* __restrict__ loc_out, uint32_t* __restrict__ val_out) {
    __shared__ uint32_t cnt[kSmemBinsMax];
    __shared__ unsigned long long base[kSmemBinsMax];
    const uint32_t S = 1u << g.h;
    const bool has_val = values != nullptr;
    const uint64_t tile = uint64_t(kThreads) * kItems;
    for (uint64_t t0 = blockIdx.x * tile; t0 < n; t0 += uint64_t(gridDim.x) * tile) {
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        uint64_t loc[kItems];
        uint32_t sh[kItems], rank[kItems], val[kItems];
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            uint64_t i = t0 + uint64_t(k) * kThreads + threadIdx.x;
            sh[k] = 0xFFFFFFFFu;
            if (i < n) {
                Sig s = sig_in ? sig_in[i] : sig_u64(__ldg(keys + i), g.kh, g.kl);
                sh[k] = uint32_t(shard_of(s, g.h));
                loc[k] = local_of(s, g.h);
                val[k] = has_val ? load_value(values, g.b, i) : 0u;
                rank[k] = atomicAdd(&cnt[sh[k]], 1u);
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x)
            if (cnt[i]) base[i] = atomicAdd(&cursor[i], (unsigned long long)cnt[i]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            if (sh[k] != 0xFFFFFFFFu) {
                uint64_t pos = base[sh[k]] + rank[k];
                loc_out[pos] = loc[k];
                if (has_val) val_out[pos] = val[k];
            }
        }
        __syncthreads();
    }
}

// Many shards (h > 12): one global atomic per key.
__global__ void __launch_bounds__(kThreads) k_scatter_wide(const uint64_t* __restrict__ keys,
                                                           const Sig* __restrict__ sig_in,
                                                           const void* __restrict__ values, uint64_t n, Geom g,
                                                           unsigned long long* __restrict__ cursor,
                                                           uint64_t* __restrict__ loc_out,
                                                           uint32_t* __restrict__ val_out) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        Sig s = sig_in ? sig_in[i] : sig_u64(__ldg(keys + i), g.kh, g.kl);
        uint64_t pos = atomicAdd(&cursor[shard_of(s, g.h)], 1ull);
        loc_out[pos] = local_of(s, g.h);
        if (values) val_out[pos] = load_value(values, g.b, i);
    }
}

// ---------------------------------------------------------------- signatures

__global__ void k_sigs_u64(const uint64_t* __restrict__ keys, uint64_t n, uint64_t kh, uint64_t kl,
                           Sig* __restrict__ out) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride)
        out[i] = sig_u64(__ldg(keys + i), kh, kl);
}

__global__ void k_sigs_bytes(const uint8_t* __restrict__ buf, const uint64_t* __restrict__ offs, uint64_t n,
                             uint64_t kh, uint64_t kl, Sig* __restrict__ out) {
    const uint64_t total = __ldg(offs + n);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        uint64_t o0 = __ldg(offs + i), o1 = __ldg(offs + i + 1);
        out[i] = sig_bytes(buf, total, o0, o1 - o0, kh, kl);
    }
}

// --------------------------------------------------- fuse regime: incidence

// Shard of bucketed edge e: binary search over shard_start[0..S].
__device__ __forceinline__ uint32_t shard_of_edge(const unsigned long long* __restrict__ start, uint32_t S,
                                                  uint64_t e) {
    uint32_t lo = 0, hi = S;  // invariant: start[lo] <= e < start[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Vertex word: bits 0..4 degree (<= 31), bits 5..31 XOR of incident shard-local
// edge indices (Sec. 4.3, XOR trick). Degree overflow is reported, not wrapped.
__global__ void __launch_bounds__(kThreads) k_accumulate(const uint64_t* __restrict__ loc, uint64_t n,
                                                         const unsigned long long* __restrict__ start, uint32_t S,
                                                         Geom g, uint32_t* __restrict__ W, uint32_t* err) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < n; e += stride) {
        uint32_t s = shard_of_edge(start, S, e);
        uint32_t el = uint32_t(e - start[s]);
        uint64_t v[3];
        edge_of(g, __ldg(loc + e), v);
        uint64_t base = uint64_t(s) * g.cells;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t* w = W + base + v[k];
            uint32_t old = atomicAdd(w, 1u);
            atomicXor(w, el << 5);
            if ((old & 31u) == 31u) atomicOr(err, kErrDegOverflow);
        }
    }
}

// ------------------------------------------------------------ fuse regime: peel

struct PeelArgs {
    const uint64_t* loc;
    const unsigned long long* start;  // S+1 shard starts in the bucketed arrays
    uint32_t S;
    Geom g;
    uint32_t* W;                      // S*cells vertex words
    uint32_t* claimed;                // one bit per edge
    uint32_t* front[2];               // frontier buffers (global vertex ids)
    uint64_t front_cap;
    uint32_t* order;                  // peeled edges: (edge << 2) | side
    uint32_t* round_off;              // round r occupies order[round_off[r] .. round_off[r+1])
    uint32_t round_cap;
    uint32_t* ctr;                    // [0],[1] frontier sizes, [2] order count, [3] rounds
    GridBar* bar;
    uint32_t* err;
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Warp-aggregated append of `want` items; returns each lane's first slot.
__device__ __forceinline__ uint32_t warp_append(uint32_t* ctr, uint32_t want) {
    const unsigned lane = lane_id();
    uint32_t incl = want;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= unsigned(d)) incl += y;
    }
    uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + incl - want;
}

// Grid barrier whose last arriving block closes round r: records where the
// next round's peeled edges start, clears the frontier just consumed, and
// counts the round. Everything it touches is quiescent at that point.
__device__ bool peel_barrier(const PeelArgs& a, unsigned nblocks, uint32_t r) {
    __syncthreads();
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_fail = 0;
        volatile unsigned* vgen = &a.bar->gen;
        volatile uint32_t* verr = a.err;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(&a.bar->count, 1u);
        if (arrived == nblocks - 1) {
            uint32_t nr = r + 1;
            if (nr < a.round_cap) a.round_off[nr] = *reinterpret_cast<volatile uint32_t*>(&a.ctr[2]);
            else atomicOr(a.err, kErrFrontier);
            a.ctr[r & 1] = 0;
            a.ctr[3] = nr;
            a.bar->count = 0;
            __threadfence();
            atomicAdd(&a.bar->gen, 1u);
        } else {
            uint32_t polls = 0;
            while (*vgen == gen) {
                if (*verr & kErrTimeout) break;
                if (++polls > (1u << 22)) {
                    atomicOr(a.err, kErrTimeout);
                    break;
                }
                if (polls > 64) __nanosleep(256);
            }
        }
        __threadfence();
        if (*verr & (kErrTimeout | kErrFrontier)) s_fail = 1;
    }
    __syncthreads();
    return s_fail == 0;
}

__global__ void __launch_bounds__(kThreads) k_peel(PeelArgs a) {
    const unsigned nblocks = gridDim.x;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t V = uint64_t(a.S) * a.g.cells;
    const uint64_t warp0 = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u);
    const unsigned lane = lane_id();

    // Round 0 frontier: every vertex of degree one.
    for (uint64_t v0 = warp0; v0 < V; v0 += nthreads) {
        uint64_t v = v0 + lane;
        bool one = v < V && (__ldcg(a.W + v) & 31u) == 1u;
        uint32_t slot = warp_append(&a.ctr[0], one ? 1u : 0u);
        if (one) {
            if (slot < a.front_cap) a.front[0][slot] = uint32_t(v);
            else atomicOr(a.err, kErrFrontier);
        }
    }
    // r = 0xFFFFFFFF closes the initialisation "round": it clears ctr[1] and
    // leaves round_off[0] (zeroed by the host) in place.
    if (!peel_barrier(a, nblocks, 0xFFFFFFFFu)) return;

    for (uint32_t r = 0;; r++) {
        const uint32_t cur = r & 1, nxt = cur ^ 1;
        const uint32_t sz = *reinterpret_cast<volatile uint32_t*>(&a.ctr[cur]);
        if (sz == 0) break;
        const uint32_t* F = a.front[cur];
        uint32_t* G = a.front[nxt];
        for (uint64_t i0 = warp0; i0 < sz; i0 += nthreads) {
            uint64_t i = i0 + lane;
            bool peel = false;
            uint32_t e = 0, side = 0, el = 0;
            uint32_t other[2] = {0, 0};
            bool push[2] = {false, false};
            if (i < sz) {
                uint32_t v = __ldcg(F + i);
                uint32_t w = __ldcg(a.W + v);
                if ((w & 31u) == 1u) {
                    uint32_t s = uint32_t(uint64_t(v) / a.g.cells);
                    el = w >> 5;
                    e = uint32_t(a.start[s] + el);
                    uint64_t local = __ldg(a.loc + e);
                    uint32_t bit = 1u << (e & 31u);
                    uint32_t prev = atomicOr(a.claimed + (e >> 5), bit);
                    if (!(prev & bit)) {
                        peel = true;
                        uint64_t vv[3];
                        edge_of(a.g, local, vv);
                        uint64_t base = uint64_t(s) * a.g.cells;
                        uint32_t lv = uint32_t(v - base);
                        side = (vv[0] == lv) ? 0u : (vv[1] == lv) ? 1u : 2u;
                        int o = 0;
#pragma unroll
                        for (int k = 0; k < 3; k++)
                            if (uint32_t(k) != side) other[o++] = uint32_t(base + vv[k]);
#pragma unroll
                        for (int k = 0; k < 2; k++) {
                            uint32_t* wp = a.W + other[k];
                            uint32_t old = __ldcg(wp);
                            for (;;) {
                                uint32_t nw = ((old ^ (el << 5)) & ~31u) | ((old & 31u) - 1u);
                                uint32_t got = atomicCAS(wp, old, nw);
                                if (got == old) {
                                    push[k] = (nw & 31u) == 1u;
                                    break;
                                }
                                old = got;
                            }
                        }
                    }
                }
            }
            uint32_t slot = warp_append(&a.ctr[2], peel ? 1u : 0u);
            if (peel) a.order[slot] = (e << 2) | side;
            uint32_t np = uint32_t(push[0]) + uint32_t(push[1]);
            uint32_t fs = warp_append(&a.ctr[nxt], np);
            if (np) {
                if (fs + np <= a.front_cap) {
                    int q = 0;
                    if (push[0]) G[fs + q++] = other[0];
                    if (push[1]) G[fs + q] = other[1];
                } else {
                    atomicOr(a.err, kErrFrontier);
                }
            }
        }
        if (!peel_barrier(a, nblocks, r)) return;
    }
}

// ------------------------------------------------------- fuse regime: assign

struct AssignArgs {
    const uint64_t* loc;
    const uint32_t* val;              // NULL for a filter (fingerprints instead)
    const unsigned long long* start;
    uint32_t S;
    Geom g;
    const uint32_t* order;
    const uint32_t* round_off;
    uint32_t rounds;
    uint8_t* data;
    GridBar* bar;
    uint32_t* err;
};

// Rounds in reverse peel order. An edge peeled in round r from vertex v has
// its other two vertices either never peeled or peeled in a later round, so
// they are final when round r is assigned, and no two edges of one round
// write the same cell (Sec. 4.3: assignment pops E in reverse).
__global__ void __launch_bounds__(kThreads) k_assign(AssignArgs a) {
    const unsigned nblocks = gridDim.x;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
    for (uint32_t r = a.rounds; r-- > 0;) {
        const uint32_t lo = __ldg(a.round_off + r), hi = __ldg(a.round_off + r + 1);
        for (uint64_t i = lo + tid; i < hi; i += nthreads) {
            uint32_t ent = __ldg(a.order + i);
            uint32_t e = ent >> 2, side = ent & 3u;
            uint32_t s = shard_of_edge(a.start, a.S, e);
            uint64_t local = __ldg(a.loc + e);
            uint64_t vv[3];
            edge_of(a.g, local, vv);
            uint64_t base = uint64_t(s) * a.g.cells;
            uint32_t x = a.val ? __ldg(a.val + e) : fingerprint(local, a.g.b);
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (uint32_t(k) != side) x ^= cell_get_cg(a.data, a.g.b, base + vv[k]);
            cell_put_zero(a.data, a.g.b, base + vv[side], x);
        }
        if (r > 0 && !grid_sync(a.bar, nblocks, a.err)) return;
    }
}

// ------------------------------------------------------------------ launchers

static int g_num_sms = 0;

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

static unsigned stream_grid(uint64_t work, int per_thread = 1) {
    uint64_t blocks = (work + uint64_t(kThreads) * per_thread - 1) / (uint64_t(kThreads) * per_thread);
    uint64_t cap = uint64_t(num_sms()) * 8;
    if (blocks > cap) blocks = cap;
    return unsigned(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_hist(int key_kind, const void* keys, const uint64_t* offs, uint64_t n, const Geom& g,
                        uint32_t* hist, Sig* sig_out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (key_kind == 0)
        k_hist_u64<<<stream_grid(n), kThreads, 0, st>>>(static_cast<const uint64_t*>(keys), n, g, hist);
    else
        k_hist_bytes<<<stream_grid(n), kThreads, 0, st>>>(static_cast<const uint8_t*>(keys), offs, n, g, hist,
                                                          sig_out);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const uint64_t* keys_u64, const Sig* sig_in, const void* values, uint64_t n,
                           const Geom& g, unsigned long long* cursor, uint64_t* loc_out, uint32_t* val_out,
                           cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if ((1u << g.h) <= uint32_t(kSmemBinsMax))
        k_scatter<<<stream_grid(n, kItems), kThreads, 0, st>>>(keys_u64, sig_in, values, n, g, cursor, loc_out,
                                                               val_out);
    else
        k_scatter_wide<<<stream_grid(n), kThreads, 0, st>>>(keys_u64, sig_in, values, n, g, cursor, loc_out,
                                                            val_out);
    return cudaGetLastError();
}

cudaError_t launch_sigs(int key_kind, const void* keys, const uint64_t* offs, uint64_t n, uint64_t kh,
                        uint64_t kl, Sig* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (key_kind == 0)
        k_sigs_u64<<<stream_grid(n), kThreads, 0, st>>>(static_cast<const uint64_t*>(keys), n, kh, kl, out);
    else
        k_sigs_bytes<<<stream_grid(n), kThreads, 0, st>>>(static_cast<const uint8_t*>(keys), offs, n, kh, kl, out);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const uint64_t* loc, uint64_t n, const unsigned long long* start, uint32_t S,
                              const Geom& g, uint32_t* W, uint32_t* err, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_accumulate<<<stream_grid(n), kThreads, 0, st>>>(loc, n, start, S, g, W, err);
    return cudaGetLastError();
}

static unsigned coop_grid(const void* fn) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return unsigned(per_sm) * unsigned(num_sms());
}

cudaError_t launch_peel(const FusePeelBuffers& b, const Geom& g, cudaStream_t st) {
    PeelArgs a;
    a.loc = b.loc;
    a.start = b.start;
    a.S = b.S;
    a.g = g;
    a.W = b.W;
    a.claimed = b.claimed;
    a.front[0] = b.front0;
    a.front[1] = b.front1;
    a.front_cap = b.front_cap;
    a.order = b.order;
    a.round_off = b.round_off;
    a.round_cap = b.round_cap;
    a.ctr = b.ctr;
    a.bar = b.bar;
    a.err = b.err;
    void* args[] = {&a};
    unsigned grid = coop_grid(reinterpret_cast<const void*>(k_peel));
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_peel), dim3(grid), dim3(kThreads), args, 0,
                                       st);
}

cudaError_t launch_assign(const FusePeelBuffers& b, const uint32_t* val, const Geom& g, uint32_t rounds,
                          uint8_t* data, cudaStream_t st) {
    if (rounds == 0) return cudaSuccess;
    AssignArgs a;
    a.loc = b.loc;
    a.val = val;
    a.start = b.start;
    a.S = b.S;
    a.g = g;
    a.order = b.order;
    a.round_off = b.round_off;
    a.rounds = rounds;
    a.data = data;
    a.bar = b.bar;
    a.err = b.err;
    void* args[] = {&a};
    unsigned grid = coop_grid(reinterpret_cast<const void*>(k_assign));
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_assign), dim3(grid), dim3(kThreads), args,
                                       0, st);
}

}  // namespace vf
