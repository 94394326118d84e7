// Construction kernels of libvfunc (sm_103a):
//   k_hist_*      signature hash + per-shard histogram (Sec. 4: shard = top h bits)
//   k_scatter_*   bucket (local signature, value) by shard (radix scatter)
//   k_accumulate  fuse regime: degree and XOR-of-edge incidence per vertex (Sec. 4.3)
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
// cursor[s] starts at shard_start[s]. SIG: signatures given (byte keys, sig_in)
// instead of hashing the keys. A tile's steps form a dependent chain (loads,
// shared ranks, the global reservation, the writes), so each block loads the
// keys of its next tile before working on the current one: their latency
// overlaps this tile's reservation instead of adding to it.
constexpr int kItems = 4;

template <bool SIG>
__global__ void __launch_bounds__(kThreads) k_scatter(const uint64_t* __restrict__ keys,
                                                      const Sig* __restrict__ sig_in, const void* __restrict__ values,
                                                      uint64_t n, Geom g, unsigned long long* __restrict__ cursor,
                                                      uint64_t* __restrict__ loc_out, uint32_t* __restrict__ val_out,
                                                      uint32_t s_lo, uint32_t s_hi) {
    __shared__ uint32_t cnt[kSmemBinsMax];
    __shared__ unsigned long long base[kSmemBinsMax];
    const uint32_t S = 1u << g.h;
    const bool has_val = values != nullptr;
    const uint64_t tile = uint64_t(kThreads) * kItems;
    const uint64_t stride = uint64_t(gridDim.x) * tile;
    uint64_t nk[kItems];  // the next tile's keys (SIG: its signatures)
    Sig ns[kItems];
    auto fetch = [&](uint64_t t) {
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            const uint64_t i = t + uint64_t(k) * kThreads + threadIdx.x;
            if (i < n) {
                if constexpr (SIG) ns[k] = sig_in[i];
                else nk[k] = __ldg(keys + i);
            }
        }
    };
    uint64_t t0 = blockIdx.x * tile;
    if (t0 < n) fetch(t0);
    for (; t0 < n; t0 += stride) {
        Sig cur[kItems];
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            const uint64_t i = t0 + uint64_t(k) * kThreads + threadIdx.x;
            if (i < n) {
                if constexpr (SIG) cur[k] = ns[k];
                else cur[k] = sig_u64(nk[k], g.kh, g.kl);
            }
        }
        if (t0 + stride < n) fetch(t0 + stride);
        for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        uint64_t loc[kItems];
        uint32_t sh[kItems], rank[kItems], val[kItems];
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            uint64_t i = t0 + uint64_t(k) * kThreads + threadIdx.x;
            sh[k] = 0xFFFFFFFFu;
            if (i < n) {
                const uint32_t shard = uint32_t(shard_of(cur[k], g.h));
                if (shard >= s_lo && shard < s_hi) {  // only the shard group being built
                    sh[k] = shard;
                    loc[k] = local_of(cur[k], g.h);
                    val[k] = has_val ? load_value(values, g.b, i) : 0u;
                    rank[k] = atomicAdd(&cnt[shard], 1u);
                }
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
                                                           uint32_t* __restrict__ val_out, uint32_t s_lo,
                                                           uint32_t s_hi) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        Sig s = sig_in ? sig_in[i] : sig_u64(__ldg(keys + i), g.kh, g.kl);
        const uint32_t shard = uint32_t(shard_of(s, g.h));
        if (shard < s_lo || shard >= s_hi) continue;
        uint64_t pos = atomicAdd(&cursor[shard], 1ull);
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
                                                         Geom g, uint32_t* __restrict__ W, uint32_t* err,
                                                         const uint32_t* __restrict__ drop) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < n; e += stride) {
        if (drop && ((__ldg(drop + (e >> 5)) >> (e & 31u)) & 1u)) continue;  // dropped duplicate
        uint32_t s = shard_of_edge(start, S, e);
        uint32_t el = uint32_t(e - start[s]);
        uint64_t v[4];
        edge_of(g, __ldg(loc + e), v);
        uint64_t base = uint64_t(s) * g.cells;
        const int kk = g.k == 4 ? 4 : 3;
        for (int k = 0; k < kk; k++) {
            uint32_t* w = W + base + v[k];
            uint32_t old = atomicAdd(w, 1u);
            atomicXor(w, el << 5);
            if ((old & 31u) == 31u) atomicOr(err, kErrDegOverflow);
        }
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
                           uint32_t s_lo, uint32_t s_hi, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if ((1u << g.h) <= uint32_t(kSmemBinsMax))
        if (sig_in)
            k_scatter<true><<<stream_grid(n, kItems), kThreads, 0, st>>>(keys_u64, sig_in, values, n, g, cursor,
                                                                         loc_out, val_out, s_lo, s_hi);
        else
            k_scatter<false><<<stream_grid(n, kItems), kThreads, 0, st>>>(keys_u64, sig_in, values, n, g, cursor,
                                                                          loc_out, val_out, s_lo, s_hi);
    else
        k_scatter_wide<<<stream_grid(n), kThreads, 0, st>>>(keys_u64, sig_in, values, n, g, cursor, loc_out,
                                                            val_out, s_lo, s_hi);
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
                              const Geom& g, uint32_t* W, uint32_t* err, const uint32_t* drop, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_accumulate<<<stream_grid(n), kThreads, 0, st>>>(loc, n, start, S, g, W, err, drop);
    return cudaGetLastError();
}

}  // namespace vf
