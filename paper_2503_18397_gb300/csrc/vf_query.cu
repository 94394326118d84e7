// Query kernel of libvfunc (sm_103a): signature -> shard (top h bits) ->
// cell offset shard*cells (no offset array, Sec. 4) -> three cells -> XOR
// (eq. MWHC, k = 3) -> [filter: compare with the fingerprint].
//
// Each thread takes kQ keys spaced one grid-stride apart (coalesced key loads)
// and issues all 3*kQ cell loads before using any, so every warp keeps 96
// independent random 32-byte sector reads in flight.
#include "vf_internal.h"

namespace vf {

constexpr int kQThreads = 256;
constexpr int kQ = 4;

template <int WIDTH>
__device__ __forceinline__ uint32_t cell_q(const uint8_t* data, int b, uint64_t i) {
    if constexpr (WIDTH == 8) return __ldg(data + i);
    else if constexpr (WIDTH == 16) return __ldg(reinterpret_cast<const uint16_t*>(data) + i);
    else if constexpr (WIDTH == 32) return __ldg(reinterpret_cast<const uint32_t*>(data) + i);
    else return cell_get_nc(data, b, i);
}

// K: vertices per edge (3, or 4 for a 4-uniform fuse graph).
template <int WIDTH, bool FILTER, bool BYTES, int K>
__global__ void __launch_bounds__(kQThreads) k_query(const void* __restrict__ keys, const uint64_t* __restrict__ offs,
                                                     uint64_t m, Geom g, const uint8_t* __restrict__ data,
                                                     void* __restrict__ out) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t total = BYTES ? __ldg(offs + m) : 0;
    for (uint64_t i0 = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i0 < m; i0 += stride * kQ) {
        uint64_t idx[kQ], loc[kQ], cell[kQ][K];
        bool ok[kQ];
#pragma unroll
        for (int k = 0; k < kQ; k++) {
            idx[k] = i0 + uint64_t(k) * stride;
            ok[k] = idx[k] < m;
            Sig s{0, 0};
            if (ok[k]) {
                if constexpr (BYTES) {
                    uint64_t o0 = __ldg(offs + idx[k]), o1 = __ldg(offs + idx[k] + 1);
                    s = sig_bytes(static_cast<const uint8_t*>(keys), total, o0, o1 - o0, g.kh, g.kl);
                } else {
                    // keys are read once: evict-first, so the cells they probe stay in L2
                    s = sig_u64(__ldcs(static_cast<const uint64_t*>(keys) + idx[k]), g.kh, g.kl);
                }
            }
            uint64_t base = shard_of(s, g.h) * g.cells;
            loc[k] = local_of(s, g.h);
            uint64_t v[4];
            edge_of(g, loc[k], v);
#pragma unroll
            for (int j = 0; j < K; j++) cell[k][j] = base + v[j];
        }
        uint32_t x[kQ][K];
#pragma unroll
        for (int k = 0; k < kQ; k++)
#pragma unroll
            for (int j = 0; j < K; j++) x[k][j] = ok[k] ? cell_q<WIDTH>(data, g.b, cell[k][j]) : 0u;
#pragma unroll
        for (int k = 0; k < kQ; k++) {
            if (!ok[k]) continue;
            uint32_t r = x[k][0] ^ x[k][1] ^ x[k][2];
            if constexpr (K == 4) r ^= x[k][3];
            if constexpr (FILTER) {
                static_cast<uint8_t*>(out)[idx[k]] = uint8_t(r == fingerprint(loc[k], g.b));
            } else {
                if (g.b <= 8) static_cast<uint8_t*>(out)[idx[k]] = uint8_t(r);
                else if (g.b <= 16) static_cast<uint16_t*>(out)[idx[k]] = uint16_t(r);
                else static_cast<uint32_t*>(out)[idx[k]] = r;
            }
        }
    }
}

template <int WIDTH, bool FILTER>
static void launch_q(bool bytes, const void* keys, const uint64_t* offs, uint64_t m, const Geom& g,
                     const uint8_t* data, void* out, cudaStream_t st) {
    uint64_t blocks = (m + uint64_t(kQThreads) * kQ - 1) / (uint64_t(kQThreads) * kQ);
    uint64_t cap = uint64_t(num_sms()) * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (g.k == 4) {
        if (bytes)
            k_query<WIDTH, FILTER, true, 4><<<unsigned(blocks), kQThreads, 0, st>>>(keys, offs, m, g, data, out);
        else
            k_query<WIDTH, FILTER, false, 4><<<unsigned(blocks), kQThreads, 0, st>>>(keys, offs, m, g, data, out);
    } else if (bytes) {
        k_query<WIDTH, FILTER, true, 3><<<unsigned(blocks), kQThreads, 0, st>>>(keys, offs, m, g, data, out);
    } else {
        k_query<WIDTH, FILTER, false, 3><<<unsigned(blocks), kQThreads, 0, st>>>(keys, offs, m, g, data, out);
    }
}

template <bool FILTER>
static void launch_w(bool bytes, const void* keys, const uint64_t* offs, uint64_t m, const Geom& g,
                     const uint8_t* data, void* out, cudaStream_t st) {
    switch (g.b) {
        case 8: launch_q<8, FILTER>(bytes, keys, offs, m, g, data, out, st); break;
        case 16: launch_q<16, FILTER>(bytes, keys, offs, m, g, data, out, st); break;
        case 32: launch_q<32, FILTER>(bytes, keys, offs, m, g, data, out, st); break;
        default: launch_q<0, FILTER>(bytes, keys, offs, m, g, data, out, st); break;
    }
}

// ------------------------------------------------------- cross-structure batch

constexpr int kReqCache = 4096;

// Requests against many resident structures in one launch: request r owns
// keys [key_off, key_off + m) of the launch's key space. Neighbouring keys of a
// warp mostly share a request, so descriptor reads are broadcasts.
__global__ void __launch_bounds__(kQThreads) k_query_batch(const QueryReq* __restrict__ reqs, uint32_t count,
                                                           uint64_t total) {
    __shared__ uint64_t s_off[kReqCache];
    const bool cached = count <= kReqCache;
    if (cached)
        for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) s_off[i] = reqs[i].key_off;
    __syncthreads();
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < total; g += stride) {
        uint32_t lo = 0, hi = count;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            const uint64_t o = cached ? s_off[mid] : reqs[mid].key_off;
            if (o <= g) lo = mid; else hi = mid;
        }
        const QueryReq& r = reqs[lo];
        const uint64_t i = g - r.key_off;
        const Sig s = sig_u64(__ldg(r.keys + i), r.g.kh, r.g.kl);
        const uint64_t base = shard_of(s, r.g.h) * r.g.cells;
        const uint64_t local = local_of(s, r.g.h);
        uint64_t v[4];
        edge_of(r.g, local, v);
        if (r.g.b > 32) {  // values wider than 32 bits
            uint64_t y = cell_get64(r.data, r.g.b, base + v[0]) ^ cell_get64(r.data, r.g.b, base + v[1]) ^
                         cell_get64(r.data, r.g.b, base + v[2]);
            if (r.g.k == 4) y ^= cell_get64(r.data, r.g.b, base + v[3]);
            if (r.g.kind == 1) static_cast<uint8_t*>(r.out)[i] = uint8_t(y == fingerprint64(local, r.g.b));
            else static_cast<uint64_t*>(r.out)[i] = y;
            continue;
        }
        uint32_t x = cell_get_nc(r.data, r.g.b, base + v[0]) ^ cell_get_nc(r.data, r.g.b, base + v[1]) ^
                     cell_get_nc(r.data, r.g.b, base + v[2]);
        if (r.g.k == 4) x ^= cell_get_nc(r.data, r.g.b, base + v[3]);
        if (r.g.kind == 1) static_cast<uint8_t*>(r.out)[i] = uint8_t(x == fingerprint(local, r.g.b));
        else if (r.g.b <= 8) static_cast<uint8_t*>(r.out)[i] = uint8_t(x);
        else if (r.g.b <= 16) static_cast<uint16_t*>(r.out)[i] = uint16_t(x);
        else static_cast<uint32_t*>(r.out)[i] = x;
    }
}

cudaError_t launch_query_batch(const QueryReq* reqs, uint32_t count, uint64_t total, cudaStream_t st) {
    if (total == 0 || count == 0) return cudaSuccess;
    uint64_t blocks = (total + kQThreads - 1) / kQThreads;
    const uint64_t cap = uint64_t(num_sms()) * 16;
    if (blocks > cap) blocks = cap;
    k_query_batch<<<unsigned(blocks < 1 ? 1 : blocks), kQThreads, 0, st>>>(reqs, count, total);
    return cudaGetLastError();
}

cudaError_t launch_query(int key_kind, const void* keys, const uint64_t* offs, uint64_t m, const Geom& g,
                         const uint8_t* data, void* out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    bool bytes = key_kind != 0;
    if (g.b > 32) return launch_query_wide(keys, bytes ? offs : nullptr, m, g, data, out, st);
    if (g.kind == 1) launch_w<true>(bytes, keys, offs, m, g, data, out, st);
    else launch_w<false>(bytes, keys, offs, m, g, data, out, st);
    return cudaGetLastError();
}

}  // namespace vf
