// Values wider than 32 bits (b = 33..64) in libvfunc. The system of
// eq. (MWHC) is linear over GF(2)^b, one bit plane at a time, so a b-bit
// structure is the pair of a 32-bit slice (bits 0..31 of every value or
// fingerprint) and a (b-32)-bit slice (bits 32..b-1), solved on the same
// hypergraph with the same seed, then packed into one array of b-bit cells
// (b = 64 native, otherwise the bit array of Sec. 5 with one pad word).
#include "vf_internal.h"

namespace vf {

constexpr int kWT = 256;

static unsigned wide_grid(uint64_t work) {
    uint64_t blocks = (work + kWT - 1) / kWT;
    const uint64_t cap = uint64_t(num_sms()) * 8;
    if (blocks > cap) blocks = cap;
    return unsigned(blocks < 1 ? 1 : blocks);
}

// values (u64) -> low 32 bits (u32) and bits 32..b-1 in the narrowest type
// holding b-32 bits (the layout the slice build reads).
__global__ void __launch_bounds__(kWT) k_split64(const uint64_t* __restrict__ v, uint64_t n, int b,
                                                 uint32_t* __restrict__ lo, void* __restrict__ hi) {
    const int hb = b - 32;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t x = __ldg(v + i);
        lo[i] = uint32_t(x);
        const uint32_t h = uint32_t(x >> 32);
        if (hb <= 8) static_cast<uint8_t*>(hi)[i] = uint8_t(h);
        else if (hb <= 16) static_cast<uint16_t*>(hi)[i] = uint16_t(h);
        else static_cast<uint32_t*>(hi)[i] = h;
    }
}

// Output word w of the b-bit array holds bits [64w, 64w + 64): the cells that
// overlap it (at most three for b > 32) are gathered from both slices.
__global__ void __launch_bounds__(kWT) k_pack_wide(const uint32_t* __restrict__ lo, const uint8_t* __restrict__ hi,
                                                   uint64_t cells, int b, uint64_t words,
                                                   uint64_t* __restrict__ out) {
    const int hb = b - 32;
    for (uint64_t w = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; w < words;
         w += uint64_t(gridDim.x) * blockDim.x) {
        uint64_t acc = 0;
        if (b == 64) {
            if (w < cells) acc = uint64_t(__ldg(lo + w)) | (uint64_t(cell_get_nc(hi, hb, w)) << 32);
        } else {
            const uint64_t bit0 = w * 64;
            uint64_t c = bit0 / uint64_t(b);
            for (; c < cells && c * uint64_t(b) < bit0 + 64; c++) {
                const uint64_t v = uint64_t(__ldg(lo + c)) | (uint64_t(cell_get_nc(hi, hb, c)) << 32);
                const int64_t sh = int64_t(c * uint64_t(b)) - int64_t(bit0);
                acc |= sh >= 0 ? v << sh : v >> (-sh);
            }
        }
        out[w] = acc;
    }
}

// Queries of a b-bit structure, b > 32: three 64-bit cell reads, XOR, and the
// 64-bit value or the comparison with the full fingerprint.
__global__ void __launch_bounds__(kWT) k_query_wide(const void* __restrict__ keys, const uint64_t* __restrict__ offs,
                                                    uint64_t m, Geom g, const uint8_t* __restrict__ data,
                                                    void* __restrict__ out) {
    const uint64_t total = offs ? __ldg(offs + m) : 0;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < m; i += uint64_t(gridDim.x) * blockDim.x) {
        Sig s;
        if (offs) {
            const uint64_t o0 = __ldg(offs + i), o1 = __ldg(offs + i + 1);
            s = sig_bytes(static_cast<const uint8_t*>(keys), total, o0, o1 - o0, g.kh, g.kl);
        } else {
            s = sig_u64(__ldg(static_cast<const uint64_t*>(keys) + i), g.kh, g.kl);
        }
        const uint64_t base = shard_of(s, g.h) * g.cells;
        const uint64_t local = local_of(s, g.h);
        uint64_t v[4];
        edge_of(g, local, v);
        uint64_t x = cell_get64(data, g.b, base + v[0]) ^ cell_get64(data, g.b, base + v[1]) ^
                     cell_get64(data, g.b, base + v[2]);
        if (g.k == 4) x ^= cell_get64(data, g.b, base + v[3]);
        if (g.kind == 1) static_cast<uint8_t*>(out)[i] = uint8_t(x == fingerprint64(local, g.b));
        else static_cast<uint64_t*>(out)[i] = x;
    }
}

cudaError_t launch_split64(const uint64_t* v, uint64_t n, int b, uint32_t* lo, void* hi, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_split64<<<wide_grid(n), kWT, 0, st>>>(v, n, b, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_pack_wide(const uint32_t* lo, const uint8_t* hi, uint64_t cells, int b, uint64_t words,
                             uint64_t* out, cudaStream_t st) {
    if (words == 0) return cudaSuccess;
    k_pack_wide<<<wide_grid(words), kWT, 0, st>>>(lo, hi, cells, b, words, out);
    return cudaGetLastError();
}

cudaError_t launch_query_wide(const void* keys, const uint64_t* offs, uint64_t m, const Geom& g, const uint8_t* data,
                              void* out, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    k_query_wide<<<wide_grid(m), kWT, 0, st>>>(keys, offs, m, g, data, out);
    return cudaGetLastError();
}

}  // namespace vf
