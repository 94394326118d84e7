// Device-side definitions shared by the kernels of libvfunc: signature hash,
// shard and local signature, 3-hyperedge generation, fingerprints, cell access,
// a bounded grid barrier and the per-structure descriptor.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vf {

// Nothing-up-my-sleeve constants (hex digits of pi, golden ratio).
constexpr uint64_t kLaneHi = 0x243F6A8885A308D3ull;
constexpr uint64_t kLaneLo = 0x13198A2E03707344ull;
constexpr uint64_t kEdgeSalt = 0xA4093822299F31D0ull;
constexpr uint64_t kEdgeSalt2 = 0x082EFA98EC4E6C89ull;
constexpr uint64_t kFpSalt = 0x452821E638D01377ull;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

constexpr int kRegimeFuse = 1;
constexpr int kRegimeLge = 2;
constexpr int kRegimeMwhc = 3;

// Status bits written by kernels into a device word.
constexpr uint32_t kErrDegOverflow = 1u << 0;   // a vertex exceeded 31 incident edges
constexpr uint32_t kErrTimeout = 1u << 1;       // a bounded wait gave up
constexpr uint32_t kErrFrontier = 1u << 2;      // frontier or round buffer overflow
constexpr uint32_t kErrCapacity = 1u << 3;      // shard larger than the solver handles
constexpr uint32_t kErrUnsolvable = 1u << 4;    // a shard's system has no solution
constexpr uint32_t kErrLgeSize = 1u << 5;       // LGE shard beyond the solver: active variables or coefficient rows
constexpr uint32_t kErrLevel = 1u << 6;         // asynchronous peel: too many levels (use the round solver)
constexpr uint32_t kErrDupKey = 1u << 7;        // a function was given one key with two different values

// Stafford Mix13, the SplitMix64 output function.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t mulhi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// Everything a kernel needs to map a key to its cells.
struct Geom {
    uint64_t kh, kl;      // lane keys: mix64(seed ^ kLaneHi), mix64(seed ^ kLaneLo)
    uint64_t cells;       // cells per shard
    uint64_t span;        // fuse: l * seg (range of the first vertex); MWHC: vertices per part
    int32_t lg_seg;       // fuse: log2 segment size
    int32_t h;            // shard bits
    int32_t regime;
    int32_t b;
    int32_t kind;         // 0 function, 1 filter
    int32_t fpb;          // filter: bits of the full fingerprint (0: b); a structure wider than 32 bits
    int32_t fps;          //   is built as 32-bit slices, this one holding fingerprint bits [fps, fps + b)
    int32_t k;            // vertices per edge: 3, or 4 (4-uniform fuse graph)
};

// ----------------------------------------------------------------- signatures

struct Sig {
    uint64_t hi, lo;
};

__device__ __forceinline__ Sig sig_u64(uint64_t key, uint64_t kh, uint64_t kl) {
    return Sig{mix64(key + kh), mix64(key ^ kl)};
}

// Little-endian bytes [start, start + nb) of a byte buffer of `total` bytes,
// nb <= 8, zero-padded. Two aligned 8-byte loads when they stay inside the
// buffer, byte loads at its tail.
__device__ __forceinline__ uint64_t load_le(const uint8_t* buf, uint64_t total, uint64_t start, uint32_t nb) {
    uintptr_t addr = reinterpret_cast<uintptr_t>(buf) + start;
    uintptr_t a = addr & ~uintptr_t(7);
    uint32_t sh = uint32_t(addr & 7);
    uint64_t w;
    if (a >= reinterpret_cast<uintptr_t>(buf) && a + 16 <= reinterpret_cast<uintptr_t>(buf) + total) {
        const uint64_t* p = reinterpret_cast<const uint64_t*>(a);
        uint64_t lo = __ldg(p);
        if (sh == 0) {
            w = lo;
        } else {
            uint64_t hi = __ldg(p + 1);
            w = (lo >> (8 * sh)) | (hi << (64 - 8 * sh));
        }
    } else {
        w = 0;
        for (uint32_t j = 0; j < nb; j++) w |= uint64_t(__ldg(buf + start + j)) << (8 * j);
    }
    if (nb < 8) w &= (uint64_t(1) << (8 * nb)) - 1;
    return w;
}

__device__ __forceinline__ Sig sig_bytes(const uint8_t* buf, uint64_t total, uint64_t off, uint64_t len,
                                         uint64_t kh, uint64_t kl) {
    uint64_t a = kh ^ (len * kGolden);
    uint64_t b = kl ^ len;
    uint64_t nw = (len + 7) >> 3;
    for (uint64_t i = 0; i < nw; i++) {
        uint64_t left = len - 8 * i;
        uint64_t w = load_le(buf, total, off + 8 * i, left >= 8 ? 8u : uint32_t(left));
        a = mix64(a ^ w);
        b = mix64(b + w);
    }
    return Sig{mix64(a), mix64(b)};
}

// ------------------------------------------------------- shard, local, edges

// Shard = top h bits of the signature (Sec. 4).
__device__ __forceinline__ uint64_t shard_of(const Sig& s, int h) { return h == 0 ? 0 : s.hi >> (64 - h); }

// Local signature = the 64 bits following the shard bits (subsigning, Sec. 4.4).
__device__ __forceinline__ uint64_t local_of(const Sig& s, int h) {
    return h == 0 ? s.hi : (s.hi << h) | (s.lo >> (64 - h));
}

// Vertices of a key's hyperedge inside its shard (g.k of them, 3 or 4).
//  fuse: first vertex by fixed-point inversion of the local signature over
//  l*seg (monotone), then one vertex in each of the next k-1 segments (the
//  fourth offset of a 4-uniform fuse graph from a second remix);
//  LGE regime: three distinct uniform vertices over the shard's cells.
__device__ __forceinline__ void edge_of(const Geom& g, uint64_t local, uint64_t v[4]) {
    if (g.regime == kRegimeFuse) {
        uint64_t v0 = mulhi(local, g.span);
        uint64_t s = v0 >> g.lg_seg;
        uint64_t r = mix64(local ^ kEdgeSalt);
        uint64_t mask = (g.lg_seg >= 64) ? ~0ull : ((uint64_t(1) << g.lg_seg) - 1);
        v[0] = v0;
        v[1] = ((s + 1) << g.lg_seg) + (r & mask);
        v[2] = ((s + 2) << g.lg_seg) + ((r >> 32) & mask);
        if (g.k == 4) v[3] = ((s + 3) << g.lg_seg) + (mix64(local ^ kEdgeSalt2) & mask);
    } else if (g.regime == kRegimeMwhc) {
        // MWHC (Sec. 4.1, k-partite): one uniform vertex in each third of the shard
        const uint64_t P = g.span;
        v[0] = mulhi(local, P);
        v[1] = P + mulhi(mix64(local ^ kEdgeSalt), P);
        v[2] = 2 * P + mulhi(mix64(local ^ kEdgeSalt2), P);
    } else {
        uint64_t V = g.cells;
        uint64_t r = mix64(local ^ kEdgeSalt);
        uint64_t q = mix64(local ^ kEdgeSalt2);
        uint64_t d1 = 1 + mulhi(r, V - 1);
        uint64_t t = 1 + mulhi(q, V - 2);
        uint64_t d2 = t >= d1 ? t + 1 : t;
        uint64_t v0 = mulhi(local, V);
        uint64_t v1 = v0 + d1;
        uint64_t v2 = v0 + d2;
        v[0] = v0;
        v[1] = v1 >= V ? v1 - V : v1;
        v[2] = v2 >= V ? v2 - V : v2;
    }
}

// Vertex k of a fuse edge whose first vertex lies in segment t - k, as an
// offset from the first cell of segment t: the cell edge_of gives, less
// (t << lg_seg). For k >= 1 the segment is already known, so only the remix
// that places the vertex inside it is computed; for k = 0 the offset is
// v0 - (t << lg_seg), which wraps to a huge value if v0 lies outside segment t.
__device__ __forceinline__ uint64_t fuse_vertex_in_segment(const Geom& g, uint64_t local, uint32_t k, uint64_t t) {
    const uint64_t mask = (uint64_t(1) << g.lg_seg) - 1;
    if (k == 0) return mulhi(local, g.span) - (t << g.lg_seg);
    if (k == 3) return mix64(local ^ kEdgeSalt2) & mask;
    const uint64_t r = mix64(local ^ kEdgeSalt);
    return (k == 1 ? r : r >> 32) & mask;
}

// Filter fingerprint: top b bits of a remix of the local signature (Sec. 4.5).
__device__ __forceinline__ uint64_t fingerprint64(uint64_t local, int b) { return mix64(local ^ kFpSalt) >> (64 - b); }

// Bits [fps, fps + b) of the fpb-bit fingerprint (fpb = 0: b bits, the whole one).
__device__ __forceinline__ uint32_t fingerprint_slice(uint64_t local, int b, int fpb, int fps) {
    const uint64_t s = fingerprint64(local, fpb ? fpb : b) >> fps;
    return b >= 32 ? uint32_t(s) : uint32_t(s) & ((1u << b) - 1u);
}

__device__ __forceinline__ uint32_t fingerprint(uint64_t local, int b) { return fingerprint_slice(local, b, 0, 0); }

// ------------------------------------------------------------------- cells

// Cell i of a b-bit array with 32 < b <= 64 (b = 64 native; otherwise a bit
// array whose last word is followed by a pad word, so reading q + 1 is safe).
__device__ __forceinline__ uint64_t cell_get64(const uint8_t* __restrict__ data, int b, uint64_t i) {
    const uint64_t* w = reinterpret_cast<const uint64_t*>(data);
    if (b == 64) return __ldg(w + i);
    const uint64_t bit = i * uint64_t(b);
    const uint64_t q = bit >> 6;
    const uint32_t o = uint32_t(bit & 63);
    uint64_t x = __ldg(w + q) >> o;
    if (o + b > 64) x |= __ldg(w + q + 1) << (64 - o);
    return x & ((uint64_t(1) << b) - 1);
}

__device__ __forceinline__ bool native_width(int b) { return b == 8 || b == 16 || b == 32; }

// Read cell i (read-only data: non-coherent cache path).
__device__ __forceinline__ uint32_t cell_get_nc(const uint8_t* data, int b, uint64_t i) {
    if (b == 8) return __ldg(data + i);
    if (b == 16) return __ldg(reinterpret_cast<const uint16_t*>(data) + i);
    if (b == 32) return __ldg(reinterpret_cast<const uint32_t*>(data) + i);
    uint64_t bit = i * uint64_t(b);
    const uint64_t* w = reinterpret_cast<const uint64_t*>(data);
    uint64_t q = bit >> 6;
    uint32_t o = uint32_t(bit & 63);
    uint64_t x = __ldg(w + q) >> o;
    if (o + b > 64) x |= __ldg(w + q + 1) << (64 - o);
    return uint32_t(x & ((uint64_t(1) << b) - 1));
}

// Read cell i written earlier in the same kernel by another SM (L2 path).
__device__ __forceinline__ uint32_t cell_get_cg(const uint8_t* data, int b, uint64_t i) {
    if (b == 8) return __ldcg(data + i);
    if (b == 16) return __ldcg(reinterpret_cast<const uint16_t*>(data) + i);
    if (b == 32) return __ldcg(reinterpret_cast<const uint32_t*>(data) + i);
    uint64_t bit = i * uint64_t(b);
    const uint64_t* w = reinterpret_cast<const uint64_t*>(data);
    uint64_t q = bit >> 6;
    uint32_t o = uint32_t(bit & 63);
    uint64_t x = __ldcg(w + q) >> o;
    if (o + b > 64) x |= __ldcg(w + q + 1) << (64 - o);
    return uint32_t(x & ((uint64_t(1) << b) - 1));
}

// Write a value into a cell that is still zero. Bit-packed cells may share a
// 64-bit word with cells written concurrently, hence atomicXor there.
__device__ __forceinline__ void cell_put_zero(uint8_t* data, int b, uint64_t i, uint32_t x) {
    if (b == 8) { data[i] = uint8_t(x); return; }
    if (b == 16) { reinterpret_cast<uint16_t*>(data)[i] = uint16_t(x); return; }
    if (b == 32) { reinterpret_cast<uint32_t*>(data)[i] = x; return; }
    uint64_t bit = i * uint64_t(b);
    unsigned long long* w = reinterpret_cast<unsigned long long*>(data);
    uint64_t q = bit >> 6;
    uint32_t o = uint32_t(bit & 63);
    uint64_t xv = uint64_t(x) & ((uint64_t(1) << b) - 1);
    if (xv == 0) return;
    atomicXor(w + q, (unsigned long long)(xv << o));
    if (o + b > 64) atomicXor(w + q + 1, (unsigned long long)(xv >> (64 - o)));
}

// -------------------------------------------------------- bounded grid barrier

// Grid-wide barrier for cooperative launches (all blocks co-resident). The
// wait is bounded: after ~2^22 polls with back-off it records kErrTimeout in
// *err and returns, so a kernel never spins forever.
struct GridBar {
    unsigned int count;
    unsigned int gen;
};

__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned int nblocks, uint32_t* err) {
    __syncthreads();
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_fail = 0;
        volatile unsigned int* vgen = &bar->gen;
        unsigned int gen = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(&bar->count, 1u);
        if (arrived == nblocks - 1) {
            bar->count = 0;
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            uint32_t polls = 0;
            volatile uint32_t* verr = err;
            while (*vgen == gen) {
                if (*verr & kErrTimeout) {
                    s_fail = 1;
                    break;
                }
                if (++polls > (1u << 22)) {
                    atomicOr(err, kErrTimeout);
                    s_fail = 1;
                    break;
                }
                if (polls > 64) __nanosleep(256);
            }
        }
        __threadfence();
        if (*reinterpret_cast<volatile uint32_t*>(err) & kErrTimeout) s_fail = 1;
    }
    __syncthreads();
    return s_fail == 0;
}

}  // namespace vf
