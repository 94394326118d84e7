// Serialized form of a built structure (libvfunc): a 4096-byte header of
// little-endian fields followed by the data array, and the file I/O of
// resumable builds that checkpoint one shard group at a time (Sec. 6).
//
// Header (byte offset: field):
//   0 magic "VFSTORE1" | 8 u32 version | 12 u32 header bytes (4096)
//   16 u64 data offset (4096) | 24 u64 data bytes | 32 u64 groups total
//   40 u64 groups done | 48 u64 shard-count digest | 56 u64 parameter digest
//   64.. the vf_info fields, u64 / i32 / f64 in declaration order, then
//   u64 dropped duplicates and i32 key kind.
// The data array starts at byte 4096 in the device layout (shard s owns cells
// [s*cells, (s+1)*cells); b in {8,16,32,64}: native little-endian; otherwise a
// bit array with one pad word), so a file can be mapped and used in place.
#include <cstdio>
#include <cstring>
#include <vector>

#include "vf_internal.h"
#include "vfunc.h"

namespace vf {

namespace {

void put_u64(uint8_t* p, uint64_t v) {
    for (int i = 0; i < 8; i++) p[i] = uint8_t(v >> (8 * i));
}
uint64_t get_u64(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v |= uint64_t(p[i]) << (8 * i);
    return v;
}
void put_u32(uint8_t* p, uint32_t v) {
    for (int i = 0; i < 4; i++) p[i] = uint8_t(v >> (8 * i));
}
uint32_t get_u32(const uint8_t* p) {
    uint32_t v = 0;
    for (int i = 0; i < 4; i++) v |= uint32_t(p[i]) << (8 * i);
    return v;
}

const char kMagic[8] = {'V', 'F', 'S', 'T', 'O', 'R', 'E', '1'};
constexpr uint32_t kVersion = 2;  // 2: the arity k follows the key kind

// Sequential field writer / reader over the header.
struct Cursor {
    uint8_t* w = nullptr;
    const uint8_t* r = nullptr;
    size_t off = 64;
    void u64(uint64_t v) { put_u64(w + off, v), off += 8; }
    void i32(int32_t v) { put_u32(w + off, uint32_t(v)), off += 4; }
    void f64(double v) {
        uint64_t x;
        std::memcpy(&x, &v, 8);
        u64(x);
    }
    uint64_t ru64() { return off += 8, get_u64(r + off - 8); }
    int32_t ri32() { return off += 4, int32_t(get_u32(r + off - 4)); }
    double rf64() {
        uint64_t x = ru64();
        double v;
        std::memcpy(&v, &x, 8);
        return v;
    }
};

}  // namespace

void store_encode(const StoreHeader& h, uint8_t* out) {
    std::memset(out, 0, kStoreHeaderBytes);
    std::memcpy(out, kMagic, 8);
    put_u32(out + 8, kVersion);
    put_u32(out + 12, uint32_t(kStoreHeaderBytes));
    put_u64(out + 16, kStoreHeaderBytes);
    put_u64(out + 24, h.info.data_bytes);
    put_u64(out + 32, h.groups_total);
    put_u64(out + 40, h.groups_done);
    put_u64(out + 48, h.counts_digest);
    put_u64(out + 56, h.params_digest);
    Cursor c;
    c.w = out;
    const vf_info& i = h.info;
    c.u64(i.n), c.u64(i.n_eff);
    c.i32(i.kind), c.i32(i.b), c.i32(i.regime), c.i32(i.h), c.i32(i.h_bb), c.i32(i.h_dup);
    c.u64(i.shards), c.u64(i.M), c.f64(i.c), c.i32(i.lg_seg);
    c.u64(i.seg), c.u64(i.l), c.u64(i.T), c.u64(i.cells), c.u64(i.total_cells), c.u64(i.data_bytes);
    c.u64(i.seed), c.i32(i.retries), c.u64(i.peeled), c.u64(i.core), c.u64(i.rounds);
    c.u64(h.dropped), c.i32(h.key_kind);
    c.i32(i.k);
}

static uint64_t data_bytes_of(const vf_info& i) {
    if (i.b == 8 || i.b == 16 || i.b == 32 || i.b == 64) return i.total_cells * uint64_t(i.b / 8);
    return ((i.total_cells * uint64_t(i.b) + 63) / 64 + 1) * 8;
}

bool store_decode(const uint8_t* in, uint64_t avail, StoreHeader& h) {
    if (avail < kStoreHeaderBytes || std::memcmp(in, kMagic, 8) != 0) return false;
    if (get_u32(in + 8) != kVersion || get_u32(in + 12) != kStoreHeaderBytes) return false;
    if (get_u64(in + 16) != kStoreHeaderBytes) return false;
    std::memset(&h, 0, sizeof h);
    h.groups_total = get_u64(in + 32);
    h.groups_done = get_u64(in + 40);
    h.counts_digest = get_u64(in + 48);
    h.params_digest = get_u64(in + 56);
    Cursor c;
    c.r = in;
    vf_info& i = h.info;
    i.n = c.ru64(), i.n_eff = c.ru64();
    i.kind = c.ri32(), i.b = c.ri32(), i.regime = c.ri32(), i.h = c.ri32(), i.h_bb = c.ri32(), i.h_dup = c.ri32();
    i.shards = c.ru64(), i.M = c.ru64(), i.c = c.rf64(), i.lg_seg = c.ri32();
    i.seg = c.ru64(), i.l = c.ru64(), i.T = c.ru64(), i.cells = c.ru64(), i.total_cells = c.ru64();
    i.data_bytes = c.ru64();
    i.seed = c.ru64(), i.retries = c.ri32(), i.peeled = c.ru64(), i.core = c.ru64(), i.rounds = c.ru64();
    h.dropped = c.ru64(), h.key_kind = c.ri32();
    i.k = c.ri32();
    // consistency: a corrupt or foreign file is rejected, never half-used
    if (get_u64(in + 24) != i.data_bytes) return false;
    if (i.kind != VF_FUNC && i.kind != VF_FILTER) return false;
    if (i.b < 1 || i.b > 64 || i.h < 0 || i.h > 40) return false;
    if (i.regime != VF_REGIME_FUSE && i.regime != VF_REGIME_LGE && i.regime != VF_REGIME_MWHC) return false;
    if (i.shards != (uint64_t(1) << i.h) || i.cells == 0 || i.cells >= (uint64_t(1) << 32)) return false;
    if (i.total_cells != i.shards * i.cells || i.data_bytes != data_bytes_of(i)) return false;
    if (i.k != 3 && !(i.k == 4 && i.regime == VF_REGIME_FUSE)) return false;
    if (i.regime == VF_REGIME_FUSE &&
        (i.lg_seg < 0 || i.lg_seg > 31 || i.seg != (uint64_t(1) << i.lg_seg) || i.T != i.l + uint64_t(i.k) - 1 ||
         i.cells != i.T * i.seg))
        return false;
    if (i.regime == VF_REGIME_MWHC && i.cells % 3 != 0) return false;
    if (h.groups_done > h.groups_total || h.groups_total == 0 || h.groups_total > i.shards) return false;
    if (i.n_eff > i.n || h.dropped > i.n) return false;
    return true;
}

// ---------------------------------------------------------------- file I/O

bool file_read_at(std::FILE* f, uint64_t off, void* dst, uint64_t bytes) {
    if (std::fseek(f, long(off), SEEK_SET) != 0) return false;
    return std::fread(dst, 1, bytes, f) == bytes;
}

bool file_write_at(std::FILE* f, uint64_t off, const void* src, uint64_t bytes) {
    if (std::fseek(f, long(off), SEEK_SET) != 0) return false;
    return std::fwrite(src, 1, bytes, f) == bytes;
}

// Device <-> file in bounded host chunks.
cudaError_t file_to_device(std::FILE* f, uint64_t off, uint8_t* dev, uint64_t bytes, bool* io_ok) {
    constexpr uint64_t kChunk = uint64_t(64) << 20;
    std::vector<uint8_t> buf(size_t(bytes < kChunk ? bytes : kChunk));
    *io_ok = true;
    for (uint64_t done = 0; done < bytes;) {
        const uint64_t k = bytes - done < kChunk ? bytes - done : kChunk;
        if (!file_read_at(f, off + done, buf.data(), k)) {
            *io_ok = false;
            return cudaSuccess;
        }
        cudaError_t e = cudaMemcpy(dev + done, buf.data(), k, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        done += k;
    }
    return cudaSuccess;
}

cudaError_t device_to_file(std::FILE* f, uint64_t off, const uint8_t* dev, uint64_t bytes, bool* io_ok) {
    constexpr uint64_t kChunk = uint64_t(64) << 20;
    std::vector<uint8_t> buf(size_t(bytes < kChunk ? bytes : kChunk));
    *io_ok = true;
    for (uint64_t done = 0; done < bytes;) {
        const uint64_t k = bytes - done < kChunk ? bytes - done : kChunk;
        cudaError_t e = cudaMemcpy(buf.data(), dev + done, k, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        if (!file_write_at(f, off + done, buf.data(), k)) {
            *io_ok = false;
            return cudaSuccess;
        }
        done += k;
    }
    return cudaSuccess;
}

}  // namespace vf
