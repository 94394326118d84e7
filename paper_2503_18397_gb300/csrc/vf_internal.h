// Internal declarations shared by the translation units of libvfunc.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "vf_device.cuh"
#include "vfunc.h"

// A built structure (opaque in the C ABI).
struct vf_struct {
    vf_info info;
    vf::Geom geom;
    uint8_t* data;  // device, info.data_bytes (+ padding)
    int device;
};

namespace vf {

// Geometry kernels need for a structure described by `in`.
Geom geom_of(const vf_info& in);

// ---- serialized form (csrc/vf_store.cu)
constexpr uint64_t kStoreHeaderBytes = 4096;
struct StoreHeader {
    vf_info info;
    uint64_t groups_total, groups_done;  // shard groups of the build; done == total: complete
    uint64_t counts_digest;              // digest of the per-shard key counts
    uint64_t params_digest;              // digest of the parameters that shape the structure
    uint64_t dropped;                    // duplicate filter keys dropped so far
    int32_t key_kind;
};
void store_encode(const StoreHeader& h, uint8_t* out);  // out: kStoreHeaderBytes
bool store_decode(const uint8_t* in, uint64_t avail, StoreHeader& h);
bool file_read_at(std::FILE* f, uint64_t off, void* dst, uint64_t bytes);
bool file_write_at(std::FILE* f, uint64_t off, const void* src, uint64_t bytes);
cudaError_t file_to_device(std::FILE* f, uint64_t off, uint8_t* dev, uint64_t bytes, bool* io_ok);
cudaError_t device_to_file(std::FILE* f, uint64_t off, const uint8_t* dev, uint64_t bytes, bool* io_ok);

int num_sms();

// Where a caller's pointer lives: host memory (or unknown to CUDA), device or
// managed memory the current device can use, or device memory of another
// device (which the kernels here cannot read without peer access).
enum class MemWhere { kHost, kHere, kElsewhere };
MemWhere mem_where(const void* p);
// VF_EINVAL (with a message naming `what`) if p is device memory of another device.
vf_status check_here(const void* p, const char* what);
// Failure-injection hook of vf_debug_faults: attempts below this count fail.
int debug_fail_attempts();

// Message returned by vf_last_error() on the calling thread.
void set_last_error(const char* msg);

// Two-level grid barrier state (zeroed before each cooperative launch).
struct Bar2 {
    unsigned int count;
    unsigned int gen;
    unsigned int grp[64];
};

// Fuse-regime (global-memory) solver of one attempt: peeling and assignment.
struct FuseSolveArgs {
    const uint64_t* loc;              // bucketed local signatures
    const uint32_t* val;              // bucketed values, NULL for a filter
    const unsigned long long* start;  // S+1 shard starts
    uint32_t S;
    Geom g;
    uint32_t* W;                      // S*cells vertex words
    uint32_t* claimed;                // one bit per edge
    uint64_t claimed_bits;            // edges
    uint2* front[2];                  // frontier entries (vertex, edge)
    uint64_t front_cap;
    uint4* rec;                       // assignment records, one per peeled edge
    uint32_t* rec3;                   // 4-uniform: each record's third other vertex (NULL when k = 3)
    uint32_t* round_off;              // round r's records: rec[round_off[r] .. round_off[r+1])
    uint32_t round_cap;
    uint32_t* ctr;                    // [0],[1] frontier sizes, [2] records, [3] rounds
    Bar2* bar;
    uint32_t* err;
    uint8_t* data;                    // assignment target
    uint64_t cell_base;               // cell of the first vertex (shard groups)
    uint32_t rounds;                  // assignment: rounds recorded by the peel
};

cudaError_t launch_hist(int key_kind, const void* keys, const uint64_t* offs, uint64_t n, const Geom& g,
                        uint32_t* hist, Sig* sig_out, cudaStream_t st);
// Buckets the keys whose shard lies in [s_lo, s_hi) (a shard group).
cudaError_t launch_scatter(const uint64_t* keys_u64, const Sig* sig_in, const void* values, uint64_t n,
                           const Geom& g, unsigned long long* cursor, uint64_t* loc_out, uint32_t* val_out,
                           uint32_t s_lo, uint32_t s_hi, cudaStream_t st);
cudaError_t launch_sigs(int key_kind, const void* keys, const uint64_t* offs, uint64_t n, uint64_t kh,
                        uint64_t kl, Sig* out, cudaStream_t st);
// drop: optional bitmap of edges to leave out (duplicate filter keys).
cudaError_t launch_accumulate(const uint64_t* loc, uint64_t n, const unsigned long long* start, uint32_t S,
                              const Geom& g, uint32_t* W, uint32_t* err, const uint32_t* drop, cudaStream_t st);
cudaError_t launch_peel(FuseSolveArgs a, cudaStream_t st);
cudaError_t launch_assign(FuseSolveArgs a, cudaStream_t st);

// Fuse-regime asynchronous solver: worklist peeling that records the peeled
// edges in slot order, then a dataflow assignment in reverse slot order.
// Counter words (u32 index into ctr), one 128-byte line each.
enum : uint32_t {
    kFlowHead = 0,      // u64: queue slots taken by consumers
    kFlowSlots = 32,    // u64: queue slots filled (high half; the low half is unused)
    kFlowDone = 96,     // u64: queue items whose chain has ended
    kFlowNext = 128,    // u64: assignment: next record position to take
    kFlowPeeled = 160,  // edges peeled
    kFlowErr = 192,     // error bits
    kFlowWords = 224
};
constexpr uint32_t kRcStride = 32;  // per-shard record counters, one 128-byte line each
struct FlowArgs {
    const uint64_t* loc;              // bucketed local signatures
    const uint32_t* val;              // bucketed values, NULL for a filter
    const unsigned long long* start;  // S+1 shard starts
    uint32_t S;
    Geom g;
    uint32_t* W;                      // S*cells vertex words (degree, sum of edge indices)
    unsigned long long* queue;        // work items (vertex << 32 | edge); all ones = empty
    unsigned long long* fv;           // assignment: S*cells value words, value | 1 << 32 once final
                                      // (the queue's memory, reused)
    uint64_t queue_cap;
    uint32_t* claimed;                // one bit per edge
    uint64_t claimed_bits;            // edges
    uint32_t* pv;                     // one bit per vertex: an edge was peeled from it
    uint4* rec;                       // per slot {peeled vertex, other, other, value}; x = ~0: empty;
                                      // shard s owns slots [s*cells, (s+1)*cells)
    uint32_t* rec3;                   // k = 4: per slot the third other vertex (else NULL)
    uint32_t* rc;                     // record slots taken per shard, one counter per kRcStride words
    uint64_t nrec;                    // assignment: record slots taken by the peel, all shards
    uint64_t rmax;                    // assignment: the most slots any shard took
    uint32_t epsg;                    // fuse regime: edges per start segment (signature prefetch), 0: none
    uint32_t* ctr;                    // kFlowWords counter words
    uint32_t* err;                    // == ctr + kFlowErr
    uint8_t* data;                    // assignment target
    uint64_t cell_base;               // cell of the first vertex (shard groups)
    uint32_t assign_limit;            // polls after which an assignment wait gives up (0: default)
    uint32_t stall;                   // test hook: no vertex starts final, so every wait runs out
};
cudaError_t launch_incidence32(const uint64_t* loc, uint64_t n, const unsigned long long* start, uint32_t S,
                               const Geom& g, uint32_t* W, uint32_t* err, const uint32_t* drop, cudaStream_t st);
// The same over segment-ordered edges (launch_segment_order): a block per
// (shard, segment) accumulates every contribution to that segment in shared
// memory and stores its vertex words (W needs no zeroing); seg_ends: the
// segment order's bin ends. Fuse graphs (k = 3 or 4), segments of 2^5..2^18
// cells, one segment per bin (incidence_seg_fits); cudaErrorInvalidValue
// otherwise.
bool incidence_seg_fits(const Geom& g);
// xor_words: the round solver's words (degree, XOR of the edge indices).
cudaError_t launch_incidence_seg(const uint64_t* loc, uint64_t n, const unsigned long long* start, uint32_t S,
                                 const Geom& g, const unsigned long long* seg_ends, uint32_t* W, uint32_t* err,
                                 const uint32_t* drop, bool xor_words, cudaStream_t st);
// Marks in `drop` (if given) every edge not set in `claimed` (if given) whose
// (shard, local signature) an earlier such edge already has; table: cap (a
// power of two, >= 2x the edges inserted) zeroed words; *ndrop counts the
// marks, per_shard[s] (if given) those of shard s. With `val` (functions),
// copies whose values differ are counted in *nconflict and not marked.
cudaError_t launch_find_dups(const uint64_t* loc, const uint32_t* val, uint64_t n, const unsigned long long* start,
                             uint32_t S, const uint32_t* claimed, unsigned long long* table, uint64_t cap,
                             uint32_t* drop, unsigned long long* ndrop, unsigned long long* per_shard,
                             unsigned long long* nconflict, cudaStream_t st);
// Peels the shards in batches whose waves fit in L2 (flow_batches launches
// of initial items + worklist peel), then counts the peeled edges.
cudaError_t launch_flow_peel(const FlowArgs& a, cudaStream_t st);
uint32_t flow_batches(const FlowArgs& a);
cudaError_t launch_flow_assign(const FlowArgs& a, cudaStream_t st);
// Counting sort of each shard's edges by the segment of their first vertex
// (fuse regime; locality of the peeling waves): loc/val to loc_out/val_out;
// counts: segment_order_bins(g, S) words of scratch.
cudaError_t launch_segment_order(const uint64_t* loc, const uint32_t* val, uint64_t n,
                                 const unsigned long long* start, uint32_t S, const Geom& g, unsigned long long* counts,
                                 uint64_t* loc_out, uint32_t* val_out, cudaStream_t st);
uint64_t segment_order_bins(const Geom& g, uint32_t S);

// Fuse-regime wave solver (csrc/vf_wave.cu): 64-bit vertex words that hold the
// degree, the other two vertices and the value of the edges' sum; phase I in
// grid-wide rounds, phase II with one CTA per shard; records assigned in
// reverse rounds.
constexpr uint32_t kWFCap = 8192;       // phase II frontier entries per round in shared memory
constexpr uint32_t kWRCap = 1u << 16;   // phase II rounds per shard
constexpr uint32_t kWMaxShards = 1024;
struct WaveArgs {
    const uint64_t* loc;              // bucketed local signatures
    const uint32_t* val;              // bucketed values, NULL for a filter
    const unsigned long long* start;  // S+1 shard starts
    const uint32_t* drop;             // edges left out (duplicates), or NULL
    uint32_t S;
    Geom g;
    uint64_t n;                       // edges
    unsigned long long* W;            // S*cells vertex words
    uint32_t* stamp;                  // S*cells: bits 0..15 round a vertex entered the frontier, 16..31 round it died
    uint32_t* fv[2];                  // phase I frontier: vertex
    unsigned long long* fw[2];        //   and its word at degree one
    uint64_t fcap;
    uint32_t* sfv;                    // phase II spill areas: shard s, frontier buffer k at (2s+k)*scap
    unsigned long long* sfw;
    uint64_t scap;
    uint4* rec;                       // records {peeled vertex, other, other, value}: phase I, then per-shard regions
    uint32_t* off1;                   // phase I: records of round r are [off1[r-1], off1[r])
    uint32_t* off2;                   // phase II: shard s, round k: [off2[s*kWRCap+k], off2[s*kWRCap+k+1]) after base2[s]
    uint32_t* rounds2;                // phase II rounds per shard
    unsigned long long* base2;        // first record of each shard's phase II region
    uint32_t* peel1;                  // per shard: edges peeled in phase I
    uint32_t* front1;                 // per shard: phase I frontier entries of the next round
    uint32_t* ctr;                    // counter words (csrc/vf_wave.cu)
    Bar2* bar;
    uint8_t* data;                    // assignment target
    uint64_t cell_base;               // cell of the first vertex (shard groups)
};
bool wave_eligible(const Geom& g, uint32_t S);
// Incidence (64-bit words) and the round-1 frontier of every degree-one vertex.
cudaError_t launch_wave_incidence(const WaveArgs& a, cudaStream_t st);
// The cooperative peeling kernel: phase I, then phase II.
cudaError_t launch_wave_peel(WaveArgs a, cudaStream_t st);
// Phase II records of every shard in reverse rounds (phase I: launch_assign).
cudaError_t launch_wave_assign(const WaveArgs& a, cudaStream_t st);
// After a failed peel: claim bits of every edge outside the 2-core.
cudaError_t launch_wave_claimed(const WaveArgs& a, uint32_t* claimed, cudaStream_t st);
constexpr uint32_t kWaveCtrWords = 224;
constexpr uint32_t kWaveCtrErr = 192, kWaveCtrPeeled = 96, kWaveCtrR0 = 128, kWaveCtrRec = 64;

// LGE regime: one CTA per shard (peel + lazy Gaussian elimination + assign).
// A task is one shard of one structure; a launch may mix structures.
struct LgeTask {
    uint64_t loc_off;    // first key of the shard in the bucketed loc / val arrays
    uint64_t cell_base;  // first cell of the shard in `data`
    uint8_t* data;       // the structure's data array
    uint32_t m;          // keys in the shard
    uint32_t cells;      // cells per shard
    int32_t b;
    int32_t kind;        // 0 function (values from `val`), 1 filter (fingerprints)
    uint32_t item;       // structure index: failures are recorded in item_fail[item]
    uint8_t fpb, fps;    // filter fingerprint slice (see Geom)
    uint16_t pad;
};

struct LgeArgs {
    const LgeTask* tasks;
    uint32_t ntasks;
    const uint64_t* loc;              // bucketed local signatures
    const uint32_t* val;              // bucketed values (functions)
    uint32_t* item_fail;              // per-structure failure bits (kErr*)
    uint32_t* scratch;                // per-CTA global scratch
    uint64_t scratch_words_per_cta;
    uint32_t m_cap, v_cap;            // largest shard / cell count the scratch layout holds
    uint32_t* err;                    // OR of all failure bits
    uint32_t* stats;                  // [0] peeled edges, [1] core edges, [2] task counter (medium
                                      // configuration), [3] dropped duplicates, [4] spill-list counter,
                                      // [5] spilled tasks, [6] task counter (small configuration)
    uint32_t* item_dup;               // per-structure dropped duplicate filter keys, or NULL
    // Two-configuration launch: the spill list (room for ntasks indices) that the
    // small configuration fills; NULL runs the large configuration alone.
    uint32_t* spill;
    const uint32_t* spill_in;         // set by launch_lge for the last launch
    const uint32_t* spilled;          // count of spill_in (device), set by launch_lge
    uint32_t n_mid;                   // tasks[0, n_mid) have more than kLgeSmallTaskKeys keys
                                      // (lge_partition); the rest go to the small configuration
    uint32_t task_lo, ctr;            // set by launch_lge: first task and counter word of a launch
};
// Tasks of at most this many keys run in the small configuration (three CTAs
// per SM); larger ones in the medium one (two per SM).
constexpr uint32_t kLgeSmallTaskKeys = 7168;
// Stable partition: tasks above kLgeSmallTaskKeys first; returns their count.
uint32_t lge_partition(std::vector<LgeTask>& tasks, uint64_t small_keys = kLgeSmallTaskKeys);
// Layout (in 32-bit words) of one CTA's LGE scratch slab for shards of at most
// m keys and V cells.
constexpr uint32_t kMaxActive = 4096;  // active variables per shard (up to kLgeBigShard keys)
constexpr uint32_t kLPoolPerKey = 40;  // words of coefficient rows per shard key (up to kLgeBigShard keys)
// Above kLgeBigShard keys (the regime's default largest shard) both grow with
// the shard: ~6.6% of a shard's keys become active variables, and the affine
// rows take ~0.0011 m words per key.
constexpr uint32_t kLgeBigShard = 24576;
struct LgeOffsets {
    uint64_t cev, porder, proff, f0, f1, cand, core, eqst, inc_off, inc_cur, inc_list, vstate, act, actv,
        solves, soff, srec, dense, lc, L, lpool, total;
    uint32_t a_cap;  // active variables a shard may have
};

__host__ __device__ constexpr uint64_t lge_take(uint64_t& p, uint64_t words) {
    uint64_t r = p;
    p += (words + 3) & ~uint64_t(3);
    return r;
}

__host__ __device__ constexpr LgeOffsets lge_offsets(uint32_t m, uint32_t V) {
    LgeOffsets o{};
    uint64_t p = 0;
    o.cev = lge_take(p, 3ull * m);
    o.porder = lge_take(p, m);
    o.proff = lge_take(p, V + 2ull);
    o.f0 = lge_take(p, V);
    o.f1 = lge_take(p, V);
    o.cand = lge_take(p, V);
    o.core = lge_take(p, m);
    o.eqst = lge_take(p, m);
    o.inc_off = lge_take(p, V + 1ull);
    o.inc_cur = lge_take(p, V);
    o.inc_list = lge_take(p, 3ull * m);
    o.vstate = lge_take(p, V);
    o.act = lge_take(p, V);
    const uint64_t big = m > kLgeBigShard ? m - kLgeBigShard : 0;
    o.a_cap = uint32_t(kMaxActive + big / 8);
    o.actv = lge_take(p, o.a_cap);
    o.solves = lge_take(p, m);
    o.soff = lge_take(p, uint64_t(m) + V + 4);
    o.srec = lge_take(p, 4ull * m);  // one uint4 per solve
    o.dense = lge_take(p, m);
    o.lc = lge_take(p, m);
    o.lpool = uint64_t(m) * (kLPoolPerKey + big / 500) + 4096;
    o.L = lge_take(p, o.lpool);
    o.total = p;
    return o;
}

cudaError_t launch_lge(const LgeArgs& a, unsigned grid, cudaStream_t st);
unsigned lge_grid();
uint64_t lge_scratch_words_per_cta(uint32_t m_cap, uint32_t v_cap);

// One structure of a batched build (device descriptor).
struct BatchItem {
    const uint64_t* keys;  // this structure's keys
    const void* vals;      // its values (functions) or NULL
    uint64_t key_off;      // first index of its keys in the batch's key space
    uint64_t kh, kl;       // lane keys of its seed
    uint32_t n;
    int32_t h;             // shard bits
    uint32_t hist_off;     // first (structure, shard) slot
    int32_t b;
};

cudaError_t launch_batch_hist(const BatchItem* items, const uint64_t* key_off, uint32_t count, uint64_t total,
                              uint32_t* hist, cudaStream_t st);
cudaError_t launch_batch_scatter(const BatchItem* items, const uint64_t* key_off, uint32_t count, uint64_t total,
                                 unsigned long long* cursor, uint64_t* loc, uint32_t* val, cudaStream_t st);

// One request of a cross-structure query batch (device descriptor).
struct QueryReq {
    Geom g;
    const uint8_t* data;
    const uint64_t* keys;
    void* out;
    uint64_t key_off;
    uint64_t m;
};
cudaError_t launch_query_batch(const QueryReq* reqs, uint32_t count, uint64_t total, cudaStream_t st);

cudaError_t launch_query(int key_kind, const void* keys, const uint64_t* offs, uint64_t m, const Geom& g,
                         const uint8_t* data, void* out, cudaStream_t st);

// Values wider than 32 bits (csrc/vf_wide.cu): split u64 values into the two
// slices' value arrays, pack two solved slices into b-bit cells (words =
// data_bytes / 8 of the b-bit structure), query a b-bit structure.
cudaError_t launch_split64(const uint64_t* v, uint64_t n, int b, uint32_t* lo, void* hi, cudaStream_t st);
cudaError_t launch_pack_wide(const uint32_t* lo, const uint8_t* hi, uint64_t cells, int b, uint64_t words,
                             uint64_t* out, cudaStream_t st);
cudaError_t launch_query_wide(const void* keys, const uint64_t* offs, uint64_t m, const Geom& g, const uint8_t* data,
                              void* out, cudaStream_t st);

}  // namespace vf
