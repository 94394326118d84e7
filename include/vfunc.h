/*
 * vfunc.h -- C ABI of the GB300 (sm_103a) implementation of epsilon-cost-sharded
 * hypergraph static functions (VFunc) and static filters (VFilter), after
 * S. Vigna, "epsilon-Cost Sharding: Scaling Hypergraph-Based Static Functions
 * and Filters to Trillions of Keys" (arXiv 2503.18397).
 *
 * Conventions shared by every entry point:
 *  - Pointers to keys, values and outputs may be DEVICE pointers (any CUDA
 *    allocation of the current device, e.g. a torch tensor's data_ptr()) or
 *    HOST pointers (pageable or pinned). Host inputs are copied to the device
 *    inside the call; a host output makes the call wait for its result.
 *  - The caller owns every buffer it passes. The library owns a vf_struct and
 *    its device memory until vf_free.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is ordered on it.
 *  - Every call returns a vf_status and never throws or aborts; CUDA errors map
 *    to VF_ECUDA and vf_last_error() gives the message of the calling thread.
 *  - Keys are either 64-bit integers (VF_KEYS_U64, `keys` = uint64_t[n],
 *    `offsets` = NULL) or byte strings (VF_KEYS_BYTES, `keys` = packed bytes,
 *    `offsets` = uint64_t[n+1], string i = keys[offsets[i] .. offsets[i+1])).
 *  - Values / outputs use the narrowest unsigned type that holds b bits:
 *    uint8_t for b <= 8, uint16_t for b <= 16, uint32_t for b <= 32; only the
 *    low b bits of a value are stored. Filter query outputs are uint8_t 0/1.
 */
#ifndef VFUNC_H
#define VFUNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vf_struct vf_struct;

typedef enum {
    VF_OK = 0,
    VF_EINVAL = 1,    /* bad argument (b out of 1..32, NULL where data is needed, ...) */
    VF_ENOMEM = 2,    /* device or host allocation failed */
    VF_EBUILD = 3,    /* every attempt (seed, seed+1, ..., seed+max_retries) failed */
    VF_EDUP = 4,      /* duplicate keys with different values make a function impossible */
    VF_ETIMEOUT = 5,  /* a bounded device-side wait gave up; results are invalid */
    VF_ECUDA = 6,     /* a CUDA runtime call failed */
    VF_ECAPACITY = 7, /* a size exceeds a documented limit of this implementation */
    VF_EAGAIN = 8,    /* vf_build_resumable stopped after max_groups shard groups; call again */
    VF_EIO = 9        /* a file could not be read or written, or is not a valid serialized form */
} vf_status;

enum { VF_FUNC = 0, VF_FILTER = 1 };
enum { VF_KEYS_U64 = 0, VF_KEYS_BYTES = 1 };
enum { VF_MODE_AUTO = 0, VF_MODE_FUSE = 1, VF_MODE_LGE = 2, VF_MODE_MWHC = 3 };
enum { VF_REGIME_FUSE = 1, VF_REGIME_LGE = 2, VF_REGIME_MWHC = 3 };
/* Fuse-regime solver. All peel the same hypergraph (Sec. 4.3) and give the
 * same query results; they differ in how the work is scheduled on the GPU.
 * VF_SOLVER_FLOW (default): asynchronous worklist peeling that records
 * peeled edges in an order whose reverse is a valid assignment order, then a
 * dataflow assignment. VF_SOLVER_ROUNDS: peeling in synchronous rounds with
 * a grid barrier, assignment in reverse rounds. VF_SOLVER_WAVE: vertex words
 * that sum the degree, the other two vertices and the value of the incident
 * edges, so a peeling step is one fetch-and-add per vertex; grid-wide rounds
 * for the initial cascades, then one CTA per shard for the waves that sweep
 * its segments (Sec. 4.5); assignment in reverse rounds. It needs fuse graphs
 * with k = 3, b <= 57 - 2 lg_seg and at most 1024 shards; other structures, and
 * shards whose waves outgrow its per-round capacity, are solved by
 * VF_SOLVER_FLOW. */
enum { VF_SOLVER_FLOW = 0, VF_SOLVER_ROUNDS = 1, VF_SOLVER_WAVE = 2 };

/* Build parameters. vf_params_default() fills the paper's defaults. */
typedef struct {
    int kind;                /* VF_FUNC (Problem 1) or VF_FILTER (Problem 2) */
    int b;                   /* value bits (function) or fingerprint bits (filter), 1..64;
                                a filter's false-positive rate is 2^-b (Sec. 3.1). Values
                                and outputs are u8/u16/u32/u64 for b <= 8/16/32/64. Above
                                32 bits vf_build solves the low 32 and the high b-32 bit
                                planes as two slices on one hypergraph (same seed) and
                                packs them; batched, resumable and allocation-free
                                builds take b <= 32 */
    int key_kind;            /* VF_KEYS_U64 or VF_KEYS_BYTES */
    int mode;                /* VF_MODE_AUTO: LGE regime below lge_threshold keys, fuse
                                regime above (Sec. 4.2); or force one regime.
                                VF_MODE_MWHC: the MWHC construction (Sec. 4.1):
                                3-partite random 3-hypergraphs, c = 1.23, shard bits
                                min(eq. logballsbins, eq. dupmwhc); the paper's
                                configuration uses eps = 0.01, eta = 0.001 */
    int max_retries;         /* a failed attempt restarts everything with seed+1 (Sec. 4) */
    uint64_t seed;           /* global seed; there is no per-shard seed (Sec. 4) */
    double eps;              /* epsilon of epsilon-cost sharding, eq. (ballsbins); 0.001 */
    double eta;              /* duplicate-edge budget of eq. (logdupfuse) (0.1) or of
                                eq. (dupmwhc) in MWHC mode */
    uint64_t lge_threshold;  /* 800000 keys (Sec. 4.2) */
    uint64_t lge_target;     /* LGE regime: shard bits chosen so mean shard <= this (16384) */
    uint64_t lge_max_shard;  /* LGE regime: shard bits grow until no shard exceeds this
                                (24576); larger shards are solved too (up to 65535
                                cells per shard), with a per-shard pool that grows
                                with the shard (see VF_ECAPACITY under vf_build) */
    int fuse_solver;         /* VF_SOLVER_FLOW (default), VF_SOLVER_ROUNDS or VF_SOLVER_WAVE */
    int arity;               /* vertices per edge of a fuse-regime structure: 3 (default) or 4
                                (4-uniform fuse graphs, Sec. 4.2 with k = 4: one more probe per
                                query for less space; VF_SOLVER_FLOW and VF_SOLVER_ROUNDS peel
                                it, VF_SOLVER_WAVE hands it to VF_SOLVER_FLOW). The LGE and
                                MWHC regimes are 3-uniform whatever this says. */
} vf_params;

/* Geometry and outcome of a built structure. */
typedef struct {
    uint64_t n;              /* keys given */
    uint64_t n_eff;          /* keys solved (a filter drops duplicate local signatures) */
    int kind, b, regime;     /* regime: VF_REGIME_FUSE or VF_REGIME_LGE */
    int h;                   /* shard bits: 2^h shards on the top signature bits (Sec. 4) */
    int h_bb, h_dup;         /* eq. (logballsbins) and eq. (logdupfuse) / eq. (dupmwhc);
                                -1 in LGE regime */
    uint64_t shards;
    uint64_t M;              /* keys in the largest shard; every shard gets cells for M */
    double c;                /* expansion factor: 1.105 (large sharded fuse), 1.12, or
                                1.23 (MWHC: cells = 3 parts of cells / 3) */
    int lg_seg;              /* fuse: log2 of the segment size (eq. nln or eq. ln) */
    uint64_t seg, l, T;      /* fuse: segment size, start segments, segments (l = T - 2) */
    uint64_t cells;          /* cells per shard; shard s owns cells [s*cells, (s+1)*cells) */
    uint64_t total_cells;
    uint64_t data_bytes;     /* size of the data array (b in {8,16,32,64}: native; else bits) */
    uint64_t seed;           /* seed of the successful attempt */
    int retries;             /* failed attempts before it */
    uint64_t peeled, core;   /* edges peeled / edges solved by elimination (last attempt) */
    uint64_t rounds;         /* fuse regime, VF_SOLVER_ROUNDS and VF_SOLVER_WAVE: synchronous
                                peeling rounds of the last attempt (wave: grid-wide rounds plus
                                the most rounds of a shard), summed over shard groups; 0 otherwise */
    int k;                   /* vertices per edge: 3, or 4 for a 4-uniform fuse graph */
} vf_info;

void vf_params_default(vf_params *p);

/* Build a VFunc (values != NULL, kind VF_FUNC) or a VFilter (values == NULL,
 * kind VF_FILTER) over n keys: hash to 128-bit signatures, shard on the top h
 * bits (epsilon-cost sharding, Sec. 4), generate each shard's 3-hyperedges
 * (fuse graph, Sec. 4.2), peel (Sec. 4.3), solve 2-cores by lazy Gaussian
 * elimination in the LGE regime (Sec. 4.2), assign in reverse peel order.
 * Waits for completion (the shard sizes and the outcome are read back).
 * Above 2^30 keys (64-bit keys, fuse regime, up to 2^36) the shards are built
 * one group of consecutive shards (<= 2^30 keys) at a time, so scratch memory
 * is bounded by the group, not by n (Sec. 6, shard-at-a-time construction).
 * Scratch memory comes from the device's default stream-ordered pool; the
 * first build on a device sets that pool to keep up to min(1/8 of device
 * memory, 32 GiB) of freed memory cached for the process (release threshold).
 * Repeated keys (Sec. 4.4: inside a shard, the local signature stands for
 * the key; for 64-bit keys equal local signatures are exactly equal keys, for
 * byte strings a collision of those 64 + h signature bits between different
 * strings counts as a repeat): a filter keeps one copy, a function keeps one
 * copy of each repeated (key, value) pair, and a function key given with two
 * different values ends the build with VF_EDUP at the first attempt (no seed
 * can solve it). vf_info.n_eff counts the keys kept; M counts every key given.
 * Pointers may be host memory or device memory of the current device.
 * Errors: VF_EINVAL (also: a pointer to another device's memory), VF_ENOMEM,
 * VF_EBUILD, VF_EDUP, VF_ETIMEOUT, VF_ECUDA, VF_ECAPACITY
 * (a fuse shard above 2^27 keys; more than 2^30 keys with byte strings or in
 * the LGE regime; an LGE shard whose 2-core needs more active variables or
 * coefficient rows than the solver's per-shard pool: 4096 active variables
 * and 40 words per key up to 24576 keys, growing beyond; a 24576-key shard
 * uses ~1500 and ~30). Only unsolvable systems are retried. */
vf_status vf_build(const void *keys, const uint64_t *offsets, const void *values, uint64_t n,
                   const vf_params *params, void *stream, vf_struct **out);

/* Resumable build (Sec. 6: shards are built one group of consecutive shards
 * at a time). Builds exactly what vf_build builds from the same arguments, in
 * shard groups of at most group_keys keys (0: 2^30), writing every finished
 * group into the file `checkpoint` (the serialized form below, with a header
 * field counting the groups written). With max_groups > 0 a call returns
 * VF_EAGAIN after writing that many groups; a later call with the same keys,
 * values and parameters continues from the file (same seed, same shard
 * histogram, same parameters; anything else starts the file afresh). On
 * VF_OK the file holds the complete structure (vf_load reads it) and *out is
 * the structure. A failed attempt (seed) restarts the file with seed+1.
 * Errors: those of vf_build, VF_EAGAIN, VF_EIO. */
vf_status vf_build_resumable(const void *keys, const uint64_t *offsets, const void *values, uint64_t n,
                             const vf_params *params, const char *checkpoint, uint64_t group_keys,
                             uint32_t max_groups, void *stream, vf_struct **out);

/* Serialized form: a 4096-byte header of little-endian fields (magic
 * "VFSTORE1", version 2, the vf_info of the build, group progress, digests)
 * followed at byte 4096 by the data array in its device layout (shard s owns
 * cells [s*cells, (s+1)*cells); b in {8,16,32} native, else a bit array plus
 * one pad word), so a file can be mapped and its cells read in place.
 * vf_serialize writes 4096 + data_bytes bytes into host memory `buf` (with
 * buf == NULL only *size is set; a smaller capacity is VF_EINVAL).
 * vf_deserialize / vf_load validate the header (VF_EIO if corrupt, foreign or
 * incomplete) and copy the cells to a new structure on the current device. */
vf_status vf_serialize(const vf_struct *s, void *buf, uint64_t capacity, uint64_t *size);
vf_status vf_deserialize(const void *buf, uint64_t size, void *stream, vf_struct **out);
vf_status vf_save(const vf_struct *s, const char *path);
vf_status vf_load(const char *path, void *stream, vf_struct **out);

/* Query m keys (eq. MWHC with k = 3): shard from the top signature bits, cell
 * offset shard*cells with no offset array (Sec. 4), XOR of three cells; a
 * filter compares with the key's fingerprint (Sec. 3.1). For a key outside
 * the set a function returns an arbitrary but deterministic value (Problem 1).
 * Asynchronous on `stream` unless a host pointer is involved. With 64-bit keys
 * in host memory or a host output, the keys are processed in chunks of 2^23
 * that alternate between two library-owned streams (copy in, probe, copy out
 * per chunk), so transfers overlap the probes; `stream` is ordered before and
 * after them, and the call returns once a host output is complete. */
vf_status vf_query(const vf_struct *s, const void *keys, const uint64_t *offsets, uint64_t m,
                   void *out, void *stream);

/* Queries against many resident structures in one launch (the serving
 * pattern): request i answers m 64-bit keys against structure s exactly as
 * vf_query would. keys and out must be device memory; the descriptor table is
 * copied before the call returns, the launch is asynchronous on `stream`. */
typedef struct {
    const vf_struct *s;
    const uint64_t *keys;
    uint64_t m;
    void *out;               /* function: value type of b; filter: uint8 0/1 */
} vf_query_req;

vf_status vf_query_batch(const vf_query_req *reqs, uint32_t count, void *stream);

vf_status vf_get_info(const vf_struct *s, vf_info *info);

/* Parameter planning without building: regime and shard bits for n keys
 * (eq. logballsbins / logdupfuse, Sec. 4.2) and the geometry a largest shard of
 * M keys would get. Pure host computation. */
vf_status vf_plan(const vf_params *params, uint64_t n, uint64_t M, vf_info *out);

/* Device address and size of the data array (read-only for the caller). */
vf_status vf_data(const vf_struct *s, const void **dev_ptr, uint64_t *bytes);

/* Copy the data array to host memory of at least vf_info.data_bytes bytes. */
vf_status vf_export(const vf_struct *s, void *host_dst);

/* 128-bit signatures of n keys under `seed` (out: uint64_t[2n], high word
 * first) -- the first step of build and query, exposed for inspection. */
vf_status vf_signatures(int key_kind, const void *keys, const uint64_t *offsets, uint64_t n,
                        uint64_t seed, uint64_t *out, void *stream);

/* Batched construction of many independent structures (the batching
 * pattern: thousands of structures of uneven sizes built together). All
 * structures' keys are hashed, histogrammed and bucketed by two batched
 * kernels; every LGE-regime shard of every structure is then one task of a
 * single persistent solver launch (tasks largest first when `lpt`), the
 * scatter and that launch captured in one CUDA graph when `use_graph`.
 * Structures at or above `lge_threshold` keys take the fuse regime, one
 * solver each. A structure whose attempt fails is retried alone with its
 * next seed (Sec. 4), up to common->max_retries times. Keys are 64-bit
 * integers (device or host pointers). */
typedef struct {
    const uint64_t *keys;
    const void *values;      /* function: values of the type of b; filter: NULL */
    uint64_t n;
    int kind, b;
    uint64_t seed;
} vf_batch_item;

typedef struct {
    uint64_t lge_threshold;  /* structures with fewer keys use the LGE regime (paper: 800000) */
    uint64_t lge_target;     /* LGE regime: mean keys per shard */
    int lpt;                 /* solve shards largest first */
    int use_graph;           /* scatter + solver as one CUDA graph */
    uint64_t small_cta_keys; /* CTA configuration of the LGE solver: shards of at most this
                                many keys run 3 CTAs of 192 threads per SM, larger ones 2
                                CTAs of 256 threads (7168; 0: every shard in the latter).
                                It changes no seed, retry count or member's value,
                                only the speed. */
} vf_batch_opts;

vf_status vf_batch_opts_default(vf_batch_opts *opts);

/* out: count structure pointers (all NULL on failure). common: eps, eta,
 * lge_max_shard, max_retries (kind, b, seed and the LGE sizes come from the
 * items and opts). Errors as vf_build. */
vf_status vf_build_batch(const vf_batch_item *items, uint32_t count, const vf_params *common,
                         const vf_batch_opts *opts, void *stream, vf_struct **out);

/* Autotuner: times candidate opts (fuse/LGE threshold at the given one or
 * none, mean LGE shard 8192 or 16384 keys, largest-first or natural task
 * order, small CTA configuration for shards up to 7168 keys or not) on a
 * sample of the batch (every k-th structure, ~5% of the keys)
 * and returns the fastest; results are cached per batch shape (count, total
 * keys, largest structure). best_ms: the sample's build time (-1 if cached). */
vf_status vf_tune_batch(const vf_batch_item *items, uint32_t count, const vf_params *common, void *stream,
                        vf_batch_opts *best, double *best_ms);

/* Per-phase device timing (CUDA events recorded on the launching stream
 * around every kernel of build and query). Phases, in order: hash+histogram,
 * scatter, incidence, peel, assign, LGE solver, query. vf_timing_read waits
 * for the recorded events, adds their durations (milliseconds) and kernel
 * launch counts into ms[7] / launches[7], and clears the record. Off by default;
 * timing serialises nothing but adds event records. Not thread-safe. */
vf_status vf_timing_enable(int on);
vf_status vf_timing_read(double *ms, uint64_t *launches);

/* Allocation-free build of a small structure. The paper has no counterpart;
 * this entry point exists for callers that must not allocate device memory
 * during a build: code whose device memory is owned by its own pool or
 * arena, and latency-sensitive paths where a cudaMalloc/cudaFree could
 * synchronise the device or fail under memory pressure. It builds one shard
 * in the lazy-Gaussian-elimination regime (params->mode and the LGE sizes are
 * ignored): the same hash, seed, retries and geometry as vf_build in mode
 * VF_MODE_AUTO or VF_MODE_LGE with lge_target and lge_max_shard of at least
 * n (the defaults for n <= 16384), which also build one LGE shard. The
 * fail_attempts hook of vf_debug_faults applies to it as to vf_build.
 *  keys    device uint64_t[n]; values: device array of the value type of b
 *          (function) or NULL (filter); data: device buffer of at least
 *          data_capacity >= vf_info.data_bytes bytes (get it from vf_plan with
 *          M = n), written with the structure's cells; info: host, receives
 *          the geometry, seed and retries, as vf_get_info would.
 *  All scratch lives in one static device array of about 4.6 MB that every
 *  GPU loading the library keeps until the process exits; no call allocates
 *  or frees memory. The first call on a device looks up that array's device
 *  address; make it before any stream capture. All calls share the array,
 *  so calls that overlap on the GPU (other streams, other host threads) race
 *  and must be serialised by the caller. Waits for completion.
 *  A launch error left pending by the caller's earlier work is cleared on entry.
 *  Errors: VF_ECAPACITY (n > 16384), VF_EINVAL (host pointers or another
 *  device's memory, data buffer too small, byte-string keys, bad b/kind),
 *  VF_EBUILD, VF_EDUP (a key given with two values), VF_ECUDA. */
vf_status vf_build_static(const uint64_t *keys, const void *values, uint64_t n, const vf_params *params,
                          void *data, uint64_t data_capacity, vf_info *info, void *stream);

/* Fault injection for tests of the failure paths (the paper has no
 * counterpart; its failure model is a failed attempt retried with the next
 * seed, Sec. 4). Process-wide, off by default (0, 0, 0); not for production.
 *   fail_attempts: the first fail_attempts attempts of every vf_build (and
 *     vf_build_static) report
 *     failure after solving, so the build retries with seed+1, seed+2, ... as
 *     it does after a 2-core or an unsolvable system (VF_EBUILD once
 *     max_retries is exceeded).
 *   assign_poll_limit: polls after which a wait of the fuse-regime dataflow
 *     assignment gives up (0: the default, ~8 s).
 *   stall_assign: no vertex starts final in that assignment, so every wait
 *     runs out; the build returns VF_ETIMEOUT and the CUDA context stays usable.
 * Errors: VF_EINVAL (fail_attempts < 0). */
vf_status vf_debug_faults(int fail_attempts, uint32_t assign_poll_limit, int stall_assign);

/* Random 32-byte sector reads per second that this device delivers from a
 * table of table_bytes bytes (the paper has no counterpart; a measurement
 * aid for the query's roofline). A query reads three cells at random
 * positions of a data array, one sector each; small arrays are served from
 * L2, large ones from HBM, whose rate for scattered sectors is far below its
 * copy bandwidth. The probe allocates the table on the current device,
 * issues 12 independent random 4-byte loads per thread over a grid of 8
 * blocks of 256 threads per SM, reports the best of six timed launches and
 * frees everything. Waits for completion. Errors: VF_EINVAL (NULL result,
 * table below 4096 bytes), VF_ENOMEM, VF_ECUDA. */
vf_status vf_sector_rate(uint64_t table_bytes, void *stream, double *sectors_per_s);

/* Release a structure (NULL is accepted). */
vf_status vf_free(vf_struct *s);

/* Message of the last failing call on this thread ("" if none). */
const char *vf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
