/*
 * Plain CPU oracle for epsilon-cost-sharded VFunc / VFilter
 * (Vigna, "epsilon-Cost Sharding: Scaling Hypergraph-Based Static Functions and
 * Filters to Trillions of Keys", arXiv 2503.18397).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the independent reference that the
 * CUDA path is checked against. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. The product library never links,
 * includes or calls anything in this directory, and this directory includes
 * nothing from the product.
 *
 * Everything here is deliberately slow and plain: one key at a time, a
 * stack-based peeling visit, plain Gaussian elimination over GF(2). The only
 * concurrency is optional (orc_params.threads): independent shards, and
 * contiguous ranges of keys, handed to a pool of threads.
 *
 * Parity status of each function is stated next to its declaration.
 */
#ifndef VF_ORACLE_H
#define VF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FUNC = 0, ORC_FILTER = 1 };
enum { ORC_KEYS_U64 = 0, ORC_KEYS_BYTES = 1 };
enum { ORC_MODE_AUTO = 0, ORC_MODE_FUSE = 1, ORC_MODE_LGE = 2, ORC_MODE_MWHC = 3 };
enum { ORC_REGIME_FUSE = 1, ORC_REGIME_LGE = 2, ORC_REGIME_MWHC = 3 };
/* ORC_EDUP: a function was given the same key with two different values
 * (no seed can solve it, so it is not retried). */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EBUILD = 3, ORC_EDUP = 4 };

typedef struct {
    int kind;             /* ORC_FUNC or ORC_FILTER */
    int b;                /* value / fingerprint bits, 1..64 */
    int key_kind;         /* ORC_KEYS_U64 or ORC_KEYS_BYTES */
    int mode;             /* ORC_MODE_* */
    int max_retries;      /* extra attempts with seed+1, seed+2, ... */
    uint64_t seed;
    double eps;           /* epsilon of epsilon-cost sharding */
    double eta;           /* duplicate-edge failure budget of eq. (logdupfuse) / eq. (dupmwhc) */
    uint64_t lge_threshold;  /* auto mode: n below this -> LGE regime */
    uint64_t lge_target;     /* LGE regime: wanted mean keys per shard */
    uint64_t lge_max_shard;  /* LGE regime: largest allowed shard */
    int threads;          /* signatures and shards computed by this many threads (1: one after the other);
                           * shards are independent, so the result does not depend on it */
    int arity;            /* fuse regime: 3 (default) or 4 vertices per edge; other regimes are 3-uniform */
} orc_params;

typedef struct {
    uint64_t n;           /* keys given */
    uint64_t n_eff;       /* keys after de-duplication */
    int kind, b, regime;
    int h;                /* shard bits; shards = 2^h */
    int h_bb, h_dup;      /* the two bounds h is the minimum of (fuse and MWHC regimes) */
    uint64_t shards;
    uint64_t M;           /* largest shard */
    double c;             /* expansion factor */
    int lg_seg;           /* fuse: log2 segment size */
    uint64_t seg, l, T;   /* fuse: segment size, start segments, segments */
    uint64_t cells;       /* cells per shard */
    uint64_t total_cells; /* shards * cells */
    uint64_t data_bytes;  /* bytes of the data array */
    uint64_t seed;        /* seed of the successful attempt */
    int retries;          /* failed attempts before it */
    uint64_t peeled, core;/* edges peeled / left in 2-cores (last attempt) */
    int k;                /* vertices per edge (3, or 4 for 4-uniform fuse graphs) */
} orc_info;

void orc_params_default(orc_params *p);

/* Stafford's Mix13 finalizer, the output function of SplitMix64
 * (Steele, Lea, Flood 2014). Pinned by the published SplitMix64 test vector. */
uint64_t orc_mix64(uint64_t z);
/* High 64 bits of a 64x64-bit product (fixed-point inversion). */
uint64_t orc_mulhi(uint64_t a, uint64_t b);

/* 128-bit signature (repo-defined; the paper fixes none, Sec. 4.3 "Peel by
 * Signature"). out[0] = high word (shard bits on top), out[1] = low word. */
void orc_sig_u64(uint64_t key, uint64_t seed, uint64_t out[2]);
void orc_sig_bytes(const uint8_t *p, uint64_t len, uint64_t seed, uint64_t out[2]);

/* Lambert W, principal branch, x >= 0. */
double orc_lambert_w0(double x);
/* eq. (logballsbins), alpha = 1. */
int orc_h_ballsbins(uint64_t n, double eps);
/* eq. (logdupfuse) with the eq. (nln) coefficients alpha=0.41, beta=-3. */
int orc_h_dupfuse(uint64_t n, double eta, double c);
/* eq. (dupmwhc) expressed in bits: floor(lg sqrt(-2 n (c/3)^3 ln(1-eta))). */
int orc_h_dupmwhc(uint64_t n, double eta, double c);
/* Product prod_{i<t}(1 - i/n) of Sec. 4.1 (probability of no repeat). */
double orc_no_repeat_prob(double n, uint64_t t);

/* Shard bits for n keys (before the largest shard is known). */
int orc_plan_h(const orc_params *p, uint64_t n, int *regime, int *h_bb, int *h_dup);
/* Fill c, lg_seg, seg, l, T, cells of info from regime, k and M (Sec. 4.2).
 * Parity unpinned for k = 4 (the paper prints no arity-4 parameters). */
void orc_geometry(orc_info *info);

/* Shard, local signature, edge and fingerprint of a signature. */
uint64_t orc_shard(const uint64_t sig[2], int h);
uint64_t orc_local(const uint64_t sig[2], int h);
void orc_edge(const orc_info *info, uint64_t local, uint64_t v[4]);  /* info->k vertices */
uint64_t orc_fingerprint(uint64_t local, int b);

/* Build. keys: uint64 array (ORC_KEYS_U64) or packed bytes with offsets[n+1].
 * values: func only, uint8/16/32/64 per b (<=8, <=16, <=32, <=64 bits); low b bits used.
 * Keys with equal (shard, local signature) are the same key: a filter keeps one
 * copy, a function one copy of each repeated (key, value) pair, and a key with
 * two different values returns ORC_EDUP at once (info then describes that attempt).
 * On success *data is a malloc'ed array of info->data_bytes bytes. */
int orc_build(const orc_params *p, const void *keys, const uint64_t *offsets,
              const void *values, uint64_t n, orc_info *info, uint8_t **data);
void orc_free(void *ptr);

/* Query m keys against (info, data). out: func -> value type of b; filter -> uint8 0/1. */
void orc_query(const orc_info *info, const uint8_t *data, int key_kind, const void *keys,
               const uint64_t *offsets, uint64_t m, void *out);
/* orc_query with the keys split into `threads` contiguous ranges, one per thread. */
void orc_query_mt(const orc_info *info, const uint8_t *data, int key_kind, const void *keys,
                  const uint64_t *offsets, uint64_t m, void *out, int threads);

/* Cell access (Sec. 5 layout: native array for b in {8,16,32,64}, else a bit array). */
uint64_t orc_cell_get(const uint8_t *data, int b, uint64_t i);

/* Helpers exposed for pin tests on explicit tiny hypergraphs.
 * orc_peel: stack peel of m 3-edges on V vertices; returns number peeled and
 * writes per-edge peel order/side when non-NULL.
 * orc_gf2_solve: plain GE; returns 1 if solvable and writes w[V]. */
uint64_t orc_peel(uint64_t V, uint64_t m, const uint32_t *edges, uint32_t *order, uint8_t *side);
int orc_gf2_solve(uint64_t V, uint64_t m, const uint32_t *edges, const uint64_t *rhs, uint64_t *w);
/* The same for edges of k vertices each. */
uint64_t orc_peel_k(uint64_t V, uint64_t m, int k, const uint32_t *edges, uint32_t *order, uint8_t *side);
int orc_gf2_solve_k(uint64_t V, uint64_t m, int k, const uint32_t *edges, const uint64_t *rhs, uint64_t *w);

/* Batch forms of orc_sig_* and orc_edge used by the tests. */
void orc_sigs(int key_kind, const void *keys, const uint64_t *offsets, uint64_t n, uint64_t seed,
              uint64_t *out);
void orc_edges_of(const orc_info *in, const uint64_t *locals, uint64_t n, uint64_t *out);  /* n x in->k */

#ifdef __cplusplus
}
#endif
#endif
