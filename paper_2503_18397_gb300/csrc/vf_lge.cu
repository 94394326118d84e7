// LGE-regime solver of libvfunc (sm_103a): one CTA per shard, shards taken
// from a global counter so uneven shards balance across SMs.
//
// Per shard, all synchronisation is __syncthreads (no spin-waits):
//  1. incidence: degree (8-bit lanes) and XOR of shard-local edge indices
//     (16-bit lanes) per vertex, in shared memory (Sec. 4.3, XOR trick);
//  2. peeling in synchronous rounds; each round first reads every frontier
//     vertex's (degree, XOR) and only then removes edges, so a vertex's only
//     edge is read consistently; edges are claimed with a bit per edge;
//  3. lazy Gaussian elimination of the 2-core (Sec. 3.3, GOV): variables start
//     idle; an equation with one idle variable is solved for it and the
//     variable is eliminated from the other equations; when none is left, the
//     heaviest idle variables are made active (a batch of ~2.5% of the open
//     equations at a time); equations left with no idle variable form the
//     dense system over the active variables;
//  4. every solved variable is an affine function of the active ones; the
//     bit-packed coefficient rows (32 active variables per word) are built
//     round by round (from one record per solve gathered after step 3), the
//     dense rows are reduced by Gauss-Jordan elimination in shared memory, or
//     in the CTA's slab when they do not fit (free variables = 0), solved
//     variables are evaluated forward, and peeled edges are assigned in
//     reverse peel order.
//
// Three configurations of the kernel share this code. Each round of steps 2-3
// ends in a CTA barrier, so one CTA per SM leaves the SM idle at every
// barrier; several CTAs per SM overlap several shards instead. Shards of at
// most kLgeSmallTaskKeys keys run in the small configuration (192 threads,
// 72 KB of shared memory, three CTAs per SM), larger ones in the medium one
// (256 threads, 108 KB, two per SM). A shard whose peel arrays do not fit is
// handed, unchanged, to the spill list, which the large configuration (512
// threads, 200 KB, one CTA per SM) then solves from the start: all solve the
// same system, so which one ran changes neither the outcome nor the retry count. A shard beyond the solver's pool
// (active variables, coefficient rows) fails with kErrLgeSize, a capacity
// error that ends the build rather than a retry.
#include <algorithm>
#include <atomic>

#include "vf_internal.h"

namespace vf {

constexpr uint32_t kMaxBatch = 256;
// large configuration: 512 threads, 200 KB dynamic shared memory, 1 CTA per SM
constexpr int kBigT = 512;
constexpr uint32_t kBigWords = 50 * 1024;
// medium configuration: 256 threads, 108 KB, 2 CTAs per SM
constexpr int kMidT = 256;
constexpr uint32_t kMidWords = 27 * 1024;
// small configuration: 192 threads, 72 KB, 3 CTAs per SM
constexpr int kSmallT = 192;
constexpr uint32_t kSmallWords = 18 * 1024;
constexpr uint32_t kNone = 0xFFFFFFFFu;

uint64_t lge_scratch_words_per_cta(uint32_t m_cap, uint32_t v_cap) { return lge_offsets(m_cap, v_cap).total; }

__device__ __forceinline__ uint32_t rhs_of(const LgeArgs& a, const LgeTask& t, uint64_t ge) {
    return t.kind == 0 ? __ldg(a.val + ge) : fingerprint_slice(__ldg(a.loc + ge), t.b, t.fpb, t.fps);
}

__device__ __forceinline__ uint32_t deg_of(const uint32_t* degw, uint32_t v) {
    return (degw[v >> 2] >> ((v & 3u) * 8u)) & 255u;
}
__device__ __forceinline__ uint32_t xr_of(const uint32_t* xrw, uint32_t v) {
    return (xrw[v >> 1] >> ((v & 1u) * 16u)) & 0xFFFFu;
}

// Inclusive-to-exclusive scan of arr[0..len) in global memory by one CTA.
__device__ void cta_exclusive_scan(uint32_t* arr, uint32_t len, uint32_t* s_part) {
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    const uint32_t chunk = (len + T - 1) / T;
    const uint32_t lo = min(len, tid * chunk), hi = min(len, lo + chunk);
    uint32_t sum = 0;
    for (uint32_t i = lo; i < hi; i++) sum += arr[i];
    s_part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (uint32_t t = 0; t < T; t++) {
            uint32_t x = s_part[t];
            s_part[t] = run;
            run += x;
        }
    }
    __syncthreads();
    uint32_t run = s_part[tid];
    for (uint32_t i = lo; i < hi; i++) {
        uint32_t x = arr[i];
        arr[i] = run;
        run += x;
    }
    __syncthreads();
}

// Drops the 128-byte L2 lines wholly inside [p, p + words) without writing
// them back (discard.global.L2: the line's contents become undefined).
__device__ __forceinline__ void discard_words(const uint32_t* p, uint64_t words) {
    const uint64_t lo = (reinterpret_cast<uint64_t>(p) + 127u) & ~uint64_t(127);
    const uint64_t hi = (reinterpret_cast<uint64_t>(p + words)) & ~uint64_t(127);
    for (uint64_t x = lo + uint64_t(threadIdx.x) * 128u; x < hi; x += uint64_t(blockDim.x) * 128u)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(x) : "memory");
}

// Everything a shard wrote to the CTA's slab is dead once the shard is done,
// and every array is written before it is read by the next shard. Without
// this, the 304 slabs resident at once (more than L2 holds) are written back
// to DRAM line by line as they are evicted; discarding them instead keeps L2
// for live lines. `m`, `V`: the finished shard's keys and cells; `lused`:
// words of coefficient rows (and slab-resident dense system) it wrote.
__device__ void discard_slab(const uint32_t* scr, const LgeOffsets& o, uint32_t m, uint32_t V, uint64_t lused) {
    const uint64_t mm = m, vv = V;
    discard_words(scr + o.cev, 3 * mm);
    discard_words(scr + o.porder, mm);
    discard_words(scr + o.proff, vv + 2);
    discard_words(scr + o.f0, vv);
    discard_words(scr + o.f1, vv);
    discard_words(scr + o.cand, vv);
    discard_words(scr + o.core, mm);
    discard_words(scr + o.eqst, mm);
    discard_words(scr + o.inc_off, vv + 1);
    discard_words(scr + o.inc_cur, vv);
    discard_words(scr + o.inc_list, 3 * mm);
    discard_words(scr + o.vstate, vv);
    discard_words(scr + o.act, vv);
    discard_words(scr + o.actv, o.a_cap);
    discard_words(scr + o.solves, mm);
    discard_words(scr + o.soff, mm + vv + 4);
    discard_words(scr + o.srec, 4 * mm);
    discard_words(scr + o.dense, mm);
    discard_words(scr + o.lc, mm);
    discard_words(scr + o.L, lused < o.lpool ? lused : o.lpool);
}

// Hands task s to the spill list (small configuration) and reports whether
// it did; the large configuration has no spill list and fails the shard.
__device__ __forceinline__ bool spill_task(const LgeArgs& a, uint32_t s) {
    if (!a.spill) return false;
    if (threadIdx.x == 0) a.spill[atomicAdd(&a.stats[5], 1u)] = s;
    return true;
}

template <int kLT, uint32_t kLgeSmemWords, int kMinBlocks>
__global__ void __launch_bounds__(kLT, kMinBlocks) k_lge(LgeArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t s_shard, s_fail;
    __shared__ uint32_t s_cnt[4];
    __shared__ uint32_t s_C, s_rem, s_A, s_S, s_D, s_r, s_apos, s_nact, s_nbatch, s_piv, s_lo, s_dup;
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_batch[kMaxBatch];
    __shared__ uint32_t s_part[kLT];

    const uint32_t tid = threadIdx.x, T = blockDim.x;
    const LgeOffsets o = lge_offsets(a.m_cap, a.v_cap);
    uint32_t* scr = a.scratch + uint64_t(blockIdx.x) * a.scratch_words_per_cta;
    uint32_t* cev = scr + o.cev;
    uint32_t* porder = scr + o.porder;
    uint32_t* proff = scr + o.proff;
    uint32_t* fr[2] = {scr + o.f0, scr + o.f1};
    uint32_t* cand = scr + o.cand;
    uint32_t* core = scr + o.core;
    uint32_t* eqst = scr + o.eqst;
    uint32_t* inc_off = scr + o.inc_off;
    uint32_t* inc_cur = scr + o.inc_cur;
    uint32_t* inc_list = scr + o.inc_list;
    uint32_t* vstate = scr + o.vstate;
    uint32_t* act = scr + o.act;
    uint32_t* actv = scr + o.actv;
    uint32_t* solves = scr + o.solves;
    uint32_t* soff = scr + o.soff;
    uint4* srec = reinterpret_cast<uint4*>(scr + o.srec);
    uint32_t* dense = scr + o.dense;
    uint32_t* lc = scr + o.lc;
    uint32_t* L = scr + o.L;
    constexpr uint32_t kBad = kErrUnsolvable | kErrCapacity | kErrLgeSize | kErrDegOverflow | kErrDupKey;

    // The large configuration behind a small one takes its tasks from the
    // spill list (written by the previous launch), otherwise from all tasks.
    const bool from_spill = a.spilled != nullptr;
    const uint32_t ntasks = from_spill ? *a.spilled : a.ntasks;
    // the previous shard's sizes, for discarding its slab lines (uniform)
    uint32_t prev_m = 0, prev_v = 0;
    uint64_t prev_l = 0;
    for (;;) {
        __shared__ uint32_t s_skip;
        // every path to here ends its shard with a barrier; the barrier below
        // orders the discards before the next shard's first slab write
        if (prev_m | prev_v) discard_slab(scr, o, prev_m, prev_v, prev_l);
        prev_m = prev_v = 0;
        prev_l = 0;
        if (tid == 0) {
            const uint32_t q = atomicAdd(&a.stats[from_spill ? 4 : a.ctr], 1u);
            s_shard = q < ntasks ? (from_spill ? a.spill_in[q] : a.task_lo + q) : kNone;
            s_skip = s_shard != kNone &&
                     (*reinterpret_cast<volatile uint32_t*>(a.item_fail + a.tasks[s_shard].item) & kBad) != 0;
            s_fail = 0;
            s_dup = 0;
        }
        __syncthreads();
        const uint32_t s = s_shard;
        if (s == kNone) break;
        if (s_skip) {  // another shard of this structure already failed: the attempt is void
            __syncthreads();
            continue;
        }
        const LgeTask task = a.tasks[s];
        const uint64_t e0 = task.loc_off;
        const uint32_t m = task.m;
        const uint32_t V = task.cells;
        const uint64_t cbase = task.cell_base;
        const int b = task.b;
        uint8_t* const data = task.data;
        Geom gg;
        gg.kh = gg.kl = 0;
        gg.cells = V;
        gg.span = 0;
        gg.lg_seg = 0;
        gg.h = 0;
        gg.regime = kRegimeLge;
        gg.b = b;
        gg.kind = task.kind;
        gg.fpb = task.fpb;
        gg.fps = task.fps;
        if (m > a.m_cap || V > a.v_cap || V > 65535u || m > 65535u) {
            // (nothing was written to the slab: prev_m, prev_v stay 0)
            if (tid == 0) {
                atomicOr(a.err, kErrCapacity);
                atomicOr(a.item_fail + task.item, kErrCapacity);
            }
            __syncthreads();
            continue;
        }

        // ---------------------------------------------------------------- 1. incidence
        uint32_t* degw = sm;
        uint32_t* xrw = degw + (V + 3) / 4;
        uint32_t* clm = xrw + (V + 1) / 2;
        const uint32_t pw = (V + 3) / 4 + (V + 1) / 2 + (m + 31) / 32;
        if (pw > kLgeSmemWords) {
            if (!spill_task(a, s) && tid == 0) {
                atomicOr(a.err, kErrCapacity);
                atomicOr(a.item_fail + task.item, kErrCapacity);
            }
            __syncthreads();
            continue;
        }
        for (uint32_t i = tid; i < pw; i += T) sm[i] = 0;
        prev_m = m;  // the slab is written from here on
        prev_v = V;
        __syncthreads();
        for (uint32_t e = tid; e < m; e += T) {
            uint64_t v[4];
            edge_of(gg, __ldg(a.loc + e0 + e), v);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                uint32_t vk = uint32_t(v[k]);
                cev[3 * e + k] = vk;
                uint32_t sh8 = (vk & 3u) * 8u;
                uint32_t old = atomicAdd(&degw[vk >> 2], 1u << sh8);
                if (((old >> sh8) & 255u) == 255u) s_fail = 1;
                atomicXor(&xrw[vk >> 1], e << ((vk & 1u) * 16u));
            }
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) {
                atomicOr(a.err, kErrDegOverflow);
                atomicOr(a.item_fail + task.item, kErrDegOverflow);
            }
            __syncthreads();
            continue;
        }

        // -------------------------------------------------------------------- 2. peel
        if (tid == 0) {
            s_cnt[0] = s_cnt[1] = s_cnt[2] = s_cnt[3] = 0;
            proff[0] = 0;
        }
        __syncthreads();
        for (uint32_t v = tid; v < V; v += T)
            if (deg_of(degw, v) == 1u) fr[0][atomicAdd(&s_cnt[0], 1u)] = v;
        __syncthreads();
        uint32_t fi = 0;
        for (;;) {
            const uint32_t nF = s_cnt[fi];
            if (nF == 0) break;
            const uint32_t* F = fr[fi];
            uint32_t* G = fr[fi ^ 1];
            for (uint32_t i = tid; i < nF; i += T) {
                uint32_t v = __ldcg(&F[i]);
                cand[i] = deg_of(degw, v) == 1u ? xr_of(xrw, v) : kNone;
            }
            __syncthreads();
            for (uint32_t i = tid; i < nF; i += T) {
                uint32_t e = __ldcg(&cand[i]);
                if (e == kNone) continue;
                uint32_t bit = 1u << (e & 31u);
                if (atomicOr(&clm[e >> 5], bit) & bit) continue;
                uint32_t v = __ldcg(&F[i]);
                uint32_t side = __ldcg(&cev[3 * e]) == v ? 0u : __ldcg(&cev[3 * e + 1]) == v ? 1u : 2u;
                porder[atomicAdd(&s_cnt[2], 1u)] = (e << 2) | side;
#pragma unroll
                for (uint32_t k = 0; k < 3; k++) {
                    if (k == side) continue;
                    uint32_t u = __ldcg(&cev[3 * e + k]);
                    uint32_t sh8 = (u & 3u) * 8u;
                    uint32_t old = atomicSub(&degw[u >> 2], 1u << sh8);
                    atomicXor(&xrw[u >> 1], e << ((u & 1u) * 16u));
                    if (((old >> sh8) & 255u) == 2u) G[atomicAdd(&s_cnt[fi ^ 1], 1u)] = u;
                }
            }
            __syncthreads();
            if (tid == 0) {
                s_cnt[3]++;
                proff[s_cnt[3]] = s_cnt[2];
                s_cnt[fi] = 0;
            }
            fi ^= 1;
            __syncthreads();
        }
        const uint32_t peeled = s_cnt[2];
        const uint32_t prounds = s_cnt[3];

        // ---------------------------------------------------- 3. lazy Gaussian elimination
        uint32_t C = 0;
        if (peeled < m) {
            if (tid == 0) s_C = 0;
            __syncthreads();
            for (uint32_t e = tid; e < m; e += T)
                if (!((clm[e >> 5] >> (e & 31u)) & 1u)) core[atomicAdd(&s_C, 1u)] = e;
            for (uint32_t v = tid; v <= V; v += T) inc_off[v] = 0;
            __syncthreads();
            C = s_C;
            // Variable states and equation states move to shared memory when they
            // fit (the peel's arrays are dead now); otherwise they stay in the slab.
            // Equation word: bits 0-1 idle count, bit 2 done, bits 3.. XOR of its idle variables.
            const bool in_smem = uint64_t(V) + C <= kLgeSmemWords;
            uint32_t* vst = in_smem ? sm : vstate;
            uint32_t* est = in_smem ? sm + V : eqst;
            for (uint32_t j = tid; j < C; j += T) {
                const uint32_t* evp = cev + 3 * __ldcg(&core[j]);
                const uint32_t ev[3] = {__ldcg(evp), __ldcg(evp + 1), __ldcg(evp + 2)};
                atomicAdd(&inc_off[ev[0]], 1u);
                atomicAdd(&inc_off[ev[1]], 1u);
                atomicAdd(&inc_off[ev[2]], 1u);
                est[j] = ((ev[0] ^ ev[1] ^ ev[2]) << 3) | 3u;
            }
            for (uint32_t v = tid; v < V; v += T) vst[v] = 0;
            for (uint32_t i = tid; i < 256; i += T) s_hist[i] = 0;
            __syncthreads();
            // activation order: core degree, heaviest first (counting sort)
            for (uint32_t v = tid; v < V; v += T) {
                uint32_t d = __ldcg(&inc_off[v]);
                if (d) atomicAdd(&s_hist[min(d, 255u)], 1u);
            }
            cta_exclusive_scan(inc_off, V + 1, s_part);
            for (uint32_t v = tid; v < V; v += T) inc_cur[v] = __ldcg(&inc_off[v]);
            if (tid == 0) {
                uint32_t run = 0;
                for (int d = 255; d >= 1; d--) {
                    uint32_t x = s_hist[d];
                    s_hist[d] = run;
                    run += x;
                }
                s_nact = run;
            }
            __syncthreads();
            for (uint32_t v = tid; v < V; v += T) {
                uint32_t d = __ldcg(&inc_off[v + 1]) - __ldcg(&inc_off[v]);
                if (d) act[atomicAdd(&s_hist[min(d, 255u)], 1u)] = v;
            }
            for (uint32_t j = tid; j < C; j += T) {
                const uint32_t* evp = cev + 3 * __ldcg(&core[j]);
                const uint32_t ev[3] = {__ldcg(evp), __ldcg(evp + 1), __ldcg(evp + 2)};
                inc_list[atomicAdd(&inc_cur[ev[0]], 1u)] = j;
                inc_list[atomicAdd(&inc_cur[ev[1]], 1u)] = j;
                inc_list[atomicAdd(&inc_cur[ev[2]], 1u)] = j;
            }
            __syncthreads();
            // Duplicate keys (Sec. 4.4-4.5): equal local signatures in a shard are
            // the same key. Identical edges never peel, so every duplicate is in
            // the core, next to its copies in the incidence list of its first
            // vertex; the copy of smallest index stays. A filter's copies carry
            // the same fingerprint, a function's copies are dropped when their
            // values agree; a key with two values has no solution at any seed
            // and ends the build (kErrDupKey). A copy that differs from the first
            // copy differs from the earlier copy it meets, so one comparison each
            // finds every conflict.
            for (uint32_t j = tid; j < C; j += T) {
                const uint32_t e = __ldcg(&core[j]);
                const uint64_t x = __ldg(a.loc + e0 + e);
                const uint32_t v = __ldcg(&cev[3 * e]);
                const uint32_t q1 = __ldcg(&inc_off[v + 1]);
                for (uint32_t q = __ldcg(&inc_off[v]); q < q1; q++) {
                    const uint32_t e2 = __ldcg(&core[__ldcg(&inc_list[q])]);
                    if (e2 < e && __ldg(a.loc + e0 + e2) == x) {
                        if (task.kind == 0 && __ldg(a.val + e0 + e2) != __ldg(a.val + e0 + e)) {
                            s_fail = 3;
                        } else {
                            est[j] |= 4u;  // done: no equation of its own
                            atomicAdd(&s_dup, 1u);
                        }
                        break;
                    }
                }
            }
            __syncthreads();
            if (s_fail == 3) {
                if (tid == 0) {
                    atomicOr(a.err, kErrDupKey);
                    atomicOr(a.item_fail + task.item, kErrDupKey);
                }
                __syncthreads();
                continue;
            }
            // The incidence offsets (at most 3C) go to shared memory as 16-bit
            // entries after the states when they fit: the elimination rounds then
            // read only the incidence list itself from the slab.
            uint16_t* ioff16 = nullptr;
            if (in_smem && 3ull * C < 65536 && uint64_t(V) + C + (V + 2) / 2 <= kLgeSmemWords) {
                ioff16 = reinterpret_cast<uint16_t*>(sm + V + C);
                for (uint32_t v = tid; v <= V; v += T) ioff16[v] = uint16_t(__ldcg(&inc_off[v]));
            }
            auto off_of = [&](uint32_t v) -> uint32_t { return ioff16 ? uint32_t(ioff16[v]) : __ldcg(&inc_off[v]); };
            // The rest of shared memory holds the first qcap entries of the two
            // round queues; entries beyond stay in the slab's queues.
            uint32_t qcap = 0;
            uint32_t* sq0 = nullptr;
            if (in_smem) {
                const uint32_t used = (V + C + (ioff16 ? (V + 2) / 2 : 0) + 3) & ~3u;
                qcap = used < kLgeSmemWords ? (kLgeSmemWords - used) / 2 : 0;
                sq0 = sm + used;
            }
            auto qpush = [&](uint32_t q, uint32_t k) {
                const uint32_t idx = atomicAdd(&s_cnt[q], 1u);
                if (idx < qcap) sq0[q * qcap + idx] = k;
                else fr[q][idx] = k;
            };
            auto qread = [&](uint32_t q, uint32_t i) -> uint32_t {
                return i < qcap ? sq0[q * qcap + i] : __ldcg(&fr[q][i]);
            };
            // Removes variable u (now solved from equation `skip`, or active) from
            // every other open equation; an equation left with one idle variable
            // joins the next round's queue, one left with none joins the dense
            // system. Incidence entries are loaded four at a time, before any
            // equation is touched, so their global loads overlap.
            auto remove_var = [&](uint32_t u, uint32_t skip, uint32_t gq) {
                const uint32_t q1 = off_of(u + 1);
                for (uint32_t q = off_of(u); q < q1; q += 4) {
                    uint32_t ks[4];
#pragma unroll
                    for (uint32_t t = 0; t < 4; t++) ks[t] = q + t < q1 ? __ldcg(&inc_list[q + t]) : kNone;
#pragma unroll
                    for (uint32_t t = 0; t < 4; t++) {
                        const uint32_t k = ks[t];
                        if (k == kNone || k == skip || (est[k] & 4u)) continue;
                        const uint32_t old = atomicSub(&est[k], 1u);
                        atomicXor(&est[k], u << 3);
                        const uint32_t c = (old & 3u) - 1u;
                        if (c == 1u) {
                            qpush(gq, k);
                        } else if (c == 0u) {
                            atomicOr(&est[k], 4u);
                            dense[atomicAdd(&s_D, 1u)] = k;
                            atomicSub(&s_rem, 1u);
                        }
                    }
                }
            };
            if (tid == 0) {
                s_rem = C - s_dup;
                s_A = s_S = s_D = s_r = s_apos = s_lo = 0;
                s_cnt[0] = s_cnt[1] = 0;
                soff[0] = 0;
            }
            fi = 0;
            const uint32_t max_rounds = m + V + 2;
            const unsigned lane = tid & 31u, warp = tid >> 5;
            __syncthreads();
            for (;;) {
                if (s_rem == 0 || s_fail) break;
                if (s_r >= max_rounds) {
                    if (tid == 0) s_fail = 2;
                    __syncthreads();
                    break;
                }
                const uint32_t nF = s_cnt[fi];
                if (nF == 0) {
                    // Activate the next heaviest idle variables that still occur in
                    // open equations: the block examines a window of the activation
                    // order in parallel and keeps the first K eligible ones.
                    // batches of 2.5% of the open equations: smaller batches end with
                    // slightly fewer active variables but need many more rounds (per
                    // 9.8K-key shard, 1%: 194 rounds, 655 active; 2.5%: 112 and 704,
                    // 4% fewer cycles)
                    const uint32_t K = max(1u, min(kMaxBatch, s_rem / 40u));
                    const uint32_t base = s_apos;
                    const uint32_t wn = min(T, s_nact - base);
                    bool elig = false;
                    uint32_t v = 0;
                    if (tid < wn) {
                        v = __ldcg(&act[base + tid]);
                        if (vst[v] == 0) {
                            const uint32_t q1 = off_of(v + 1);
                            for (uint32_t q = off_of(v); q < q1 && !elig; q += 4) {
                                uint32_t ks[4];
#pragma unroll
                                for (uint32_t t = 0; t < 4; t++) ks[t] = q + t < q1 ? __ldcg(&inc_list[q + t]) : kNone;
#pragma unroll
                                for (uint32_t t = 0; t < 4; t++) elig |= ks[t] != kNone && (est[ks[t]] & 4u) == 0;
                            }
                        }
                    }
                    const unsigned bal = __ballot_sync(0xFFFFFFFFu, elig);
                    if (lane == 0) s_part[warp] = __popc(bal);
                    __syncthreads();
                    if (tid == 0) {
                        uint32_t run = 0;
                        for (uint32_t w = 0; w < (T + 31) / 32; w++) {
                            const uint32_t x = s_part[w];
                            s_part[w] = run;
                            run += x;
                        }
                        s_part[kLT - 1] = run;  // total eligible
                    }
                    __syncthreads();
                    const uint32_t rank = s_part[warp] + __popc(bal & ((1u << lane) - 1u));
                    const uint32_t tot = s_part[kLT - 1];
                    if (elig && rank < K) s_batch[rank] = v;
                    if (elig && rank == K - 1) s_nbatch = base + tid + 1;  // new scan position
                    __syncthreads();
                    if (tid == 0) {
                        const uint32_t nb = min(K, tot);
                        s_apos = tot >= K ? s_nbatch : base + wn;
                        s_nbatch = nb;
                        if (s_A + nb > o.a_cap || (nb == 0 && s_apos >= s_nact)) s_fail = 2;
                    }
                    __syncthreads();
                    if (s_fail) break;
                    const uint32_t nb = s_nbatch, abase = s_A;
                    for (uint32_t i = tid; i < nb; i += T) {
                        const uint32_t u = s_batch[i];
                        vst[u] = 1u | ((abase + i) << 2);
                        actv[abase + i] = u;
                        remove_var(u, kNone, fi ^ 1);
                    }
                    __syncthreads();
                    if (tid == 0) s_A += nb;
                } else {
                    const uint32_t lo = s_lo;  // solves of earlier rounds; s_S moves below
                    uint32_t mine = kNone;     // this thread's solve (rounds of at most T entries)
                    for (uint32_t i = tid; i < nF; i += T) {
                        const uint32_t j = qread(fi, i);
                        const uint32_t w = est[j];
                        if ((w & 4u) || (w & 3u) != 1u) continue;
                        const uint32_t x = w >> 3;
                        if (atomicCAS(&vst[x], 0u, 3u) != 0u) continue;
                        const uint32_t si = atomicAdd(&s_S, 1u);
                        vst[x] = 2u | (si << 2);
                        mine = (j << 16) | x;
                        solves[si] = mine;
                        atomicOr(&est[j], 4u);
                        atomicSub(&s_rem, 1u);
                    }
                    __syncthreads();
                    // eliminate each variable solved this round from its other equations
                    auto eliminate = [&](uint32_t sv) { remove_var(sv & 0xFFFFu, sv >> 16, fi ^ 1); };
                    if (nF <= T) {  // each solve is still in the register of the thread that made it
                        if (mine != kNone) eliminate(mine);
                    } else {
                        const uint32_t hi = s_S;
                        for (uint32_t si = lo + tid; si < hi; si += T) eliminate(__ldcg(&solves[si]));
                    }
                    __syncthreads();
                }
                if (tid == 0) {
                    s_r++;
                    soff[s_r] = s_S;
                    s_lo = s_S;
                    s_cnt[fi] = 0;
                }
                fi ^= 1;
                __syncthreads();
            }
            if (s_fail) {
                if (tid == 0) {
                    atomicOr(a.err, kErrLgeSize);
                    atomicOr(a.item_fail + task.item, kErrLgeSize);
                }
                __syncthreads();
                continue;
            }
            // the affine rows and the dense system need shared memory: states go back to the slab
            if (in_smem)
                for (uint32_t v = tid; v < V; v += T) vstate[v] = vst[v];
            __syncthreads();
            const uint32_t A = s_A, S = s_S, D = s_D, R = s_r;
            const uint32_t AW = (A + 31) / 32;
            const uint32_t RS = AW | 1u;  // odd row stride: conflict-free shared-memory rows
            // The dense system (rows, right-hand sides, pivot flags, column map) is
            // solved in shared memory when it fits, else in the slab after the
            // affine rows (large shards only; L2-resident, slower).
            const uint64_t rows_off = (uint64_t(S) * AW + 3) & ~uint64_t(3);
            const uint64_t dense_words = uint64_t(D) * RS + 2ull * D + A;
            const bool dense_smem = dense_words <= kLgeSmemWords;
            if (uint64_t(S) * AW > o.lpool || (!dense_smem && rows_off + dense_words > o.lpool)) {
                if (tid == 0) {
                    atomicOr(a.err, kErrLgeSize);
                    atomicOr(a.item_fail + task.item, kErrLgeSize);
                }
                __syncthreads();
                continue;
            }
            prev_l = dense_smem ? uint64_t(S) * AW : rows_off + dense_words;
            // One record per solve, gathered for all solves at once: the solved
            // cell x, its equation's edge e, the two other cells and their states
            // (final when x was solved: active, or solved in an earlier round). The
            // rounds below then wait on two dependent loads instead of five.
            // Shared memory is idle until the dense system is built: the affine
            // rounds read the records from its top end when they fit, and so does
            // the back-substitution if the dense system leaves them room.
            uint4* const srs = 4ull * S <= kLgeSmemWords ? reinterpret_cast<uint4*>(sm + (kLgeSmemWords - 4 * S)) : nullptr;
            for (uint32_t si = tid; si < S; si += T) {
                const uint32_t sv = __ldcg(&solves[si]);
                const uint32_t x = sv & 0xFFFFu, e = __ldcg(&core[sv >> 16]);
                const uint32_t c0 = __ldcg(&cev[3 * e]), c1 = __ldcg(&cev[3 * e + 1]), c2 = __ldcg(&cev[3 * e + 2]);
                const uint32_t u1 = c0 == x ? c1 : c0, u2 = c2 == x ? c1 : c2;
                const uint4 rec = make_uint4(x | (e << 16), u1 | (u2 << 16), __ldcg(&vstate[u1]), __ldcg(&vstate[u2]));
                srec[si] = rec;
                if (srs) srs[si] = rec;
            }
            __syncthreads();
            // the elimination's arrays are dead from here on (their lines are
            // dropped instead of being written back when evicted)
            discard_words(fr[0], V);
            discard_words(fr[1], V);
            discard_words(cand, V);
            discard_words(inc_off, V + 1ull);
            discard_words(inc_cur, V);
            discard_words(inc_list, 3ull * m);
            discard_words(act, V);
            discard_words(eqst, m);
            discard_words(solves, m);
            // solved variables as affine functions of the active ones, round by round
            for (uint32_t r = 0; r < R; r++) {
                const uint32_t lo = __ldcg(&soff[r]), hi = __ldcg(&soff[r + 1]);
                if (hi == lo) continue;
                const uint32_t items = (hi - lo) * AW;
                for (uint32_t it = tid; it < items; it += T) {
                    const uint32_t si = lo + it / AW, w = it % AW;
                    const uint4 q = srs ? srs[si] : __ldcg(&srec[si]);
                    const uint32_t st[2] = {q.z, q.w};
                    uint32_t acc = 0, c = 0;
#pragma unroll
                    for (int k = 0; k < 2; k++) {
                        if ((st[k] & 3u) == 1u) {
                            const uint32_t ai = st[k] >> 2;
                            if ((ai >> 5) == w) acc ^= 1u << (ai & 31u);
                        } else {
                            acc ^= __ldcg(&L[uint64_t(st[k] >> 2) * AW + w]);
                            if (w == 0) c ^= __ldcg(&lc[st[k] >> 2]);
                        }
                    }
                    L[uint64_t(si) * AW + w] = acc;
                    if (w == 0) lc[si] = c ^ rhs_of(a, task, e0 + (q.x >> 16));
                }
                __syncthreads();
            }
            uint32_t* rows = dense_smem ? sm : L + rows_off;
            uint32_t* rhs = rows + uint64_t(D) * RS;
            uint32_t* pivf = rhs + D;
            uint32_t* colrow = pivf + D;
            for (uint32_t it = tid; it < D * AW; it += T) {
                const uint32_t d = it / AW, w = it % AW;
                const uint32_t e = __ldcg(&core[__ldcg(&dense[d])]);
                uint32_t acc = 0, c = 0;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    uint32_t st = __ldcg(&vstate[__ldcg(&cev[3 * e + k])]);
                    if ((st & 3u) == 1u) {
                        uint32_t ai = st >> 2;
                        if ((ai >> 5) == w) acc ^= 1u << (ai & 31u);
                    } else {
                        acc ^= __ldcg(&L[uint64_t(st >> 2) * AW + w]);
                        c ^= __ldcg(&lc[st >> 2]);
                    }
                }
                rows[d * RS + w] = acc;
                if (w == 0) {
                    rhs[d] = c ^ rhs_of(a, task, e0 + e);
                    pivf[d] = 0;
                }
            }
            for (uint32_t c = tid; c < A; c += T) colrow[c] = kNone;
            __syncthreads();
            // the affine rows (and what built the dense rows) are dead now
            discard_words(L, uint64_t(S) * AW);
            discard_words(lc, S);
            discard_words(core, m);
            discard_words(dense, m);
            discard_words(vstate, V);
            // Gauss-Jordan over GF(2): pivot = lowest unused row with the column bit
            // once every row is a pivot no later column can have one (its active
            // variable stays free, 0): the loop ends there
            for (uint32_t col = 0, npiv = 0; col < A && npiv < D; col++) {
                const uint32_t cw = col >> 5, cb = 1u << (col & 31u);
                if (tid == 0) s_piv = kNone;
                __syncthreads();
                for (uint32_t d = tid; d < D; d += T)
                    if (!pivf[d] && (rows[d * RS + cw] & cb)) atomicMin(&s_piv, d);
                __syncthreads();
                const uint32_t p = s_piv;
                if (p == kNone) {
                    __syncthreads();
                    continue;
                }
                for (uint32_t d = tid; d < D; d += T) {
                    if (d == p || !(rows[d * RS + cw] & cb)) continue;
                    // rows d and p never alias: four words of each are loaded
                    // before any is stored, so the round trips overlap
                    uint32_t* rd = rows + d * RS;
                    const uint32_t* rp = rows + p * RS;
                    uint32_t w = cw;
                    for (; w + 4 <= AW; w += 4) {
                        const uint32_t a0 = rd[w], a1 = rd[w + 1], a2 = rd[w + 2], a3 = rd[w + 3];
                        const uint32_t b0 = rp[w], b1 = rp[w + 1], b2 = rp[w + 2], b3 = rp[w + 3];
                        rd[w] = a0 ^ b0, rd[w + 1] = a1 ^ b1, rd[w + 2] = a2 ^ b2, rd[w + 3] = a3 ^ b3;
                    }
                    for (; w < AW; w++) rd[w] ^= rp[w];
                    rhs[d] ^= rhs[p];
                }
                if (tid == 0) {
                    pivf[p] = 1;
                    colrow[col] = p;
                }
                npiv++;
                __syncthreads();
            }
            for (uint32_t d = tid; d < D; d += T)
                if (!pivf[d] && rhs[d] != 0) s_fail = 1;
            __syncthreads();
            if (s_fail) {
                if (tid == 0) {
                    atomicOr(a.err, kErrUnsolvable);
                    atomicOr(a.item_fail + task.item, kErrUnsolvable);
                }
                __syncthreads();
                continue;
            }
            for (uint32_t c = tid; c < A; c += T)
                cell_put_zero(data, b, cbase + __ldcg(&actv[c]), colrow[c] != kNone ? rhs[colrow[c]] : 0u);
            __syncthreads();
            const uint4* const srs_bs =
                srs && (!dense_smem || dense_words + 4ull * S <= kLgeSmemWords) ? srs : nullptr;
            // solved variables, in solve order (their equations as generated)
            for (uint32_t r = 0; r < R; r++) {
                const uint32_t lo = __ldcg(&soff[r]), hi = __ldcg(&soff[r + 1]);
                if (hi == lo) continue;
                for (uint32_t si = lo + tid; si < hi; si += T) {
                    const uint4 q = srs_bs ? srs_bs[si] : __ldcg(&srec[si]);
                    const uint32_t val = rhs_of(a, task, e0 + (q.x >> 16)) ^ cell_get_cg(data, b, cbase + (q.y & 0xFFFFu)) ^
                                         cell_get_cg(data, b, cbase + (q.y >> 16));
                    cell_put_zero(data, b, cbase + (q.x & 0xFFFFu), val);
                }
                __syncthreads();
            }
        }

        // -------------------------------------------- 4. reverse peel-order assignment
        for (uint32_t r = prounds; r-- > 0;) {
            const uint32_t lo = __ldcg(&proff[r]), hi = __ldcg(&proff[r + 1]);
            for (uint32_t i = lo + tid; i < hi; i += T) {
                const uint32_t ent = __ldcg(&porder[i]);
                const uint32_t e = ent >> 2, side = ent & 3u;
                uint32_t val = rhs_of(a, task, e0 + e);
#pragma unroll
                for (uint32_t k = 0; k < 3; k++)
                    if (k != side) val ^= cell_get_cg(data, b, cbase + __ldcg(&cev[3 * e + k]));
                cell_put_zero(data, b, cbase + __ldcg(&cev[3 * e + side]), val);
            }
            __syncthreads();
        }
        if (tid == 0) {
            atomicAdd(&a.stats[0], peeled);
            atomicAdd(&a.stats[1], C - s_dup);
            if (s_dup) {
                atomicAdd(&a.stats[3], s_dup);
                if (a.item_dup) atomicAdd(a.item_dup + task.item, s_dup);
            }
        }
        __syncthreads();
    }
}

#define VF_LGE_SMALL k_lge<kSmallT, kSmallWords, 3>
#define VF_LGE_MID k_lge<kMidT, kMidWords, 2>
#define VF_LGE_BIG k_lge<kBigT, kBigWords, 1>

enum LgeCfg { kCfgSmall = 0, kCfgMid = 1, kCfgBig = 2 };

// Resident CTAs of one configuration on the whole GPU (attributes set once per device).
static unsigned resident(LgeCfg c) {
    static std::atomic<uint64_t> done{0};
    static unsigned per_sm[3] = {1, 1, 1};
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(done.load() & bit)) {
        int p[3] = {0, 0, 0};
        cudaFuncSetAttribute(VF_LGE_SMALL, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmallWords * 4));
        cudaFuncSetAttribute(VF_LGE_MID, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMidWords * 4));
        cudaFuncSetAttribute(VF_LGE_BIG, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBigWords * 4));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p[0], VF_LGE_SMALL, kSmallT, kSmallWords * 4);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p[1], VF_LGE_MID, kMidT, kMidWords * 4);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p[2], VF_LGE_BIG, kBigT, kBigWords * 4);
        for (int i = 0; i < 3; i++) per_sm[i] = unsigned(p[i] < 1 ? 1 : p[i]);
        done.fetch_or(bit);
    }
    return per_sm[c] * unsigned(num_sms());
}

unsigned lge_grid() { return std::max(resident(kCfgSmall), std::max(resident(kCfgMid), resident(kCfgBig))); }

uint32_t lge_partition(std::vector<LgeTask>& tasks, uint64_t small_keys) {
    auto mid = std::stable_partition(tasks.begin(), tasks.end(),
                                     [small_keys](const LgeTask& t) { return t.m > small_keys; });
    return uint32_t(mid - tasks.begin());
}

cudaError_t launch_lge(const LgeArgs& a, unsigned grid, cudaStream_t st) {
    if (a.ntasks == 0) return cudaSuccess;
    if (!a.spill) {  // large configuration alone
        LgeArgs only = a;
        only.task_lo = 0;
        only.ctr = 2;
        VF_LGE_BIG<<<std::min(grid, resident(kCfgBig)), kBigT, kBigWords * 4, st>>>(only);
        return cudaGetLastError();
    }
    // tasks[0, n_mid): medium configuration, counter word 2; the rest: small
    // configuration, counter word 6; then the spill list (counter word 4)
    const uint32_t n_mid = std::min(a.n_mid, a.ntasks);
    if (n_mid > 0) {
        LgeArgs mid = a;
        mid.spilled = nullptr;
        mid.ntasks = n_mid;
        mid.task_lo = 0;
        mid.ctr = 2;
        VF_LGE_MID<<<std::min(std::min(grid, resident(kCfgMid)), n_mid), kMidT, kMidWords * 4, st>>>(mid);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (a.ntasks > n_mid) {
        LgeArgs small = a;
        small.spilled = nullptr;
        small.ntasks = a.ntasks - n_mid;
        small.task_lo = n_mid;
        small.ctr = 6;
        VF_LGE_SMALL<<<std::min(std::min(grid, resident(kCfgSmall)), small.ntasks), kSmallT, kSmallWords * 4, st>>>(
            small);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    LgeArgs last = a;
    last.spill = nullptr;
    last.spilled = a.stats + 5;
    last.spill_in = a.spill;
    last.task_lo = 0;
    last.ctr = 4;
    VF_LGE_BIG<<<std::min(grid, resident(kCfgBig)), kBigT, kBigWords * 4, st>>>(last);
    return cudaGetLastError();
}

}  // namespace vf
