// Wave solver of libvfunc (sm_103a): fuse-regime peeling (Sec. 4.2-4.3) with
// shard state that makes every peeling step one memory round trip, and a
// wave phase in which each shard is peeled by one CTA.
//
// Vertex word (64 bits, one per cell). For an edge with vertices in segments
// s, s+1, s+2 at in-segment offsets o0, o1, o2 and value x (the function's
// value or the filter's fingerprint), the vertex on side k gets the term
//   1 + (enc_k << 5) + (x << (7 + 2L)),  L = lg of the segment size,
//   enc_k = k | (a << 2) | (c << (2 + L)), (a, c) the offsets of the other
//   two vertices in side order.
// A word is the sum of the terms of the edges still incident to it, modulo
// 2^64. Its low 5 bits are the degree (every other part of a term is a
// multiple of 32); at degree one the word IS the one remaining term, so a
// degree-one vertex knows its edge's two other vertices and its value
// without reading the edge. This is the XOR trick of Sec. 4.3 carried to
// the whole edge: removing an edge is one 64-bit fetch-and-add per vertex.
//
// Peeling is in synchronous rounds. Round r peels the edge of every vertex
// that reached degree one in round r-1 (the frontier). Two frontier vertices
// of the same edge both see it; the one of smaller index peels it. A
// frontier vertex whose edge another vertex peeled in round r-1 (it reached
// degree one and then zero in the same round) is dead and skipped. Both
// facts are per-vertex round stamps written in round r-1 (the round a vertex
// entered the frontier, the round it died) that no thread changes during
// round r, so a round needs no claim bit and no re-read of a word: it reads
// three stamps per frontier vertex, all in flight together, and removes the
// edge from the other two vertices with one fetch-and-add each, whose
// results give the next frontier.
//
// Phase I (the seeds: every degree-one vertex of the shards, ~18% of the
// cells, and their short cascades) runs grid-wide rounds over all shards
// with a bounded grid barrier. Once every shard's frontier fits kWFCap
// entries, phase II gives each shard to one CTA: the two waves that sweep
// the shard's segments (Sec. 4.5) continue as CTA-synchronous rounds, one
// __syncthreads per round, with the frontier in shared memory (a round whose
// frontier outgrows it spills the rest to a per-shard area in global
// memory). Every edge peeled writes a record {vertex, other, other, value};
// assignment runs the rounds in reverse (phase II per shard, then phase I).
// A shard whose frontier outgrows the spill area, or that needs more than
// kWRCap rounds, reports kErrFrontier and the attempt is solved by the
// worklist solver.
#include <algorithm>
#include <atomic>

#include <cuda/atomic>

#include "vf_grid.cuh"
#include "vf_internal.h"

namespace vf {

constexpr int kWT = 1024;            // threads per CTA
constexpr int kWK = 2;               // frontier entries per thread per pass (their atomics in flight together)
constexpr uint32_t kWR1Max = 250;    // phase I rounds at most
constexpr size_t kWaveSmem = 2ull * kWFCap * 12;

// Counter words of WaveArgs::ctr (one 128-byte line each).
enum : uint32_t {
    kWcF0 = 0,                  // phase I frontier entries of even rounds
    kWcF1 = 32,                 //   and of odd rounds
    kWcRec = kWaveCtrRec,       // phase I records
    kWcPeeled = kWaveCtrPeeled, // edges peeled
    kWcR0 = kWaveCtrR0,         // first round of phase II
    kWcSwitch = 160,            // phase I is over
    kWcErr = kWaveCtrErr        // error bits
};

__device__ __forceinline__ uint32_t wave_shard_of(const unsigned long long* __restrict__ start, uint32_t S, uint64_t e) {
    uint32_t lo = 0, hi = S;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// The edge of a degree-one vertex: from its shard-local index lx and its word
// w, the shard-local indices of the two other vertices, their terms, and the
// edge's value.
struct WaveEdge {
    uint32_t p1, p2;
    unsigned long long t1, t2;
    uint32_t value;
};

__device__ __forceinline__ unsigned long long wave_term(uint32_t side, uint32_t a, uint32_t c, uint32_t x, int L) {
    const unsigned long long enc = (unsigned long long)side | ((unsigned long long)a << 2) |
                                   ((unsigned long long)c << (2 + L));
    return 1ull + (enc << 5) + ((unsigned long long)x << (7 + 2 * L));
}

__device__ __forceinline__ WaveEdge wave_decode(uint32_t lx, unsigned long long w, int L, uint32_t vmask) {
    const uint32_t m = (1u << L) - 1u;
    const unsigned long long enc = w >> 5;
    const uint32_t side = uint32_t(enc & 3u);
    const uint32_t a = uint32_t(enc >> 2) & m, c = uint32_t(enc >> (2 + L)) & m;
    const uint32_t x = uint32_t(w >> (7 + 2 * L)) & vmask;
    const uint32_t sx = lx >> L, ox = lx & m;
    uint32_t s, o0, o1, o2;
    if (side == 0) { s = sx; o0 = ox; o1 = a; o2 = c; }
    else if (side == 1) { s = sx - 1; o0 = a; o1 = ox; o2 = c; }
    else { s = sx - 2; o0 = a; o1 = c; o2 = ox; }
    const uint32_t v0 = (s << L) | o0, v1 = ((s + 1) << L) | o1, v2 = ((s + 2) << L) | o2;
    WaveEdge r;
    r.value = x;
    if (side == 0) {
        r.p1 = v1; r.t1 = wave_term(1, o0, o2, x, L);
        r.p2 = v2; r.t2 = wave_term(2, o0, o1, x, L);
    } else if (side == 1) {
        r.p1 = v0; r.t1 = wave_term(0, o1, o2, x, L);
        r.p2 = v2; r.t2 = wave_term(2, o0, o1, x, L);
    } else {
        r.p1 = v0; r.t1 = wave_term(0, o1, o2, x, L);
        r.p2 = v1; r.t2 = wave_term(1, o0, o2, x, L);
    }
    return r;
}

// One count per distinct shard among the active lanes (one atomic per shard).
__device__ __forceinline__ void add_by_shard(uint32_t* arr, uint32_t s, bool active) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, active);
    if (!active) return;
    const unsigned peers = __match_any_sync(m, s);
    if (int(lane_id32()) == __ffs(peers) - 1) atomicAdd(arr + s, uint32_t(__popc(peers)));
}

// ---------------------------------------------------------------- incidence

__global__ void __launch_bounds__(256) k_wave_incidence(WaveArgs a) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const int L = a.g.lg_seg;
    const uint32_t m = (1u << L) - 1u;
    for (uint64_t e = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; e < a.n; e += stride) {
        if (a.drop && ((__ldg(a.drop + (e >> 5)) >> (e & 31u)) & 1u)) continue;
        const uint32_t s = wave_shard_of(a.start, a.S, e);
        const uint64_t local = __ldg(a.loc + e);
        uint64_t v[4];
        edge_of(a.g, local, v);
        const uint32_t x = a.val ? __ldg(a.val + e) : fingerprint_slice(local, a.g.b, a.g.fpb, a.g.fps);
        const uint32_t o0 = uint32_t(v[0]) & m, o1 = uint32_t(v[1]) & m, o2 = uint32_t(v[2]) & m;
        const unsigned long long t[3] = {wave_term(0, o1, o2, x, L), wave_term(1, o0, o2, x, L),
                                         wave_term(2, o0, o1, x, L)};
        const uint64_t base = uint64_t(s) * a.g.cells;
        unsigned long long old[3];
#pragma unroll
        for (int k = 0; k < 3; k++) old[k] = atomicAdd(a.W + base + v[k], t[k]);
#pragma unroll
        for (int k = 0; k < 3; k++)
            if ((old[k] & 31u) == 31u) atomicOr(a.ctr + kWcErr, kErrDegOverflow);
    }
}

// Round 1 frontier: every vertex of degree one (stamped as entering in round 1).
__global__ void __launch_bounds__(256) k_wave_seed(WaveArgs a) {
    const uint64_t V = uint64_t(a.S) * a.g.cells;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t wbase = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u);
    uint16_t* const st16 = reinterpret_cast<uint16_t*>(a.stamp);
    for (uint64_t v0 = wbase; v0 < V; v0 += stride) {
        const uint64_t v = v0 + lane_id32();
        const unsigned long long w = v < V ? a.W[v] : 0ull;
        const bool one = (w & 31u) == 1u;
        const uint32_t slot = warp_reserve(a.ctr + kWcF1, one ? 1u : 0u);
        if (one) {
            if (slot < a.fcap) {
                a.fv[1][slot] = uint32_t(v);
                a.fw[1][slot] = w;
                st16[2 * v] = 1;
            } else {
                atomicOr(a.ctr + kWcErr, kErrFrontier);
            }
        }
    }
}

// Round stamps of a vertex: bits 0..15 the round it entered the frontier,
// bits 16..31 the round it died (0: never). Each is written once.
__device__ __forceinline__ uint32_t st_in(uint32_t st) { return st & 0xFFFFu; }
__device__ __forceinline__ uint32_t st_dead(uint32_t st) { return st >> 16; }

// ---------------------------------------------------------------- peeling

// Round r of one frontier entry (x, w): whether x peels its edge, and the
// edge. x is dead if it died in round r-1; otherwise the lowest-indexed
// vertex among x and the edge's other vertices that entered the frontier in
// round r-1 and are alive peels it.
__device__ __forceinline__ bool wave_claim(const WaveArgs& a, uint32_t base, uint32_t lx, unsigned long long w,
                                           uint32_t r, int L, uint32_t vmask, uint32_t cells, WaveEdge& ed) {
    ed = wave_decode(lx, w, L, vmask);
    if (ed.p1 >= cells || ed.p2 >= cells) {  // not an exact degree-one word: report, touch nothing
        atomicOr(a.ctr + kWaveCtrErr, kErrCapacity);
        return false;
    }
    const uint32_t sx = __ldcg(a.stamp + base + lx), s1 = __ldcg(a.stamp + base + ed.p1),
                   s2 = __ldcg(a.stamp + base + ed.p2);
    if (st_dead(sx) == r) return false;
    if (st_in(s1) == r && st_dead(s1) != r && ed.p1 < lx) return false;
    if (st_in(s2) == r && st_dead(s2) != r && ed.p2 < lx) return false;
    return true;
}

__global__ void __launch_bounds__(kWT, 1) k_wave_peel(WaveArgs a) {
    extern __shared__ __align__(16) unsigned char wsm[];
    const unsigned nblocks = gridDim.x;
    const int L = a.g.lg_seg;
    const uint32_t cells = uint32_t(a.g.cells);
    const uint32_t vmask = a.g.b >= 32 ? 0xFFFFFFFFu : ((1u << a.g.b) - 1u);
    uint16_t* const st16 = reinterpret_cast<uint16_t*>(a.stamp);
    uint32_t* const err = a.ctr + kWcErr;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t wbase = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u);
    const unsigned lane = lane_id32(), below = (1u << lane) - 1u;
    // A degree past 31 wrapped a word (incidence reported it): no word can be
    // trusted, the attempt fails without peeling.
    if (dev_atomic(*err).load(cuda::memory_order_relaxed) & (kErrDegOverflow | kErrFrontier)) return;

    // ---------------------------------------------------------- phase I
    for (uint32_t r = 1;; r++) {
        const uint32_t cur = r & 1u, nxt = cur ^ 1u;
        const uint32_t sz = dev_atomic(a.ctr[cur ? kWcF1 : kWcF0]).load(cuda::memory_order_relaxed);
        if (sz == 0 || dev_atomic(a.ctr[kWcSwitch]).load(cuda::memory_order_relaxed)) break;
        const uint32_t* F = a.fv[cur];
        const unsigned long long* FW = a.fw[cur];
        for (uint64_t i0 = wbase; i0 < sz; i0 += nthreads) {
            const uint64_t i = i0 + lane;
            bool peel = false;
            uint32_t x = 0, s = 0, base = 0;
            WaveEdge ed{};
            if (i < sz) {
                x = __ldcg(F + i);
                s = x / cells;
                base = s * cells;
                peel = wave_claim(a, base, x - base, __ldcg(FW + i), r, L, vmask, cells, ed);
            }
            const uint32_t q1 = base + ed.p1, q2 = base + ed.p2;
            const uint32_t rs = warp_reserve(a.ctr + kWcRec, peel ? 1u : 0u);
            unsigned long long n1 = 0, n2 = 0;
            if (peel) {
                a.rec[rs] = make_uint4(x, q1, q2, ed.value);
                n1 = atomicAdd(a.W + q1, 0ull - ed.t1) - ed.t1;
                n2 = atomicAdd(a.W + q2, 0ull - ed.t2) - ed.t2;
            }
            add_by_shard(a.peel1, s, peel);
            const bool f1 = peel && (n1 & 31u) == 1u, f2 = peel && (n2 & 31u) == 1u;
            const uint32_t fs = warp_reserve(a.ctr + (nxt ? kWcF1 : kWcF0), uint32_t(f1) + uint32_t(f2));
            if (peel) {
                uint32_t k = fs;
                if (f1) {
                    if (k < a.fcap) { a.fv[nxt][k] = q1; a.fw[nxt][k] = n1; } else atomicOr(err, kErrFrontier);
                    st16[2ull * q1] = uint16_t(r + 1);
                    k++;
                } else if ((n1 & 31u) == 0u) {
                    st16[2ull * q1 + 1] = uint16_t(r + 1);
                }
                if (f2) {
                    if (k < a.fcap) { a.fv[nxt][k] = q2; a.fw[nxt][k] = n2; } else atomicOr(err, kErrFrontier);
                    st16[2ull * q2] = uint16_t(r + 1);
                } else if ((n2 & 31u) == 0u) {
                    st16[2ull * q2 + 1] = uint16_t(r + 1);
                }
            }
            add_by_shard(a.front1, s, f1);
            add_by_shard(a.front1, s, f2);
        }
        const bool ok = bar2(a.bar, nblocks, err, [&] {
            a.off1[r] = __ldcg(a.ctr + kWcRec);
            uint32_t mx = 0;
            for (uint32_t t = 0; t < a.S; t++) {
                mx = max(mx, __ldcg(a.front1 + t));
                a.front1[t] = 0;
            }
            a.ctr[cur ? kWcF1 : kWcF0] = 0;
            a.ctr[kWcR0] = r + 1;
            if (mx <= kWFCap || r + 1 >= kWR1Max) a.ctr[kWcSwitch] = 1;
        });
        if (!ok) return;
    }

    // ---------------------------------------------------------- phase II
    const uint32_t r0 = dev_atomic(a.ctr[kWcR0]).load(cuda::memory_order_relaxed);
    const uint32_t n0 = dev_atomic(a.ctr[(r0 & 1u) ? kWcF1 : kWcF0]).load(cuda::memory_order_relaxed);
    const uint32_t n1 = dev_atomic(a.ctr[kWcRec]).load(cuda::memory_order_relaxed);
    uint32_t* sfv[2] = {reinterpret_cast<uint32_t*>(wsm), reinterpret_cast<uint32_t*>(wsm + size_t(kWFCap) * 4)};
    unsigned long long* sfw[2] = {reinterpret_cast<unsigned long long*>(wsm + 2ull * kWFCap * 4),
                                  reinterpret_cast<unsigned long long*>(wsm + 2ull * kWFCap * 4 + size_t(kWFCap) * 8)};
    // Round r counts its frontier in s_cnt[r % 3], appends the next one to
    // s_cnt[(r + 1) % 3] and clears s_cnt[(r + 2) % 3] (read in round r - 1);
    // the same rotation for the records of a round (s_rcnt). Capacity errors of
    // round r go to s_errf[r & 1]: the exit test at the top of round r reads
    // s_errf[(r - 1) & 1], which no thread writes during round r, so every
    // thread takes the same decision.
    __shared__ uint32_t s_cnt[3], s_rcnt[3], s_rec, s_errf[2];
    __shared__ unsigned long long s_base2;
    const uint32_t tid = threadIdx.x, T = blockDim.x;
    for (uint32_t s = blockIdx.x; s < a.S; s += nblocks) {
        // entries beyond the shared-memory frontier: this shard's spill areas
        uint32_t* gfv[2] = {a.sfv + (2ull * s) * a.scap, a.sfv + (2ull * s + 1) * a.scap};
        unsigned long long* gfw[2] = {a.sfw + (2ull * s) * a.scap, a.sfw + (2ull * s + 1) * a.scap};
        if (tid == 0) {
            s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
            s_rcnt[0] = s_rcnt[1] = s_rcnt[2] = 0;
            s_rec = 0;
            s_errf[0] = s_errf[1] = 0;
            // this shard's phase II records follow the phase I records and the
            // regions of the shards before it (each sized by its edges left)
            unsigned long long b2 = n1;
            for (uint32_t t = 0; t < s; t++) b2 += (__ldg(a.start + t + 1) - __ldg(a.start + t)) - __ldcg(a.peel1 + t);
            s_base2 = b2;
            a.base2[s] = b2;
            a.off2[uint64_t(s) * kWRCap] = 0;
        }
        __syncthreads();
        const uint32_t base = s * cells;
        // the shard's part of the frontier of round r0
        {
            const uint32_t b0 = r0 & 1u;
            for (uint32_t i = tid; i < n0; i += T) {
                const uint32_t x = __ldcg(a.fv[b0] + i);
                if (x / cells != s) continue;
                const uint32_t k = atomicAdd(&s_cnt[r0 % 3u], 1u);
                const unsigned long long w = __ldcg(a.fw[b0] + i);
                if (k < kWFCap) {
                    sfv[b0][k] = x - base;
                    sfw[b0][k] = w;
                } else if (k - kWFCap < a.scap) {
                    gfv[b0][k - kWFCap] = x - base;
                    gfw[b0][k - kWFCap] = w;
                } else {
                    s_errf[(r0 - 1u) & 1u] = 1;
                }
            }
        }
        __syncthreads();
        uint32_t k2 = 0;
        uint32_t rec_total = 0;
        for (uint32_t r = r0;; r++, k2++) {
            const uint32_t nc = s_cnt[r % 3u];
            if (nc == 0 || s_errf[(r - 1u) & 1u]) break;
            if (k2 + 1 >= kWRCap || r + 1 >= 0xFFFFu) {  // rounds (and 16-bit stamps) exhausted
                if (tid == 0) s_errf[r & 1u] = 1;
                __syncthreads();
                break;
            }
            if (tid == 0) {
                s_cnt[(r + 2) % 3u] = 0;
                s_rcnt[(r + 1) % 3u] = 0;
            }
            const uint32_t ef = r & 1u, cb = r & 1u, nb = cb ^ 1u;
            for (uint32_t p0 = 0; p0 < nc; p0 += uint32_t(T) * kWK) {
                uint32_t lx[kWK];
                WaveEdge ed[kWK];
                bool peel[kWK];
#pragma unroll
                for (int j = 0; j < kWK; j++) {
                    const uint32_t i = p0 + tid + uint32_t(j) * T;
                    peel[j] = false;
                    lx[j] = 0;
                    ed[j] = WaveEdge{};
                    if (i < nc) {
                        unsigned long long w;
                        if (i < kWFCap) {
                            lx[j] = sfv[cb][i];
                            w = sfw[cb][i];
                        } else {
                            lx[j] = __ldcg(gfv[cb] + (i - kWFCap));
                            w = __ldcg(gfw[cb] + (i - kWFCap));
                        }
                        peel[j] = wave_claim(a, base, lx[j], w, r, L, vmask, cells, ed[j]);
                    }
                }
                // records and next-frontier slots are reserved once per warp
                // (same-address shared atomics serialise)
                unsigned long long w1[kWK], w2[kWK];
#pragma unroll
                for (int j = 0; j < kWK; j++) {
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, peel[j]);
                    uint32_t slot = 0;
                    if (m) {
                        const int lead = __ffs(m) - 1;
                        if (int(lane) == lead) {
                            slot = atomicAdd(&s_rec, uint32_t(__popc(m)));
                            atomicAdd(&s_rcnt[r % 3u], uint32_t(__popc(m)));
                        }
                        slot = __shfl_sync(0xFFFFFFFFu, slot, lead) + uint32_t(__popc(m & below));
                    }
                    w1[j] = w2[j] = 0;
                    if (peel[j]) {
                        a.rec[s_base2 + slot] = make_uint4(base + lx[j], base + ed[j].p1, base + ed[j].p2, ed[j].value);
                        w1[j] = atomicAdd(a.W + base + ed[j].p1, 0ull - ed[j].t1);
                        w2[j] = atomicAdd(a.W + base + ed[j].p2, 0ull - ed[j].t2);
                    }
                }
#pragma unroll
                for (int j = 0; j < kWK; j++) {
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const uint32_t p = q ? ed[j].p2 : ed[j].p1;
                        const unsigned long long nw = q ? w2[j] - ed[j].t2 : w1[j] - ed[j].t1;
                        const uint32_t d = uint32_t(nw & 31u);
                        const bool one = peel[j] && d == 1u;
                        const unsigned m = __ballot_sync(0xFFFFFFFFu, one);
                        uint32_t k = 0;
                        if (m) {
                            const int lead = __ffs(m) - 1;
                            if (int(lane) == lead) k = atomicAdd(&s_cnt[(r + 1) % 3u], uint32_t(__popc(m)));
                            k = __shfl_sync(0xFFFFFFFFu, k, lead) + uint32_t(__popc(m & below));
                        }
                        if (one) {
                            if (k < kWFCap) {
                                sfv[nb][k] = p;
                                sfw[nb][k] = nw;
                            } else if (k - kWFCap < a.scap) {
                                gfv[nb][k - kWFCap] = p;
                                gfw[nb][k - kWFCap] = nw;
                            } else {
                                s_errf[ef] = 1;
                            }
                            st16[2ull * (base + p)] = uint16_t(r + 1);
                        } else if (peel[j] && d == 0u) {
                            st16[2ull * (base + p) + 1] = uint16_t(r + 1);
                        }
                    }
                }
            }
            __syncthreads();
            rec_total += s_rcnt[r % 3u];
            if (tid == 0) a.off2[uint64_t(s) * kWRCap + k2 + 1] = rec_total;
        }
        if (tid == 0) {
            a.rounds2[s] = k2;
            atomicAdd(a.ctr + kWcPeeled, s_rec);
            if (s_errf[0] | s_errf[1]) atomicOr(err, kErrFrontier);
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.ctr + kWcPeeled, n1);
}

// ---------------------------------------------------------------- assignment

// Phase II rounds of each shard in reverse, one CTA per shard. The records
// of the next round (in reverse order) are loaded while the current one is
// assigned, so a round waits only on the two cells it reads.
constexpr int kAK = 2;  // records per thread held across a round

__global__ void __launch_bounds__(kWT) k_wave_assign(WaveArgs a) {
    const int b = a.g.b;
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    for (uint32_t s = blockIdx.x; s < a.S; s += gridDim.x) {
        const uint4* rec = a.rec + a.base2[s];
        const uint32_t* off = a.off2 + uint64_t(s) * kWRCap;
        const uint32_t R = a.rounds2[s];
        uint4 nx[kAK];
        uint32_t nlo = 0, nhi = 0;
        if (R > 0) {
            nlo = __ldg(off + R - 1);
            nhi = __ldg(off + R);
#pragma unroll
            for (int j = 0; j < kAK; j++)
                if (nlo + tid + j * T < nhi) nx[j] = __ldg(rec + nlo + tid + j * T);
        }
        for (uint32_t k = R; k-- > 0;) {
            uint4 cu[kAK];
            const uint32_t lo = nlo, hi = nhi;
#pragma unroll
            for (int j = 0; j < kAK; j++) cu[j] = nx[j];
            if (k > 0) {
                nlo = __ldg(off + k - 1);
                nhi = lo;
#pragma unroll
                for (int j = 0; j < kAK; j++)
                    if (nlo + tid + j * T < nhi) nx[j] = __ldg(rec + nlo + tid + j * T);
            }
#pragma unroll
            for (int j = 0; j < kAK; j++) {
                if (lo + tid + j * T >= hi) continue;
                const uint4 r = cu[j];
                const uint32_t x =
                    r.w ^ cell_get_cg(a.data, b, a.cell_base + r.y) ^ cell_get_cg(a.data, b, a.cell_base + r.z);
                cell_put_zero(a.data, b, a.cell_base + r.x, x);
            }
            for (uint32_t i = lo + kAK * T + tid; i < hi; i += T) {  // rounds of more than kAK * T records
                const uint4 r = __ldg(rec + i);
                const uint32_t x =
                    r.w ^ cell_get_cg(a.data, b, a.cell_base + r.y) ^ cell_get_cg(a.data, b, a.cell_base + r.z);
                cell_put_zero(a.data, b, a.cell_base + r.x, x);
            }
            __syncthreads();
        }
    }
}

// Edges still in a 2-core after a failed peel: all three vertices have degree
// two or more (a peeled edge keeps its peeling vertex at degree one). Sets the
// claim bit of every other edge (and of the dropped ones).
__global__ void __launch_bounds__(256) k_wave_claimed(WaveArgs a, uint32_t* claimed) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t wb = blockIdx.x * uint64_t(blockDim.x) + (threadIdx.x & ~31u);
    const uint64_t nr = (a.n + 31) & ~uint64_t(31);
    for (uint64_t e0 = wb; e0 < nr; e0 += stride) {
        const uint64_t e = e0 + lane_id32();
        bool c = false;
        if (e < a.n) {
            if (a.drop && ((__ldg(a.drop + (e >> 5)) >> (e & 31u)) & 1u)) {
                c = true;
            } else {
                const uint32_t s = wave_shard_of(a.start, a.S, e);
                uint64_t v[4];
                edge_of(a.g, __ldg(a.loc + e), v);
                const uint64_t base = uint64_t(s) * a.g.cells;
                uint32_t dmin = 31;
#pragma unroll
                for (int k = 0; k < 3; k++) dmin = min(dmin, uint32_t(__ldcg(a.W + base + v[k]) & 31u));
                c = dmin <= 1u;
            }
        }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, c);
        if (lane_id32() == 0 && e0 < a.n) claimed[e0 >> 5] = bits;
    }
}

// ---------------------------------------------------------------- launches

bool wave_eligible(const Geom& g, uint32_t S) {
    if (g.regime != kRegimeFuse || g.k != 3 || g.lg_seg < 1 || g.lg_seg > 26 || S > kWMaxShards) return false;
    const int vbits = 64 - 7 - 2 * g.lg_seg;
    return g.b <= vbits && g.cells < (uint64_t(1) << 31);
}

static unsigned wave_grid() { return unsigned(num_sms()); }

static unsigned plain_grid(uint64_t work) {
    uint64_t blocks = (work + 255) / 256;
    const uint64_t cap = uint64_t(num_sms()) * 8;
    if (blocks > cap) blocks = cap;
    return unsigned(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_wave_incidence(const WaveArgs& a, cudaStream_t st) {
    if (a.n > 0) {
        k_wave_incidence<<<plain_grid(a.n), 256, 0, st>>>(a);
        k_wave_seed<<<plain_grid(uint64_t(a.S) * a.g.cells), 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_wave_peel(WaveArgs a, cudaStream_t st) {
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(attr_set.load() & bit)) {
        e = cudaFuncSetAttribute(k_wave_peel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kWaveSmem));
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit);
    }
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_wave_peel), dim3(wave_grid()), dim3(kWT), args,
                                       kWaveSmem, st);
}

cudaError_t launch_wave_assign(const WaveArgs& a, cudaStream_t st) {
    const unsigned grid = unsigned(std::min<uint64_t>(a.S, uint64_t(num_sms())));
    k_wave_assign<<<grid < 1 ? 1 : grid, kWT, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wave_claimed(const WaveArgs& a, uint32_t* claimed, cudaStream_t st) {
    k_wave_claimed<<<plain_grid(a.n), 256, 0, st>>>(a, claimed);
    return cudaGetLastError();
}

}  // namespace vf
