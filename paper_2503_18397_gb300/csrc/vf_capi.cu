// Host runtime and C ABI of libvfunc: parameter planning (epsilon-cost
// sharding, fuse geometry), the build pipeline with its retry loop, queries,
// and structure management. Declarations and contracts: include/vfunc.h.
#include "vfunc.h"

#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "vf_internal.h"

#include <atomic>

namespace {

thread_local std::string g_last_error;

// Test hooks (vf_debug_faults), off unless a test sets them.
std::atomic<int> g_debug_fail_attempts{0};
std::atomic<uint32_t> g_debug_assign_limit{0};
std::atomic<int> g_debug_stall_assign{0};

vf_status fail(vf_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

#define VF_CK(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(VF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

// Stream-ordered device allocation released on scope exit.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n, cudaStream_t s) {
        release();
        st = s;
        bytes = n;
        return cudaMallocAsync(&p, n ? n : 16, s);
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
    // Takes over o's memory (o is left empty).
    void adopt(DevBuf& o) {
        release();
        p = o.p;
        bytes = o.bytes;
        st = o.st;
        o.p = nullptr;
        o.bytes = 0;
    }
};

// Builds allocate their scratch (gigabytes for large fuse shards) from the
// device's default stream-ordered pool. By default the pool returns freed
// memory to the system at every synchronisation, so each build would map its
// scratch again; keep up to an eighth of the device memory (at most 32 GiB)
// cached instead. Once per device and process.
void keep_pool_warm(int dev) {
    static std::mutex mu;
    static uint64_t done = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || (done >> dev) & 1) return;
    done |= uint64_t(1) << dev;
    cudaMemPool_t pool;
    size_t free_b = 0, total_b = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    uint64_t thr = std::min<uint64_t>(uint64_t(total_b) / 8, uint64_t(32) << 30);
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess) cudaGetLastError();
}

bool on_device(const void* p) { return vf::mem_where(p) == vf::MemWhere::kHere; }

// ------------------------------------------------------------------ timing

enum Phase { kPhHist = 0, kPhScatter, kPhAccum, kPhPeel, kPhAssign, kPhLge, kPhQuery, kNumPhases };

struct TimedLaunch {
    int phase;
    int kernels;  // kernel launches between the two events
    cudaEvent_t a, b;
};

bool g_timing = false;
std::vector<TimedLaunch> g_timed;

// Records an event before a launch and one after it, on the launch's stream.
struct PhaseTimer {
    int phase;
    cudaStream_t st;
    int kernels;
    cudaEvent_t a = nullptr;
    PhaseTimer(int ph, cudaStream_t s, int k = 1) : phase(ph), st(s), kernels(k) {
        if (g_timing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
    }
    ~PhaseTimer() {
        if (!a) return;
        cudaEvent_t b = nullptr;
        if (cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(b, st);
            g_timed.push_back({phase, kernels, a, b});
        } else {
            cudaEventDestroy(a);
        }
    }
};

// ----------------------------------------------------------------- planning

// Lambert W (principal branch) by Newton's method on f(w) = w e^w - x.
double lambert_w(double x) {
    if (x <= 0.0) return 0.0;
    double w = x < 3.0 ? 0.5 * std::log1p(2.0 * x) : std::log(x) - std::log(std::log(x));
    for (int k = 0; k < 100; k++) {
        double e = std::exp(w);
        double step = (w * e - x) / (e * (w + 1.0));
        w -= step;
        if (std::fabs(step) <= 4e-16 * (1.0 + std::fabs(w))) break;
    }
    return w;
}

// eq. (logballsbins) with alpha = 1; no sharding while n eps^2 / 2 <= e.
int h_ballsbins(uint64_t n, double eps) {
    const double x = double(n) * eps * eps / 2.0;
    if (!(x > std::exp(1.0))) return 0;
    const double h = std::floor(std::log2(x) - std::log2(std::log(x)));
    return h > 0 ? int(h) : 0;
}

// eq. (logdupfuse) with the segment-size law eq. (nln): alpha 0.41, beta -3.
int h_dupfuse(uint64_t n, double eta, double c) {
    if (n == 0) return 0;
    const double a = 0.41, b = -3.0;
    const double t = (std::log2(-double(n) / (2.0 * c * std::log(1.0 - eta))) - 2.0 * b) / (2.0 * a);
    const double h = std::floor(std::log2(double(n)) - t / (std::log(2.0) * lambert_w(t)));
    return h > 0 ? int(h) : 0;
}

// eq. (dupmwhc): S <= sqrt(-2 n (c/3)^3 ln(1 - eta)), S = 2^h.
int h_dupmwhc(uint64_t n, double eta, double c) {
    const double s = std::sqrt(-2.0 * double(n) * std::pow(c / 3.0, 3.0) * std::log(1.0 - eta));
    if (!(s >= 1.0)) return 0;
    return int(std::floor(std::log2(s)));
}

void plan_h(const vf_params& p, uint64_t n, vf_info& in) {
    if (p.mode == VF_MODE_MWHC) {
        // Sec. 4.1: random 3-hypergraphs, c = 1.23; eq. (dupmwhc) combined with
        // eq. (logballsbins) by taking the smaller bound
        in.regime = VF_REGIME_MWHC;
        in.h_bb = h_ballsbins(n, p.eps);
        in.h_dup = h_dupmwhc(n, p.eta, 1.23);
        in.h = std::min(in.h_bb, in.h_dup);
        return;
    }
    const bool lge = p.mode == VF_MODE_LGE || (p.mode == VF_MODE_AUTO && n < p.lge_threshold);
    in.regime = lge ? VF_REGIME_LGE : VF_REGIME_FUSE;
    if (!lge && p.arity == 4) {
        // 4-uniform fuse graphs: Sec. 4.2's duplicate-edge estimate with k = 4,
        // exp(-m / (2 c s^3)), never binds, so eq. (logballsbins) sets the shards
        in.h_bb = h_ballsbins(n, p.eps);
        in.h_dup = -1;
        in.h = in.h_bb;
    } else if (!lge) {
        in.h_bb = h_ballsbins(n, p.eps);
        in.h_dup = h_dupfuse(n, p.eta, 1.105);
        in.h = std::min(in.h_bb, in.h_dup);
    } else {
        in.h_bb = in.h_dup = -1;
        int h = 0;
        while (h < 40 && n > (p.lge_target << h)) ++h;
        in.h = h;
    }
}

// Sec. 4.2: c = 1.105 with eq. (nln) segments for sharded shards of at least
// 10^7 keys; otherwise c = 1.12 (eq. (ln) segments in the fuse regime).
void geometry(vf_info& in) {
    const double Mf = double(in.M > 0 ? in.M : 1);
    if (in.regime == VF_REGIME_MWHC) {
        // k-partite 3-hypergraph: three parts of ceil(c M / 3) cells, at least 16
        in.c = 1.23;
        in.lg_seg = 0;
        in.seg = in.l = in.T = 0;
        const uint64_t part = uint64_t(std::ceil(in.c * Mf / 3.0));
        in.cells = 3 * std::max<uint64_t>(part, 16);
    } else if (in.regime == VF_REGIME_LGE) {
        in.c = 1.12;
        in.lg_seg = 0;
        in.seg = in.l = in.T = 0;
        uint64_t cells = uint64_t(std::ceil(in.c * Mf));
        in.cells = std::max<uint64_t>(cells, 32);
    } else if (in.k == 4) {
        // 4-uniform fuse graph (Sec. 4.2, l + 3 segments): the paper gives no
        // arity-4 parameters; Graf and Lemire's arity-4 estimates as they stand
        const double c = 0.77 + 0.305 * std::log(600000.0) / std::log(std::max(Mf, 2.0));
        in.c = std::max(1.075, c);
        double lg = std::floor(std::log(Mf) / std::log(2.91) - 0.5);
        lg = std::min(32.0, std::max(0.0, lg));
        in.lg_seg = int(lg);
        in.seg = uint64_t(1) << in.lg_seg;
        uint64_t T = uint64_t(std::ceil(in.c * Mf / double(in.seg)));
        in.T = std::max<uint64_t>(T, 4);
        in.l = in.T - 3;
        in.cells = in.T * in.seg;
    } else {
        double lg;
        if (in.h > 0 && in.M >= 10000000ull) {
            in.c = 1.105;
            lg = std::floor(0.41 * std::log(Mf) * std::log(std::log(Mf)) - 3.0);
        } else {
            in.c = 1.12;
            lg = std::floor(std::log(Mf) / std::log(3.33) + 2.25);
        }
        lg = std::min(32.0, std::max(0.0, lg));
        in.lg_seg = int(lg);
        in.seg = uint64_t(1) << in.lg_seg;
        uint64_t T = uint64_t(std::ceil(in.c * Mf / double(in.seg)));
        in.T = std::max<uint64_t>(T, 3);
        in.l = in.T - 2;
        in.cells = in.T * in.seg;
    }
    in.total_cells = in.shards * in.cells;
    if (in.b == 8 || in.b == 16 || in.b == 32 || in.b == 64)
        in.data_bytes = in.total_cells * uint64_t(in.b / 8);
    else
        in.data_bytes = ((in.total_cells * uint64_t(in.b) + 63) / 64 + 1) * 8;
}

// fpb / fps: the fingerprint slice of a 32-bit slice of a wider filter.
vf::Geom make_geom(const vf_info& in, int fpb = 0, int fps = 0) {
    vf::Geom g;
    std::memset(&g, 0, sizeof g);
    g.kh = vf::mix64(in.seed ^ vf::kLaneHi);
    g.kl = vf::mix64(in.seed ^ vf::kLaneLo);
    g.cells = in.cells;
    g.span = in.regime == VF_REGIME_MWHC ? in.cells / 3 : in.l * in.seg;
    g.lg_seg = in.lg_seg;
    g.h = in.h;
    g.regime = in.regime;
    g.b = in.b;
    g.kind = in.kind;
    g.fpb = fpb;
    g.fps = fps;
    g.k = in.k == 4 ? 4 : 3;
    return g;
}

size_t value_bytes(int b) { return b <= 8 ? 1 : b <= 16 ? 2 : b <= 32 ? 4 : 8; }

// Input staged on the device (a copy when the caller passed host memory).
struct Staged {
    const void* keys = nullptr;
    const uint64_t* offs = nullptr;
    const void* values = nullptr;
    uint64_t key_bytes = 0;
    DevBuf kbuf, obuf, vbuf;
};

vf_status stage_keys(int key_kind, const void* keys, const uint64_t* offsets, uint64_t n, cudaStream_t st,
                     Staged& s) {
    if (key_kind == VF_KEYS_U64) {
        s.key_bytes = n * 8;
        if (on_device(keys) || n == 0) {
            s.keys = keys;
        } else {
            VF_CK(s.kbuf.alloc(s.key_bytes, st));
            VF_CK(cudaMemcpyAsync(s.kbuf.p, keys, s.key_bytes, cudaMemcpyHostToDevice, st));
            s.keys = s.kbuf.p;
        }
        return VF_OK;
    }
    const bool offs_dev = on_device(offsets);
    uint64_t total = 0;
    if (offs_dev) {
        VF_CK(cudaMemcpyAsync(&total, offsets + n, 8, cudaMemcpyDeviceToHost, st));
        VF_CK(cudaStreamSynchronize(st));
        s.offs = offsets;
    } else {
        total = offsets[n];
        VF_CK(s.obuf.alloc((n + 1) * 8, st));
        VF_CK(cudaMemcpyAsync(s.obuf.p, offsets, (n + 1) * 8, cudaMemcpyHostToDevice, st));
        s.offs = s.obuf.as<uint64_t>();
    }
    s.key_bytes = total;
    if (on_device(keys) || total == 0) {
        s.keys = keys;
        if (total == 0) {
            VF_CK(s.kbuf.alloc(16, st));
            s.keys = s.kbuf.p;
        }
    } else {
        VF_CK(s.kbuf.alloc(total, st));
        VF_CK(cudaMemcpyAsync(s.kbuf.p, keys, total, cudaMemcpyHostToDevice, st));
        s.keys = s.kbuf.p;
    }
    return VF_OK;
}

template <class T>
vf_status h2d(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
    VF_CK(b.alloc(v.size() * sizeof(T), st));
    VF_CK(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return VF_OK;
}

// One attempt of the round-synchronous fuse-regime solver. Returns VF_OK,
// VF_EBUILD (peel failed: the attempt must be retried), or an error.
vf_status solve_rounds(const vf_info& in, const vf::Geom& g, const uint64_t* loc, const uint32_t* val,
                       const unsigned long long* start, uint8_t* data, cudaStream_t st, uint64_t* peeled,
                       uint64_t* rounds_out, uint64_t cell_base, const uint32_t* drop, uint64_t ndrop,
                       DevBuf* claimed_out, const unsigned long long* seg_ends = nullptr) {
    const uint64_t n = in.n_eff;
    const uint64_t V = in.total_cells;
    const bool own_incidence = seg_ends && vf::incidence_seg_fits(g);  // writes every vertex word
    DevBuf W, claimed, f0, f1, rec, rec3, roff, ctr;
    VF_CK(W.alloc(V * 4, st));
    if (!own_incidence) VF_CK(cudaMemsetAsync(W.p, 0, V * 4, st));
    VF_CK(claimed.alloc(((n + 31) / 32) * 4, st));
    if (drop)  // dropped duplicates count as claimed: they are never peeled
        VF_CK(cudaMemcpyAsync(claimed.p, drop, ((n + 31) / 32) * 4, cudaMemcpyDeviceToDevice, st));
    else
        VF_CK(cudaMemsetAsync(claimed.p, 0, ((n + 31) / 32) * 4, st));
    VF_CK(f0.alloc(V * 8, st));
    VF_CK(f1.alloc(V * 8, st));
    VF_CK(rec.alloc(std::max<uint64_t>(n, 1) * 16, st));
    if (g.k == 4) VF_CK(rec3.alloc(std::max<uint64_t>(n, 1) * 4, st));
    const uint32_t round_cap = uint32_t(std::min<uint64_t>(n + 1, uint64_t(1) << 22));
    VF_CK(roff.alloc((uint64_t(round_cap) + 1) * 4, st));
    VF_CK(cudaMemsetAsync(roff.p, 0, 4, st));
    // counters (4 x u32), error word, barrier
    const size_t ctr_bytes = 64 + sizeof(vf::Bar2);
    VF_CK(ctr.alloc(ctr_bytes, st));
    VF_CK(cudaMemsetAsync(ctr.p, 0, ctr_bytes, st));
    uint32_t* c32 = ctr.as<uint32_t>();
    vf::FuseSolveArgs a;
    std::memset(&a, 0, sizeof a);
    a.loc = loc;
    a.val = val;
    a.start = start;
    a.S = uint32_t(in.shards);
    a.g = g;
    a.W = W.as<uint32_t>();
    a.claimed = claimed.as<uint32_t>();
    a.front[0] = f0.as<uint2>();
    a.front[1] = f1.as<uint2>();
    a.front_cap = V;
    a.rec = rec.as<uint4>();
    a.rec3 = rec3.as<uint32_t>();
    a.round_off = roff.as<uint32_t>();
    a.round_cap = round_cap;
    a.ctr = c32;
    a.err = c32 + 6;
    a.bar = reinterpret_cast<vf::Bar2*>(c32 + 16);
    a.data = data;
    a.cell_base = cell_base;
    {
        PhaseTimer t(kPhAccum, st);
        if (own_incidence)
            VF_CK(vf::launch_incidence_seg(loc, n, start, a.S, g, seg_ends, a.W, a.err, drop, true, st));
        else
            VF_CK(vf::launch_accumulate(loc, n, start, a.S, g, a.W, a.err, drop, st));
    }
    {
        PhaseTimer t(kPhPeel, st);
        VF_CK(vf::launch_peel(a, st));
    }
    uint32_t h[8];
    VF_CK(cudaMemcpyAsync(h, c32, sizeof h, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    const uint32_t rounds = h[3], count = h[2], err = h[6];
    *peeled = count;
    *rounds_out = rounds;
    if (err & vf::kErrTimeout) return fail(VF_ETIMEOUT, "peeling barrier timed out");
    if (err & (vf::kErrDegOverflow | vf::kErrFrontier)) return VF_EBUILD;
    if (count != n - ndrop) {  // non-empty 2-core
        if (claimed_out) claimed_out->adopt(claimed);
        return VF_EBUILD;
    }
    VF_CK(cudaMemsetAsync(a.bar, 0, sizeof(vf::Bar2), st));
    a.rounds = rounds;
    {
        PhaseTimer t(kPhAssign, st);
        VF_CK(vf::launch_assign(a, st));
    }
    uint32_t e2 = 0;
    VF_CK(cudaMemcpyAsync(&e2, a.err, 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    if (e2 & vf::kErrTimeout) return fail(VF_ETIMEOUT, "assignment barrier timed out");
    return VF_OK;
}

// One attempt of the asynchronous fuse-regime solver. Returns VF_OK, VF_EBUILD
// (peel failed: retry), or an error.
vf_status solve_flow(const vf_info& in, const vf::Geom& g, const uint64_t* loc, const uint32_t* val,
                     const unsigned long long* start, uint8_t* data, cudaStream_t st, uint64_t* peeled,
                     uint64_t cell_base, const uint32_t* drop, uint64_t ndrop, DevBuf* claimed_out,
                     const unsigned long long* seg_ends = nullptr) {
    const uint64_t n = in.n_eff;
    const uint64_t V = in.total_cells;
    DevBuf W, queue, claimed, pv, rec, rec3, ctr;
    const bool own_incidence = seg_ends && vf::incidence_seg_fits(g);  // writes every vertex word
    VF_CK(W.alloc(V * 4, st));
    if (!own_incidence) VF_CK(cudaMemsetAsync(W.p, 0, V * 4, st));
    VF_CK(queue.alloc(V * 8, st));
    VF_CK(cudaMemsetAsync(queue.p, 0xFF, V * 8, st));
    const uint64_t ewords = std::max<uint64_t>((n + 31) / 32, 1), vwords = std::max<uint64_t>((V + 31) / 32, 1);
    VF_CK(claimed.alloc(ewords * 4, st));
    if (drop)  // dropped duplicates count as claimed: they are never peeled
        VF_CK(cudaMemcpyAsync(claimed.p, drop, ewords * 4, cudaMemcpyDeviceToDevice, st));
    else
        VF_CK(cudaMemsetAsync(claimed.p, 0, ewords * 4, st));
    VF_CK(pv.alloc(vwords * 4, st));
    VF_CK(cudaMemsetAsync(pv.p, 0, vwords * 4, st));
    VF_CK(rec.alloc(std::max<uint64_t>(V, 1) * 16, st));  // one slot per item, at most one item per vertex
    if (g.k == 4) VF_CK(rec3.alloc(std::max<uint64_t>(V, 1) * 4, st));  // the third other vertex
    VF_CK(ctr.alloc(vf::kFlowWords * 4, st));
    VF_CK(cudaMemsetAsync(ctr.p, 0, vf::kFlowWords * 4, st));
    DevBuf rc;  // record slots per shard, one 128-byte line each
    VF_CK(rc.alloc(std::max<uint64_t>(in.shards, 1) * vf::kRcStride * 4, st));
    VF_CK(cudaMemsetAsync(rc.p, 0, std::max<uint64_t>(in.shards, 1) * vf::kRcStride * 4, st));
    vf::FlowArgs a;
    std::memset(&a, 0, sizeof a);
    a.loc = loc;
    a.val = val;
    a.start = start;
    a.S = uint32_t(in.shards);
    a.g = g;
    a.W = W.as<uint32_t>();
    a.queue = queue.as<unsigned long long>();
    a.fv = a.queue;
    a.queue_cap = V;
    a.claimed = claimed.as<uint32_t>();
    a.claimed_bits = n;
    a.pv = pv.as<uint32_t>();
    a.rec = rec.as<uint4>();
    a.rec3 = g.k == 4 ? rec3.as<uint32_t>() : nullptr;
    a.rc = rc.as<uint32_t>();
    if (g.regime == VF_REGIME_FUSE && in.shards > 0) {
        const uint64_t l = g.span >> g.lg_seg;  // start segments of a shard
        a.epsg = l ? uint32_t(std::min<uint64_t>(n / in.shards / l, 0xFFFFFFFFull)) : 0u;
    }
    a.ctr = ctr.as<uint32_t>();
    a.err = a.ctr + vf::kFlowErr;
    a.data = data;
    a.cell_base = cell_base;
    a.assign_limit = g_debug_assign_limit.load();
    a.stall = g_debug_stall_assign.load() ? 1u : 0u;
    {
        PhaseTimer t(kPhAccum, st);
        if (own_incidence)
            VF_CK(vf::launch_incidence_seg(loc, n, start, a.S, g, seg_ends, a.W, a.err, drop, false, st));
        else
            VF_CK(vf::launch_incidence32(loc, n, start, a.S, g, a.W, a.err, drop, st));
    }
    {
        // per batch: (head rebase), initial items, worklist peel; then the peeled count
        PhaseTimer t(kPhPeel, st, int(3 * vf::flow_batches(a)));
        VF_CK(vf::launch_flow_peel(a, st));
    }
    std::vector<uint32_t> h(vf::kFlowWords);
    std::vector<uint32_t> hrc(std::max<uint64_t>(in.shards, 1) * vf::kRcStride);
    VF_CK(cudaMemcpyAsync(h.data(), a.ctr, vf::kFlowWords * 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaMemcpyAsync(hrc.data(), rc.p, hrc.size() * 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    const uint32_t count = h[vf::kFlowPeeled], err = h[vf::kFlowErr];
    uint64_t slots = 0, rmax = 0;
    for (uint64_t s = 0; s < in.shards; s++) {
        slots += hrc[s * vf::kRcStride];
        rmax = std::max<uint64_t>(rmax, hrc[s * vf::kRcStride]);
    }
    *peeled = count - ndrop;  // claim bits include the dropped duplicates
    if (err & vf::kErrTimeout) return fail(VF_ETIMEOUT, "asynchronous peeling wait timed out");
    if (err & (vf::kErrDegOverflow | vf::kErrFrontier)) return VF_EBUILD;
    if (count != n) {  // non-empty 2-core
        if (claimed_out) claimed_out->adopt(claimed);
        return VF_EBUILD;
    }
    if (rmax > in.cells) return fail(VF_ECUDA, "asynchronous peeling took more record slots than items");
    a.nrec = slots;
    a.rmax = rmax;
    {
        PhaseTimer t(kPhAssign, st, slots ? 2 : 1);  // final flags, dataflow assignment
        VF_CK(vf::launch_flow_assign(a, st));
    }
    uint32_t e2 = 0;
    VF_CK(cudaMemcpyAsync(&e2, a.err, 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    if (e2 & vf::kErrTimeout) return fail(VF_ETIMEOUT, "dataflow assignment wait timed out");
    return VF_OK;
}

// One attempt of the wave solver (csrc/vf_wave.cu). Returns VF_OK, VF_EBUILD
// (peel failed: retry) or an error; *fallback: the shards exceeded the wave
// phase's capacities and the attempt must be solved by another solver (the
// data array is untouched then).
vf_status solve_wave(const vf_info& in, const vf::Geom& g, const uint64_t* loc, const uint32_t* val,
                     const unsigned long long* start, uint8_t* data, cudaStream_t st, uint64_t* peeled,
                     uint64_t* rounds_out, uint64_t cell_base, const uint32_t* drop, uint64_t ndrop,
                     DevBuf* claimed_out, bool* fallback) {
    *fallback = false;
    const uint64_t n = in.n_eff;
    const uint64_t V = in.total_cells;
    const uint32_t S = uint32_t(in.shards);
    const uint64_t fcap = V / 2 + 4096;
    // phase II spill area per shard and frontier buffer: a quarter of its cells, at most 2^20 entries
    const uint64_t scap = std::min<uint64_t>(in.cells / 4 + 64, uint64_t(1) << 20);
    DevBuf W, stamp, fv, fw, sv, sw, rec, off1, off2, per, ctr;
    VF_CK(W.alloc(V * 8, st));
    VF_CK(cudaMemsetAsync(W.p, 0, V * 8, st));
    VF_CK(stamp.alloc(V * 4, st));
    VF_CK(cudaMemsetAsync(stamp.p, 0, V * 4, st));
    VF_CK(fv.alloc(2 * fcap * 4, st));
    VF_CK(fw.alloc(2 * fcap * 8, st));
    VF_CK(sv.alloc(2 * uint64_t(S) * scap * 4, st));
    VF_CK(sw.alloc(2 * uint64_t(S) * scap * 8, st));
    VF_CK(rec.alloc(std::max<uint64_t>(n, 1) * 16, st));
    VF_CK(off1.alloc(264 * 4, st));
    VF_CK(cudaMemsetAsync(off1.p, 0, 264 * 4, st));
    VF_CK(off2.alloc(uint64_t(S) * vf::kWRCap * 4, st));
    // per shard: phase II rounds (u32), base2 (u64), peel1 (u32), front1 (u32)
    VF_CK(per.alloc(uint64_t(S) * 20, st));
    VF_CK(cudaMemsetAsync(per.p, 0, uint64_t(S) * 20, st));
    const size_t ctr_bytes = vf::kWaveCtrWords * 4 + sizeof(vf::Bar2);
    VF_CK(ctr.alloc(ctr_bytes, st));
    VF_CK(cudaMemsetAsync(ctr.p, 0, ctr_bytes, st));
    const uint32_t one = 1;
    VF_CK(cudaMemcpyAsync(ctr.as<uint32_t>() + vf::kWaveCtrR0, &one, 4, cudaMemcpyHostToDevice, st));
    vf::WaveArgs a;
    std::memset(&a, 0, sizeof a);
    a.loc = loc;
    a.val = val;
    a.start = start;
    a.drop = drop;
    a.S = S;
    a.g = g;
    a.n = n;
    a.W = W.as<unsigned long long>();
    a.stamp = stamp.as<uint32_t>();
    a.fv[0] = fv.as<uint32_t>();
    a.fv[1] = fv.as<uint32_t>() + fcap;
    a.fw[0] = fw.as<unsigned long long>();
    a.fw[1] = fw.as<unsigned long long>() + fcap;
    a.fcap = fcap;
    a.sfv = sv.as<uint32_t>();
    a.sfw = sw.as<unsigned long long>();
    a.scap = scap;
    a.rec = rec.as<uint4>();
    a.off1 = off1.as<uint32_t>();
    a.off2 = off2.as<uint32_t>();
    a.base2 = per.as<unsigned long long>();
    a.rounds2 = reinterpret_cast<uint32_t*>(per.as<uint8_t>() + uint64_t(S) * 8);
    a.peel1 = a.rounds2 + S;
    a.front1 = a.peel1 + S;
    a.ctr = ctr.as<uint32_t>();
    a.bar = reinterpret_cast<vf::Bar2*>(a.ctr + vf::kWaveCtrWords);
    a.data = data;
    a.cell_base = cell_base;
    {
        PhaseTimer t(kPhAccum, st, 2);  // incidence, round-1 frontier
        VF_CK(vf::launch_wave_incidence(a, st));
    }
    {
        PhaseTimer t(kPhPeel, st);
        VF_CK(vf::launch_wave_peel(a, st));
    }
    std::vector<uint32_t> h(vf::kWaveCtrWords);
    VF_CK(cudaMemcpyAsync(h.data(), a.ctr, vf::kWaveCtrWords * 4, cudaMemcpyDeviceToHost, st));
    std::vector<uint32_t> r2(S);
    VF_CK(cudaMemcpyAsync(r2.data(), a.rounds2, uint64_t(S) * 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    const uint32_t err = h[vf::kWaveCtrErr], count = h[vf::kWaveCtrPeeled], r0 = h[vf::kWaveCtrR0];
    *peeled = count;
    *rounds_out = (r0 ? r0 - 1 : 0) + (S ? *std::max_element(r2.begin(), r2.end()) : 0);
    if (err & vf::kErrTimeout) return fail(VF_ETIMEOUT, "wave solver: grid barrier timed out");
    if (err & (vf::kErrFrontier | vf::kErrCapacity)) {  // beyond the wave phase's capacities
        *fallback = true;
        return VF_EBUILD;
    }
    if (err & vf::kErrDegOverflow) return VF_EBUILD;
    if (count != n - ndrop) {  // non-empty 2-core
        if (claimed_out) {
            VF_CK(claimed_out->alloc(std::max<uint64_t>((n + 31) / 32, 1) * 4, st));
            VF_CK(vf::launch_wave_claimed(a, claimed_out->as<uint32_t>(), st));
        }
        return VF_EBUILD;
    }
    {
        PhaseTimer t(kPhAssign, st, 2);  // phase II rounds per shard, then phase I rounds
        VF_CK(vf::launch_wave_assign(a, st));
        VF_CK(cudaMemsetAsync(a.bar, 0, sizeof(vf::Bar2), st));
        vf::FuseSolveArgs f;
        std::memset(&f, 0, sizeof f);
        f.S = S;
        f.g = g;
        f.rec = a.rec;
        f.round_off = a.off1;
        f.rounds = r0 > 1 ? r0 - 1 : 0;
        f.bar = a.bar;
        f.err = a.ctr + vf::kWaveCtrErr;
        f.data = data;
        f.cell_base = cell_base;
        VF_CK(vf::launch_assign(f, st));
    }
    uint32_t e2 = 0;
    VF_CK(cudaMemcpyAsync(&e2, a.ctr + vf::kWaveCtrErr, 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    if (e2 & vf::kErrTimeout) return fail(VF_ETIMEOUT, "wave solver: assignment barrier timed out");
    return VF_OK;
}

// One attempt of the fuse-regime solver: the asynchronous solver (default) or
// the round-synchronous one. The solvers see each shard's edges sorted by the
// segment of their first vertex (a copy of loc / val). A build
// whose peel fails is checked for duplicate local signatures among the
// unpeeled edges (identical edges never peel; Sec. 4.4: the local signature
// stands for the key in its shard). A function key given with two values ends
// the build with VF_EDUP (no seed can solve it); otherwise, if there are
// duplicates, one copy of each is kept and the same attempt is solved again
// without the others (Sec. 4.5), which *dropped reports.
vf_status solve_fuse(const vf_info& in, const vf::Geom& g, const uint64_t* loc_in, const uint32_t* val_in,
                     const unsigned long long* start, uint8_t* data, cudaStream_t st, uint64_t* peeled,
                     uint64_t* rounds_out, int solver, uint64_t* dropped, uint64_t cell_base = 0) {
    // each shard's edges in the order of their first vertex's segment (locality
    // of the peeling waves); the solvers only see edge indices within a shard
    const uint64_t n = in.n_eff;
    DevBuf sloc, sval, bins;
    const uint64_t* loc = loc_in;
    const uint32_t* val = val_in;
    if (g.regime == VF_REGIME_FUSE && n > 0) {
        PhaseTimer t(kPhScatter, st, 3);  // count, scan, scatter
        VF_CK(sloc.alloc(n * 8, st));
        if (val_in) VF_CK(sval.alloc(n * 4, st));
        VF_CK(bins.alloc(vf::segment_order_bins(g, uint32_t(in.shards)) * 8, st));
        VF_CK(vf::launch_segment_order(loc_in, val_in, n, start, uint32_t(in.shards), g,
                                       bins.as<unsigned long long>(), sloc.as<uint64_t>(), sval.as<uint32_t>(), st));
        loc = sloc.as<uint64_t>();
        val = val_in ? sval.as<uint32_t>() : nullptr;
    }
    *dropped = 0;
    DevBuf drop;
    uint64_t ndrop = 0;
    for (int pass = 0;; pass++) {
        DevBuf claimed;
        const bool dedup = pass == 0;
        vf_status rs = VF_EINVAL;
        const int use = solver;  // the wave solver takes k = 3 only (wave_eligible), else the worklist solver
        bool fallback = use == VF_SOLVER_WAVE && !vf::wave_eligible(g, uint32_t(in.shards));
        if (use == VF_SOLVER_WAVE && !fallback) {
            rs = solve_wave(in, g, loc, val, start, data, st, peeled, rounds_out, cell_base, drop.as<uint32_t>(),
                            ndrop, dedup ? &claimed : nullptr, &fallback);
            if (fallback) claimed.release();
        }
        if (use == VF_SOLVER_FLOW || fallback) {
            *rounds_out = 0;
            rs = solve_flow(in, g, loc, val, start, data, st, peeled, cell_base,
                            drop.as<uint32_t>(), ndrop, dedup ? &claimed : nullptr,
                            bins.p ? bins.as<unsigned long long>() : nullptr);
        } else if (use == VF_SOLVER_ROUNDS) {
            rs = solve_rounds(in, g, loc, val, start, data, st, peeled, rounds_out, cell_base,
                              drop.as<uint32_t>(), ndrop, dedup ? &claimed : nullptr,
                              bins.p ? bins.as<unsigned long long>() : nullptr);
        }
        if (rs != VF_EBUILD || !claimed.p) return rs;
        // unpeeled edges of a failed attempt: any duplicates?
        const uint64_t unpeeled = n - *peeled;
        uint64_t cap = 1024;
        while (cap < 2 * unpeeled) cap <<= 1;
        const uint64_t words = std::max<uint64_t>((n + 31) / 32, 1);
        DevBuf table, cnt;
        VF_CK(table.alloc(cap * 8, st));
        VF_CK(cudaMemsetAsync(table.p, 0, cap * 8, st));
        VF_CK(drop.alloc(words * 4, st));
        VF_CK(cudaMemsetAsync(drop.p, 0, words * 4, st));
        VF_CK(cnt.alloc(16, st));
        VF_CK(cudaMemsetAsync(cnt.p, 0, 16, st));
        VF_CK(vf::launch_find_dups(loc, val, n, start, uint32_t(in.shards), claimed.as<uint32_t>(),
                                   table.as<unsigned long long>(), cap, drop.as<uint32_t>(),
                                   cnt.as<unsigned long long>(), nullptr, cnt.as<unsigned long long>() + 1, st));
        uint64_t c2[2] = {0, 0};
        VF_CK(cudaMemcpyAsync(c2, cnt.p, 16, cudaMemcpyDeviceToHost, st));
        VF_CK(cudaStreamSynchronize(st));
        ndrop = c2[0];
        if (c2[1]) return fail(VF_EDUP, "a key was given twice with different values");
        if (ndrop == 0) return VF_EBUILD;  // a genuine 2-core
        *dropped = ndrop;
    }
}

// Tasks of the LGE solver for the shards of one or more structures, largest
// shard first when `lpt` (longest-processing-time order balances the CTAs).
void add_lge_tasks(std::vector<vf::LgeTask>& tasks, const std::vector<unsigned long long>& start, uint64_t base_key,
                   const vf_info& in, uint8_t* data, uint32_t item, int fpb = 0, int fps = 0) {
    for (uint64_t s = 0; s < in.shards; s++) {
        vf::LgeTask t;
        std::memset(&t, 0, sizeof t);
        t.loc_off = base_key + start[s];
        t.cell_base = s * in.cells;
        t.data = data;
        t.m = uint32_t(start[s + 1] - start[s]);
        t.cells = uint32_t(in.cells);
        t.b = in.b;
        t.kind = in.kind;
        t.item = item;
        t.fpb = uint8_t(fpb);
        t.fps = uint8_t(fps);
        if (t.m > 0) tasks.push_back(t);
    }
}

// Runs the LGE solver over `tasks`; item_fail (device, one word per
// structure) receives each structure's failure bits.
vf_status run_lge_tasks(std::vector<vf::LgeTask>& tasks, bool lpt, const uint64_t* loc, const uint32_t* val,
                        uint32_t* item_fail, cudaStream_t st, uint64_t* peeled, uint64_t* core, uint32_t* err_out,
                        uint64_t* dups) {
    *peeled = *core = *dups = 0;
    *err_out = 0;
    if (tasks.empty()) return VF_OK;
    if (lpt)
        std::stable_sort(tasks.begin(), tasks.end(),
                         [](const vf::LgeTask& x, const vf::LgeTask& y) { return x.m > y.m; });
    const uint32_t n_mid = vf::lge_partition(tasks);
    uint32_t m_cap = 1, v_cap = 32;
    for (auto& t : tasks) {
        m_cap = std::max(m_cap, t.m);
        v_cap = std::max(v_cap, t.cells);
    }
    unsigned grid = vf::lge_grid();
    grid = unsigned(std::min<uint64_t>(grid, tasks.size()));
    const uint64_t per_cta = vf::lge_scratch_words_per_cta(m_cap, v_cap);
    DevBuf scratch, misc, tbuf;
    VF_CK(scratch.alloc(per_cta * grid * 4, st));
    VF_CK(misc.alloc(64 + 4 * tasks.size(), st));  // counters, then the spill list
    VF_CK(cudaMemsetAsync(misc.p, 0, 64, st));
    vf_status rs = h2d(tbuf, tasks, st);
    if (rs != VF_OK) return rs;
    vf::LgeArgs a;
    std::memset(&a, 0, sizeof a);
    a.tasks = tbuf.as<vf::LgeTask>();
    a.ntasks = uint32_t(tasks.size());
    a.loc = loc;
    a.val = val;
    a.item_fail = item_fail ? item_fail : misc.as<uint32_t>();
    a.scratch = scratch.as<uint32_t>();
    a.scratch_words_per_cta = per_cta;
    a.m_cap = m_cap;
    a.v_cap = v_cap;
    a.err = misc.as<uint32_t>();
    a.stats = misc.as<uint32_t>() + 4;
    a.spill = misc.as<uint32_t>() + 16;
    a.n_mid = n_mid;
    {
        PhaseTimer t(kPhLge, st, 3);  // medium and small configurations, then the spill list
        VF_CK(vf::launch_lge(a, grid, st));
    }
    uint32_t h[8];
    VF_CK(cudaMemcpyAsync(h, misc.p, sizeof h, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    *peeled = h[4];
    *core = h[5];
    *dups = h[7];
    *err_out = h[0];
    if (h[0] & vf::kErrTimeout) return fail(VF_ETIMEOUT, "LGE solver wait timed out");
    return VF_OK;
}

vf_status solve_lge(const vf_info& in, const std::vector<unsigned long long>& start, const uint64_t* loc,
                    const uint32_t* val, uint8_t* data, cudaStream_t st, uint64_t* peeled, uint64_t* core,
                    uint64_t* dups, int fpb = 0, int fps = 0) {
    std::vector<vf::LgeTask> tasks;
    add_lge_tasks(tasks, start, 0, in, data, 0, fpb, fps);
    uint32_t err = 0;
    vf_status rs = run_lge_tasks(tasks, true, loc, val, nullptr, st, peeled, core, &err, dups);
    if (rs != VF_OK) return rs;
    if (err & vf::kErrDupKey) return fail(VF_EDUP, "a key was given twice with different values");
    // A capacity failure is this solver's limit, not a property of the system:
    // it ends the build (a retry would give another seed than the method's).
    if (err & vf::kErrCapacity) return fail(VF_ECAPACITY, "LGE shard exceeds the per-CTA solver capacity");
    if (err & vf::kErrLgeSize)
        return fail(VF_ECAPACITY, "LGE shard needs more active variables or coefficient rows than the solver holds");
    if (err & (vf::kErrUnsolvable | vf::kErrDegOverflow)) return VF_EBUILD;
    return VF_OK;
}


// ------------------------------------------------------------ batched builds

// One non-blocking stream per host thread and device for graph capture.
cudaStream_t capture_stream() {
    thread_local std::map<int, cudaStream_t> streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto it = streams.find(dev);
    if (it != streams.end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    streams[dev] = s;
    return s;
}

// One attempt of every pending item: plan, histogram, scatter, solve.
// Built items go to out[]; failed ones to `failed`.
vf_status build_batch_once(const vf_batch_item* items, const std::vector<uint32_t>& pending,
                           const std::vector<uint32_t>& attempt, const vf_params& common, const vf_batch_opts& opts,
                           const std::vector<const uint64_t*>& kdev, const std::vector<const void*>& vdev,
                           cudaStream_t st, int dev, vf_struct** out, std::vector<uint32_t>& failed) {
    const uint32_t P = uint32_t(pending.size());
    std::vector<vf_info> info(P);
    std::vector<uint64_t> key_off(P + 1, 0);
    for (uint32_t j = 0; j < P; j++) {
        const vf_batch_item& it = items[pending[j]];
        vf_params pi = common;
        pi.kind = it.kind;
        pi.b = it.b;
        pi.key_kind = VF_KEYS_U64;
        pi.lge_threshold = opts.lge_threshold;
        pi.lge_target = opts.lge_target;
        vf_info& in = info[j];
        std::memset(&in, 0, sizeof in);
        in.n = in.n_eff = it.n;
        in.kind = it.kind;
        in.b = it.b;
        in.seed = it.seed + attempt[pending[j]];
        in.retries = int(attempt[pending[j]]);
        plan_h(pi, it.n, in);
        in.k = (in.regime == VF_REGIME_FUSE && pi.arity == 4) ? 4 : 3;
        key_off[j + 1] = key_off[j] + it.n;
    }
    const uint64_t total = key_off[P];
    // histograms; LGE structures whose largest shard is too big get more shard bits
    std::vector<vf::BatchItem> desc(P);
    std::vector<uint32_t> hist_off(P + 1, 0), counts;
    DevBuf ddesc, doff, dhist;
    VF_CK(doff.alloc(std::max<uint64_t>(P, 1) * 8, st));
    VF_CK(cudaMemcpyAsync(doff.p, key_off.data(), P * 8, cudaMemcpyHostToDevice, st));
    for (;;) {
        for (uint32_t j = 0; j < P; j++) {
            info[j].shards = uint64_t(1) << info[j].h;
            hist_off[j + 1] = hist_off[j] + uint32_t(info[j].shards);
            vf::BatchItem& d = desc[j];
            d.keys = kdev[pending[j]];
            d.vals = info[j].kind == VF_FUNC ? vdev[pending[j]] : nullptr;
            d.key_off = key_off[j];
            d.kh = vf::mix64(info[j].seed ^ vf::kLaneHi);
            d.kl = vf::mix64(info[j].seed ^ vf::kLaneLo);
            d.n = uint32_t(info[j].n);
            d.h = info[j].h;
            d.hist_off = hist_off[j];
            d.b = info[j].b;
        }
        vf_status rs = h2d(ddesc, desc, st);
        if (rs != VF_OK) return rs;
        VF_CK(dhist.alloc(std::max<uint64_t>(hist_off[P], 1) * 4, st));
        VF_CK(cudaMemsetAsync(dhist.p, 0, hist_off[P] * 4, st));
        {
            PhaseTimer t(kPhHist, st);
            VF_CK(vf::launch_batch_hist(ddesc.as<vf::BatchItem>(), doff.as<uint64_t>(), P, total, dhist.as<uint32_t>(),
                                        st));
        }
        counts.assign(hist_off[P], 0);
        VF_CK(cudaMemcpyAsync(counts.data(), dhist.p, hist_off[P] * 4, cudaMemcpyDeviceToHost, st));
        VF_CK(cudaStreamSynchronize(st));
        bool again = false;
        for (uint32_t j = 0; j < P; j++) {
            uint64_t M = 0;
            for (uint32_t k = hist_off[j]; k < hist_off[j + 1]; k++) M = std::max<uint64_t>(M, counts[k]);
            info[j].M = M;
            if (info[j].regime == VF_REGIME_LGE && M > common.lge_max_shard && info[j].h < 30) {
                info[j].h++;
                again = true;
            }
        }
        if (!again) break;
    }
    // geometry, data arrays, scatter cursors
    std::vector<uint8_t*> data(P, nullptr);
    auto free_data = [&]() {
        for (auto* d : data)
            if (d) cudaFreeAsync(d, st);
    };
    std::vector<unsigned long long> cursor(hist_off[P]);
    for (uint32_t j = 0; j < P; j++) {
        vf_info& in = info[j];
        geometry(in);
        if ((in.regime != VF_REGIME_LGE && in.M >= (uint64_t(1) << 27)) || in.total_cells >= (uint64_t(1) << 32)) {
            free_data();
            return fail(VF_ECAPACITY, "batched structure exceeds a size limit");
        }
        if (cudaMallocAsync(reinterpret_cast<void**>(&data[j]), in.data_bytes + 16, st) != cudaSuccess) {
            free_data();
            return fail(VF_ENOMEM, "batched data allocation failed");
        }
        VF_CK(cudaMemsetAsync(data[j], 0, in.data_bytes + 16, st));
        unsigned long long run = key_off[j];
        for (uint32_t k = hist_off[j]; k < hist_off[j + 1]; k++) {
            cursor[k] = run;
            run += counts[k];
        }
    }
    DevBuf dcur, loc, val, fails;
    vf_status rs = h2d(dcur, cursor, st);
    if (rs != VF_OK) return free_data(), rs;
    VF_CK(loc.alloc(std::max<uint64_t>(total, 1) * 8, st));
    VF_CK(val.alloc(std::max<uint64_t>(total, 1) * 4, st));
    VF_CK(fails.alloc(std::max<uint64_t>(P, 1) * 8, st));  // failure bits, then dropped duplicates
    uint32_t* dups_dev = fails.as<uint32_t>() + std::max<uint64_t>(P, 1);
    // LGE tasks of every LGE structure, one solver launch for all of them
    std::vector<vf::LgeTask> tasks;
    for (uint32_t j = 0; j < P; j++) {
        if (info[j].regime != VF_REGIME_LGE) continue;
        std::vector<unsigned long long> start(info[j].shards + 1, 0);
        for (uint64_t s2 = 0; s2 < info[j].shards; s2++) start[s2 + 1] = start[s2] + counts[hist_off[j] + s2];
        add_lge_tasks(tasks, start, key_off[j], info[j], data[j], j);
    }
    if (opts.lpt)
        std::stable_sort(tasks.begin(), tasks.end(),
                         [](const vf::LgeTask& x, const vf::LgeTask& y) { return x.m > y.m; });
    const uint32_t n_mid = vf::lge_partition(tasks, opts.small_cta_keys);
    uint32_t m_cap = 1, v_cap = 32;
    for (auto& t : tasks) {
        m_cap = std::max(m_cap, t.m);
        v_cap = std::max(v_cap, t.cells);
    }
    unsigned grid = vf::lge_grid();
    grid = unsigned(std::min<uint64_t>(grid, std::max<size_t>(tasks.size(), 1)));
    const uint64_t per_cta = vf::lge_scratch_words_per_cta(m_cap, v_cap);
    DevBuf scratch, misc, tbuf;
    VF_CK(scratch.alloc(per_cta * grid * 4, st));
    VF_CK(misc.alloc(64 + 4 * tasks.size(), st));  // counters, then the spill list
    rs = h2d(tbuf, tasks, st);
    if (rs != VF_OK) return free_data(), rs;
    vf::LgeArgs a;
    std::memset(&a, 0, sizeof a);
    a.tasks = tbuf.as<vf::LgeTask>();
    a.ntasks = uint32_t(tasks.size());
    a.loc = loc.as<uint64_t>();
    a.val = val.as<uint32_t>();
    a.item_fail = fails.as<uint32_t>();
    a.item_dup = dups_dev;
    a.scratch = scratch.as<uint32_t>();
    a.scratch_words_per_cta = per_cta;
    a.m_cap = m_cap;
    a.v_cap = v_cap;
    a.err = misc.as<uint32_t>();
    a.stats = misc.as<uint32_t>() + 4;
    a.spill = misc.as<uint32_t>() + 16;
    a.n_mid = n_mid;
    // scatter + solver: one CUDA graph (or plain launches)
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(fails.p, 0, std::max<uint64_t>(P, 1) * 8, q);
        if (e == cudaSuccess) e = cudaMemsetAsync(misc.p, 0, 64, q);
        if (e == cudaSuccess)
            e = vf::launch_batch_scatter(ddesc.as<vf::BatchItem>(), doff.as<uint64_t>(), P, total,
                                         dcur.as<unsigned long long>(), loc.as<uint64_t>(), val.as<uint32_t>(), q);
        if (e == cudaSuccess) e = vf::launch_lge(a, grid, q);
        return e;
    };
    if (opts.use_graph) {
        // Captured on a private stream (the legacy default stream cannot be
        // captured); the graph then runs in order on the caller's stream.
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cs = capture_stream();
        if (!cs) return free_data(), fail(VF_ECUDA, "could not create the capture stream");
        VF_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue(cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            free_data();
            return fail(VF_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) {
            PhaseTimer t(kPhLge, st, 4);  // scatter + three solver configurations
            e = cudaGraphLaunch(exec, st);
        }
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            free_data();
            return fail(VF_ECUDA, std::string("graph launch failed: ") + cudaGetErrorString(e));
        }
    } else {
        PhaseTimer t(kPhLge, st, 4);  // scatter + three solver configurations
        cudaError_t e = enqueue(st);
        if (e != cudaSuccess) {
            free_data();
            return fail(VF_ECUDA, std::string("batched solve launch failed: ") + cudaGetErrorString(e));
        }
    }
    std::vector<uint32_t> fail_bits(P, 0), dups(P, 0);
    VF_CK(cudaMemcpyAsync(fail_bits.data(), fails.p, P * 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaMemcpyAsync(dups.data(), dups_dev, P * 4, cudaMemcpyDeviceToHost, st));
    VF_CK(cudaStreamSynchronize(st));
    for (uint32_t j = 0; j < P; j++)
        if (info[j].regime == VF_REGIME_LGE) info[j].n_eff -= dups[j];
    // fuse-regime structures (above the threshold): one solver each
    for (uint32_t j = 0; j < P; j++) {
        if (info[j].regime == VF_REGIME_LGE) continue;  // fuse and MWHC: the peeling solvers
        std::vector<unsigned long long> start(info[j].shards + 1, 0);
        for (uint64_t s2 = 0; s2 < info[j].shards; s2++) start[s2 + 1] = start[s2] + counts[hist_off[j] + s2];
        DevBuf dstart;
        rs = h2d(dstart, start, st);
        if (rs != VF_OK) return free_data(), rs;
        uint64_t peeled = 0, rounds = 0, dropped = 0;
        rs = solve_fuse(info[j], make_geom(info[j]), loc.as<uint64_t>() + key_off[j],
                        info[j].kind == VF_FUNC ? val.as<uint32_t>() + key_off[j] : nullptr,
                        dstart.as<unsigned long long>(), data[j], st, &peeled, &rounds, common.fuse_solver,
                        &dropped);
        if (rs == VF_EBUILD) fail_bits[j] |= vf::kErrUnsolvable;
        else if (rs != VF_OK) return free_data(), rs;
        info[j].peeled = peeled;
        info[j].rounds = rounds;
        info[j].n_eff -= dropped;
    }
    VF_CK(cudaStreamSynchronize(st));
    for (uint32_t j = 0; j < P; j++) {
        if (fail_bits[j] & vf::kErrDupKey) {
            free_data();
            return fail(VF_EDUP, "vf_build_batch: structure " + std::to_string(pending[j]) +
                                     " has a key given twice with different values");
        }
        if (fail_bits[j] & (vf::kErrCapacity | vf::kErrLgeSize)) {
            free_data();
            return fail(VF_ECAPACITY, "batched LGE shard exceeds the solver capacity");
        }
        if (fail_bits[j]) {
            cudaFreeAsync(data[j], st);
            data[j] = nullptr;
            failed.push_back(pending[j]);
            continue;
        }
        vf_struct* sp = new vf_struct;
        sp->info = info[j];
        sp->geom = make_geom(info[j]);
        sp->data = data[j];
        sp->device = dev;
        out[pending[j]] = sp;
        data[j] = nullptr;
    }
    return VF_OK;
}

struct TuneKey {
    uint32_t count;
    uint64_t total, nmax;
    bool operator<(const TuneKey& o) const {
        return count != o.count ? count < o.count : total != o.total ? total < o.total : nmax < o.nmax;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, vf_batch_opts> g_tune_cache;

struct ResumeOpts {
    const char* path;
    uint64_t group_keys;
    uint32_t max_groups;
};

uint64_t digest_words(const uint64_t* w, size_t n) {
    uint64_t h = 0x6A09E667F3BCC908ull;
    for (size_t i = 0; i < n; i++) h = vf::mix64(h ^ w[i]) + uint64_t(i);
    return h;
}

// Parameters that shape the structure (the solver choice does not).
uint64_t params_digest(const vf_params& p, uint64_t group_keys) {
    uint64_t e, t;
    std::memcpy(&e, &p.eps, 8);
    std::memcpy(&t, &p.eta, 8);
    const uint64_t w[] = {uint64_t(p.kind), uint64_t(p.b), uint64_t(p.key_kind), uint64_t(p.mode), e, t,
                          p.lge_threshold, p.lge_target, p.lge_max_shard, group_keys, uint64_t(p.arity)};
    return digest_words(w, sizeof w / sizeof w[0]);
}

// Byte range of the data array holding cells [c0, c1) (bit arrays: rounded
// outward; the last group also takes the pad word).
void cell_bytes(const vf_info& in, uint64_t c0, uint64_t c1, bool last, uint64_t* lo, uint64_t* hi) {
    const uint64_t b = uint64_t(in.b);
    *lo = c0 * b / 8;
    *hi = last ? in.data_bytes : (c1 * b + 7) / 8;
}

// Checkpoint file of a resumable build: the serialized form with
// groups_done < groups_total until the last shard group is written.
struct Checkpoint {
    std::FILE* f = nullptr;
    vf::StoreHeader h{};
    ~Checkpoint() {
        if (f) std::fclose(f);
    }
    vf_status write_header() {
        std::vector<uint8_t> buf(vf::kStoreHeaderBytes);
        vf::store_encode(h, buf.data());
        if (!vf::file_write_at(f, 0, buf.data(), buf.size()) || std::fflush(f) != 0)
            return fail(VF_EIO, "checkpoint: writing the header failed");
        return VF_OK;
    }
    uint64_t group_keys = 0;
    vf_status open(const char* path, const vf_info& in, const vf_params& p, const std::vector<uint32_t>& counts,
                   const std::vector<uint32_t>& group, uint8_t* data, cudaStream_t st, size_t* k0) {
        std::vector<uint64_t> cw(counts.begin(), counts.end());
        const uint64_t cd = digest_words(cw.data(), cw.size());
        const uint64_t pd = params_digest(p, group_keys);
        *k0 = 0;
        f = std::fopen(path, "r+b");
        if (f) {
            std::vector<uint8_t> buf(vf::kStoreHeaderBytes);
            vf::StoreHeader old;
            const bool same = vf::file_read_at(f, 0, buf.data(), buf.size()) &&
                              vf::store_decode(buf.data(), buf.size(), old) && old.info.seed == in.seed &&
                              old.info.n == in.n && old.info.kind == in.kind && old.info.b == in.b &&
                              old.info.regime == in.regime && old.info.h == in.h && old.info.M == in.M &&
                              old.info.cells == in.cells && old.info.data_bytes == in.data_bytes &&
                              old.info.k == in.k &&
                              old.counts_digest == cd && old.params_digest == pd &&
                              old.groups_total == group.size() - 1 && old.key_kind == p.key_kind &&
                              old.groups_done < old.groups_total;
            if (same) {
                h = old;
                *k0 = size_t(h.groups_done);
                if (*k0 > 0) {
                    uint64_t lo, hi;
                    cell_bytes(in, 0, uint64_t(group[*k0]) * in.cells, false, &lo, &hi);
                    VF_CK(cudaStreamSynchronize(st));  // the data array was zeroed on `st`
                    bool io = true;
                    VF_CK(vf::file_to_device(f, vf::kStoreHeaderBytes, data, hi, &io));
                    if (!io) return fail(VF_EIO, "checkpoint: reading completed shard groups failed");
                }
                return VF_OK;
            }
            std::fclose(f);
            f = nullptr;
        }
        f = std::fopen(path, "w+b");
        if (!f) return fail(VF_EIO, std::string("checkpoint: cannot create ") + path);
        std::memset(&h, 0, sizeof h);
        h.info = in;
        h.info.peeled = h.info.core = h.info.rounds = 0;
        h.groups_total = group.size() - 1;
        h.groups_done = 0;
        h.counts_digest = cd;
        h.params_digest = pd;
        h.key_kind = p.key_kind;
        const uint8_t zero = 0;
        if (in.data_bytes > 0 &&
            !vf::file_write_at(f, vf::kStoreHeaderBytes + in.data_bytes - 1, &zero, 1))  // size the file
            return fail(VF_EIO, "checkpoint: sizing the file failed");
        return write_header();
    }
    vf_status save_group(const vf_info& in, const std::vector<uint32_t>& group, size_t k, const uint8_t* data,
                         uint64_t peeled, uint64_t core, uint64_t rounds, uint64_t dropped) {
        uint64_t lo, hi;
        cell_bytes(in, uint64_t(group[k]) * in.cells, uint64_t(group[k + 1]) * in.cells, k + 2 == group.size(), &lo,
                   &hi);
        bool io = true;
        VF_CK(vf::device_to_file(f, vf::kStoreHeaderBytes + lo, data + lo, hi - lo, &io));
        if (!io) return fail(VF_EIO, "checkpoint: writing a shard group failed");
        h.groups_done = k + 1;
        h.info.peeled = peeled, h.info.core = core, h.info.rounds = rounds;
        h.dropped = dropped;
        return write_header();
    }
    vf_status finish(const vf_info& in) {
        h.info = in;
        return write_header();
    }
};

// The attempt (seed - params.seed) an unfinished checkpoint of this build was
// written by, or 0: every call of a resumable build starts there, so the
// progress of a retried attempt is not lost.
int checkpoint_attempt(const ResumeOpts* ro, const vf_params& p, uint64_t n) {
    std::FILE* f = std::fopen(ro->path, "rb");
    if (!f) return 0;
    std::vector<uint8_t> buf(vf::kStoreHeaderBytes);
    vf::StoreHeader h;
    int a = 0;
    if (vf::file_read_at(f, 0, buf.data(), buf.size()) && vf::store_decode(buf.data(), buf.size(), h) &&
        h.groups_done < h.groups_total && h.info.n == n && h.key_kind == p.key_kind &&
        h.params_digest == params_digest(p, ro->group_keys) && h.info.seed >= p.seed &&
        h.info.seed - p.seed <= uint64_t(p.max_retries))
        a = int(h.info.seed - p.seed);
    std::fclose(f);
    return a;
}

// One 32-bit slice of a structure wider than 32 bits: the fingerprint bits
// it holds (filters).
struct SliceOpts {
    int fpb, fps;
};

vf_status build_impl(const void* keys, const uint64_t* offsets, const void* values, uint64_t n,
                     const vf_params* params, void* stream, vf_struct** out, const ResumeOpts* ro,
                     const SliceOpts* so = nullptr);

vf_status build_impl(const void* keys, const uint64_t* offsets, const void* values, uint64_t n,
                     const vf_params* params, void* stream, vf_struct** out, const ResumeOpts* ro,
                     const SliceOpts* so) {
    g_last_error.clear();
    if (!params || !out) return fail(VF_EINVAL, "vf_build: NULL params or out");
    *out = nullptr;
    const vf_params p = *params;
    if (p.b < 1 || p.b > 32) return fail(VF_EINVAL, "b must be in 1..64 (above 32 only through vf_build)");
    if (p.kind != VF_FUNC && p.kind != VF_FILTER) return fail(VF_EINVAL, "bad kind");
    if (p.key_kind != VF_KEYS_U64 && p.key_kind != VF_KEYS_BYTES) return fail(VF_EINVAL, "bad key_kind");
    if (n > 0 && !keys) return fail(VF_EINVAL, "keys is NULL");
    if (p.key_kind == VF_KEYS_BYTES && !offsets) return fail(VF_EINVAL, "offsets is NULL");
    if (p.kind == VF_FUNC && n > 0 && !values) return fail(VF_EINVAL, "a function needs values");
    if (!(p.eps > 0.0) || !(p.eta > 0.0 && p.eta < 1.0) || p.max_retries < 0 || p.lge_target == 0 ||
        p.lge_max_shard < 2 || p.mode < VF_MODE_AUTO || p.mode > VF_MODE_MWHC || p.fuse_solver < VF_SOLVER_FLOW ||
        p.fuse_solver > VF_SOLVER_WAVE || (p.arity != 3 && p.arity != 4))
        return fail(VF_EINVAL, "bad eps / eta / retries / LGE sizes / mode / fuse solver / arity");
    for (const auto& pw : {std::make_pair(keys, "keys"), std::make_pair(static_cast<const void*>(offsets), "offsets"),
                           std::make_pair(values, "values")}) {
        const vf_status cs = vf::check_here(pw.first, pw.second);
        if (cs != VF_OK) return cs;
    }
    // More than 2^30 keys: only 64-bit keys in the fuse or MWHC regime, built
    // one shard group (<= 2^30 keys) at a time.
    const bool big = n > (uint64_t(1) << 30);
    if (big && (p.key_kind != VF_KEYS_U64 || p.mode == VF_MODE_LGE || n < p.lge_threshold || n > (uint64_t(1) << 36)))
        return fail(VF_ECAPACITY, "above 2^30 keys: 64-bit keys, fuse or MWHC regime, at most 2^36 keys");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    VF_CK(cudaGetDevice(&dev));
    keep_pool_warm(dev);

    Staged in_keys;
    vf_status rs = stage_keys(p.key_kind, keys, offsets, n, st, in_keys);
    if (rs != VF_OK) return rs;
    const void* vals_dev = nullptr;
    if (p.kind == VF_FUNC && n > 0) {
        if (on_device(values)) {
            vals_dev = values;
        } else {
            VF_CK(in_keys.vbuf.alloc(n * value_bytes(p.b), st));
            VF_CK(cudaMemcpyAsync(in_keys.vbuf.p, values, n * value_bytes(p.b), cudaMemcpyHostToDevice, st));
            vals_dev = in_keys.vbuf.p;
        }
    }

    DevBuf hist, sigs, loc, val, startb, cursor, data;
    if (p.key_kind == VF_KEYS_BYTES) VF_CK(sigs.alloc(n * sizeof(vf::Sig), st));

    vf_status last = VF_EBUILD;
    const int first_attempt = ro ? checkpoint_attempt(ro, p, n) : 0;
    for (int attempt = first_attempt; attempt <= p.max_retries; attempt++) {
        vf_info in;
        std::memset(&in, 0, sizeof in);
        in.n = in.n_eff = n;
        in.kind = p.kind;
        in.b = p.b;
        in.seed = p.seed + uint64_t(attempt);
        in.retries = attempt;
        plan_h(p, n, in);
        in.k = (in.regime == VF_REGIME_FUSE && p.arity == 4) ? 4 : 3;
        std::vector<uint32_t> counts;
        for (;;) {
            in.shards = uint64_t(1) << in.h;
            vf::Geom g0 = make_geom(in);
            VF_CK(hist.alloc(in.shards * 4, st));
            VF_CK(cudaMemsetAsync(hist.p, 0, in.shards * 4, st));
            {
                PhaseTimer t(kPhHist, st);
                VF_CK(vf::launch_hist(p.key_kind, in_keys.keys, in_keys.offs, n, g0, hist.as<uint32_t>(),
                                      sigs.as<vf::Sig>(), st));
            }
            counts.assign(in.shards, 0);
            VF_CK(cudaMemcpyAsync(counts.data(), hist.p, in.shards * 4, cudaMemcpyDeviceToHost, st));
            VF_CK(cudaStreamSynchronize(st));
            in.M = *std::max_element(counts.begin(), counts.end());
            if (in.regime == VF_REGIME_LGE && in.M > p.lge_max_shard && in.h < 40) {
                in.h++;
                continue;
            }
            break;
        }
        geometry(in);
        if (in.regime != VF_REGIME_LGE && in.M >= (uint64_t(1) << 27))
            return fail(VF_ECAPACITY, "fuse / MWHC shard above 2^27 keys");
        if (in.regime == VF_REGIME_LGE && in.M > p.lge_max_shard)
            return fail(VF_ECAPACITY, "LGE shard above lge_max_shard");
        const vf::Geom g = make_geom(in, so ? so->fpb : 0, so ? so->fps : 0);
        // shard groups: consecutive shards with at most 2^30 keys (or the resumable
        // build's group size) and 2^32 cells each
        const uint64_t group_cap =
            ro && ro->group_keys ? std::min<uint64_t>(ro->group_keys, uint64_t(1) << 30) : uint64_t(1) << 30;
        std::vector<uint32_t> group{0};
        {
            uint64_t keys_in = 0, cells_in = 0;
            for (uint32_t s = 0; s < in.shards; s++) {
                if (s > group.back() && (keys_in + counts[s] > group_cap ||
                                         cells_in + in.cells >= (uint64_t(1) << 32))) {
                    group.push_back(s);
                    keys_in = cells_in = 0;
                }
                keys_in += counts[s];
                cells_in += in.cells;
            }
            group.push_back(uint32_t(in.shards));
        }
        if (group.size() > 2 && in.regime == VF_REGIME_LGE)
            return fail(VF_ECAPACITY, "more than 2^30 keys or 2^32 cells in the LGE regime");
        uint64_t group_max = 0;
        for (size_t k = 0; k + 1 < group.size(); k++) {
            uint64_t sum = 0;
            for (uint32_t s = group[k]; s < group[k + 1]; s++) sum += counts[s];
            group_max = std::max(group_max, sum);
        }
        if (loc.bytes < std::max<uint64_t>(group_max, 1) * 8) VF_CK(loc.alloc(std::max<uint64_t>(group_max, 1) * 8, st));
        if (p.kind == VF_FUNC && val.bytes < std::max<uint64_t>(group_max, 1) * 4)
            VF_CK(val.alloc(std::max<uint64_t>(group_max, 1) * 4, st));
        VF_CK(data.alloc(in.data_bytes + 16, st));
        VF_CK(cudaMemsetAsync(data.p, 0, in.data_bytes + 16, st));
        VF_CK(cursor.alloc(in.shards * 8, st));
        uint64_t peeled = 0, core = 0, rounds = 0;
        rs = VF_OK;
        uint64_t dropped = 0;
        std::vector<unsigned long long> start;
        // resumable build: continue from this attempt's checkpoint, or start one
        Checkpoint ck;
        size_t k0 = 0;
        if (ro) {
            ck.group_keys = ro->group_keys;
            rs = ck.open(ro->path, in, p, counts, group, data.as<uint8_t>(), st, &k0);
            if (rs != VF_OK) return rs;
            peeled = ck.h.info.peeled, core = ck.h.info.core, rounds = ck.h.info.rounds, dropped = ck.h.dropped;
        }
        uint32_t groups_here = 0;
        for (size_t k = k0; k + 1 < group.size() && rs == VF_OK; k++) {
            const uint32_t g0s = group[k], g1s = group[k + 1];
            vf_info gi = in;
            gi.shards = g1s - g0s;
            start.assign(gi.shards + 1, 0);
            for (uint32_t s = g0s; s < g1s; s++) start[s - g0s + 1] = start[s - g0s] + counts[s];
            gi.n_eff = start[gi.shards];
            gi.total_cells = gi.shards * in.cells;
            // cursors of the group's shards start at the group-local shard starts
            std::vector<unsigned long long> cur(in.shards, 0);
            for (uint32_t s = g0s; s < g1s; s++) cur[s] = start[s - g0s];
            VF_CK(cudaMemcpyAsync(cursor.p, cur.data(), in.shards * 8, cudaMemcpyHostToDevice, st));
            rs = h2d(startb, start, st);
            if (rs != VF_OK) return rs;
            {
                PhaseTimer t(kPhScatter, st);
                VF_CK(vf::launch_scatter(static_cast<const uint64_t*>(in_keys.keys), sigs.as<vf::Sig>(), vals_dev, n,
                                         g, cursor.as<unsigned long long>(), loc.as<uint64_t>(), val.as<uint32_t>(),
                                         g0s, g1s, st));
            }
            uint64_t pe = 0, co = 0, rn = 0, dr = 0;
            if (in.regime != VF_REGIME_LGE)  // fuse graphs and MWHC hypergraphs peel the same way
                rs = solve_fuse(gi, g, loc.as<uint64_t>(), p.kind == VF_FUNC ? val.as<uint32_t>() : nullptr,
                                startb.as<unsigned long long>(), data.as<uint8_t>(), st, &pe, &rn,
                                p.fuse_solver, &dr, uint64_t(g0s) * in.cells);
            else
                rs = solve_lge(in, start, loc.as<uint64_t>(), p.kind == VF_FUNC ? val.as<uint32_t>() : nullptr,
                               data.as<uint8_t>(), st, &pe, &co, &dr, so ? so->fpb : 0, so ? so->fps : 0);
            peeled += pe;
            core += co;
            rounds += rn;
            dropped += dr;
            if (rs == VF_OK && ck.f) {
                rs = ck.save_group(in, group, k, data.as<uint8_t>(), peeled, core, rounds, dropped);
                if (rs != VF_OK) return rs;
                if (ro->max_groups && ++groups_here == ro->max_groups && k + 2 < group.size()) {
                    char msg[96];
                    std::snprintf(msg, sizeof msg, "checkpoint holds %zu of %zu shard groups", k + 1,
                                  group.size() - 1);
                    return fail(VF_EAGAIN, msg);
                }
            }
        }
        in.peeled = peeled;
        const uint64_t n_all = in.n_eff;
        in.n_eff = n_all - dropped;
        in.core = in.regime == VF_REGIME_LGE ? core : 0;
        in.rounds = rounds;
        if (rs == VF_OK && attempt < g_debug_fail_attempts.load()) rs = VF_EBUILD;  // test hook
        if (rs == VF_OK) {
            VF_CK(cudaStreamSynchronize(st));
            if (ck.f) {
                rs = ck.finish(in);
                if (rs != VF_OK) return rs;
            }
            vf_struct* s = new vf_struct;
            s->info = in;
            s->geom = g;
            s->data = data.as<uint8_t>();
            s->device = dev;
            data.p = nullptr;  // ownership moves to the structure
            *out = s;
            return VF_OK;
        }
        in.n_eff = n_all;
        last = rs;
        if (rs != VF_EBUILD) return rs;
    }
    return fail(last, "all attempts failed (seed .. seed+max_retries)");
}

// Values wider than 32 bits (b = 33..64): the system is linear over GF(2)^b,
// so an attempt solves the low 32 bit planes and the high b-32 bit planes as
// two slices on the same hypergraph and seed; it fails (next seed) if either
// does, as the full system would. The slices' cells are then packed into one
// b-bit array.
vf_status build_wide(const void* keys, const uint64_t* offsets, const void* values, uint64_t n, const vf_params& p,
                     void* stream, vf_struct** out) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int b = p.b, hb = b - 32;
    vf_status cs = vf::check_here(values, "values");
    if (cs != VF_OK) return cs;
    DevBuf v64, vlo, vhi;
    if (p.kind == VF_FUNC && n > 0) {
        const uint64_t* vdev = static_cast<const uint64_t*>(values);
        if (!on_device(values)) {
            VF_CK(v64.alloc(n * 8, st));
            VF_CK(cudaMemcpyAsync(v64.p, values, n * 8, cudaMemcpyHostToDevice, st));
            vdev = v64.as<uint64_t>();
        }
        VF_CK(vlo.alloc(n * 4, st));
        VF_CK(vhi.alloc(n * value_bytes(hb), st));
        VF_CK(vf::launch_split64(vdev, n, b, vlo.as<uint32_t>(), vhi.p, st));
    }
    int dev = 0;
    VF_CK(cudaGetDevice(&dev));
    vf_status last = VF_EBUILD;
    for (int attempt = 0; attempt <= p.max_retries; attempt++) {
        vf_params ps = p;
        ps.seed = p.seed + uint64_t(attempt);
        ps.max_retries = 0;
        ps.b = 32;
        vf_struct* lo = nullptr;
        vf_struct* hi = nullptr;
        const SliceOpts slo{b, 0}, shi{b, 32};
        vf_status rs = build_impl(keys, offsets, vlo.p, n, &ps, stream, &lo, nullptr, &slo);
        if (rs == VF_OK) {
            ps.b = hb;
            rs = build_impl(keys, offsets, vhi.p, n, &ps, stream, &hi, nullptr, &shi);
        }
        if (rs == VF_OK && (lo->info.total_cells != hi->info.total_cells || lo->info.h != hi->info.h)) {
            vf_free(lo);
            vf_free(hi);
            return fail(VF_ECUDA, "wide build: the two slices disagree on the geometry");
        }
        if (rs == VF_OK) {
            vf_info in = lo->info;
            in.b = b;
            in.seed = ps.seed;
            in.retries = attempt;
            in.data_bytes = b == 64 ? in.total_cells * 8 : ((in.total_cells * uint64_t(b) + 63) / 64 + 1) * 8;
            uint8_t* d = nullptr;
            cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), in.data_bytes + 16, st);
            if (e == cudaSuccess)
                e = vf::launch_pack_wide(reinterpret_cast<const uint32_t*>(lo->data), hi->data, in.total_cells, b,
                                         in.data_bytes / 8, reinterpret_cast<uint64_t*>(d), st);
            if (e == cudaSuccess) e = cudaMemsetAsync(d + in.data_bytes, 0, 16, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            vf_free(lo);
            vf_free(hi);
            if (e != cudaSuccess) {
                if (d) cudaFree(d);
                return fail(VF_ECUDA, std::string("wide build: packing failed: ") + cudaGetErrorString(e));
            }
            vf_struct* s = new vf_struct;
            s->info = in;
            s->geom = make_geom(in);
            s->data = d;
            s->device = dev;
            *out = s;
            return VF_OK;
        }
        if (lo) vf_free(lo);
        if (hi) vf_free(hi);
        last = rs;
        if (rs != VF_EBUILD) return rs;
    }
    return fail(last, "all attempts failed (seed .. seed+max_retries)");
}

}  // namespace

vf::Geom vf::geom_of(const vf_info& in) { return make_geom(in); }

vf::MemWhere vf::mem_where(const void* p) {
    if (!p) return MemWhere::kHost;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return MemWhere::kHost;
    }
    if (a.type == cudaMemoryTypeManaged) return MemWhere::kHere;
    if (a.type != cudaMemoryTypeDevice) return MemWhere::kHost;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return MemWhere::kElsewhere;
    }
    return a.device == cur ? MemWhere::kHere : MemWhere::kElsewhere;
}

vf_status vf::check_here(const void* p, const char* what) {
    if (mem_where(p) != MemWhere::kElsewhere) return VF_OK;
    return fail(VF_EINVAL, std::string(what) + " is device memory of another device than the current one");
}

int vf::debug_fail_attempts() { return g_debug_fail_attempts.load(); }

void vf::set_last_error(const char* msg) { g_last_error = msg; }

extern "C" {

void vf_params_default(vf_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->kind = VF_FUNC;
    p->b = 8;
    p->key_kind = VF_KEYS_U64;
    p->mode = VF_MODE_AUTO;
    p->max_retries = 16;
    p->seed = 0;
    p->eps = 0.001;
    p->eta = 0.1;
    p->lge_threshold = 800000;
    p->lge_target = 16384;
    p->lge_max_shard = 24576;
    p->fuse_solver = VF_SOLVER_FLOW;
    p->arity = 3;
}

const char* vf_last_error(void) { return g_last_error.c_str(); }

vf_status vf_plan(const vf_params* p, uint64_t n, uint64_t M, vf_info* out) {
    if (!p || !out) return fail(VF_EINVAL, "vf_plan: NULL argument");
    if (p->mode < VF_MODE_AUTO || p->mode > VF_MODE_MWHC) return fail(VF_EINVAL, "vf_plan: bad mode");
    vf_info in;
    std::memset(&in, 0, sizeof in);
    in.n = in.n_eff = n;
    in.kind = p->kind;
    in.b = p->b;
    in.seed = p->seed;
    if (p->arity != 3 && p->arity != 4) return fail(VF_EINVAL, "vf_plan: arity must be 3 or 4");
    plan_h(*p, n, in);
    in.k = (in.regime == VF_REGIME_FUSE && p->arity == 4) ? 4 : 3;
    in.shards = uint64_t(1) << in.h;
    in.M = M;
    geometry(in);
    *out = in;
    return VF_OK;
}

vf_status vf_build(const void* keys, const uint64_t* offsets, const void* values, uint64_t n,
                   const vf_params* params, void* stream, vf_struct** out) {
    if (params && out && params->b > 32 && params->b <= 64) {
        g_last_error.clear();
        *out = nullptr;
        if (params->kind == VF_FUNC && n > 0 && !values) return fail(VF_EINVAL, "a function needs values");
        return build_wide(keys, offsets, values, n, *params, stream, out);
    }
    return build_impl(keys, offsets, values, n, params, stream, out, nullptr);
}

vf_status vf_build_resumable(const void* keys, const uint64_t* offsets, const void* values, uint64_t n,
                             const vf_params* params, const char* checkpoint, uint64_t group_keys,
                             uint32_t max_groups, void* stream, vf_struct** out) {
    if (!checkpoint) return fail(VF_EINVAL, "vf_build_resumable: NULL checkpoint path");
    if (params && params->b > 32) return fail(VF_EINVAL, "vf_build_resumable: b above 32 (use vf_build)");
    ResumeOpts ro{checkpoint, group_keys, max_groups};
    return build_impl(keys, offsets, values, n, params, stream, out, &ro);
}

// Two non-blocking streams per host thread and device for pipelined queries.
bool pipe_streams(cudaStream_t out[2]) {
    thread_local std::map<int, std::pair<cudaStream_t, cudaStream_t>> streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    auto it = streams.find(dev);
    if (it == streams.end()) {
        cudaStream_t a = nullptr, b = nullptr;
        if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess) return false;
        if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
            cudaStreamDestroy(a);
            return false;
        }
        it = streams.emplace(dev, std::make_pair(a, b)).first;
    }
    out[0] = it->second.first;
    out[1] = it->second.second;
    return true;
}

// Keys per chunk of a pipelined query (64 MB of 64-bit keys).
constexpr uint64_t kPipeChunk = uint64_t(1) << 23;

// Queries of 64-bit keys of which the keys or the outputs (or both) are host
// memory: chunks of kPipeChunk keys alternate between two streams, each chunk
// copied in (one cudaMemcpyAsync), probed, and copied out on its stream, so
// the host-to-device copy of one chunk overlaps the probe of the previous one
// and the device-to-host copy of the one before. Each stream reuses its own
// staging slot, so stream order alone keeps a slot from being overwritten
// while in use. Ordered after earlier work on `st`; `st` waits for both.
vf_status query_pipelined(const vf_struct* s, const uint64_t* keys, bool keys_dev, uint64_t m, void* out,
                          bool out_dev, size_t ob, cudaStream_t st) {
    cudaStream_t q[2];
    if (!pipe_streams(q)) return fail(VF_ECUDA, "vf_query: could not create the pipeline streams");
    const uint64_t chunk = std::min(m, kPipeChunk);
    DevBuf kb, obuf;
    if (!keys_dev) VF_CK(kb.alloc(2 * chunk * 8, st));
    if (!out_dev) VF_CK(obuf.alloc(2 * chunk * ob, st));
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (auto& e : ev) VF_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    auto destroy = [&]() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    };
    cudaError_t e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q[0], ev[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q[1], ev[0], 0);
    const uint64_t nchunks = (m + chunk - 1) / chunk;
    {
        PhaseTimer t(kPhQuery, st, int(nchunks));
        for (uint64_t c = 0; c < nchunks && e == cudaSuccess; c++) {
            const uint64_t i0 = c * chunk, len = std::min(chunk, m - i0);
            const int j = int(c & 1);
            const uint64_t* kd = keys_dev ? keys + i0 : kb.as<uint64_t>() + uint64_t(j) * chunk;
            if (!keys_dev) e = cudaMemcpyAsync(const_cast<uint64_t*>(kd), keys + i0, len * 8, cudaMemcpyHostToDevice, q[j]);
            uint8_t* od = out_dev ? static_cast<uint8_t*>(out) + i0 * ob : obuf.as<uint8_t>() + uint64_t(j) * chunk * ob;
            if (e == cudaSuccess) e = vf::launch_query(VF_KEYS_U64, kd, nullptr, len, s->geom, s->data, od, q[j]);
            if (e == cudaSuccess && !out_dev)
                e = cudaMemcpyAsync(static_cast<uint8_t*>(out) + i0 * ob, od, len * ob, cudaMemcpyDeviceToHost, q[j]);
        }
        // `st` (and with it the staging buffers' release) waits for both streams
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], q[0]);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], q[1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[1], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[2], 0);
    }
    if (e == cudaSuccess && !out_dev) e = cudaStreamSynchronize(st);
    destroy();
    if (e != cudaSuccess) return fail(VF_ECUDA, std::string("vf_query (pipelined): ") + cudaGetErrorString(e));
    return VF_OK;
}

vf_status vf_query(const vf_struct* s, const void* keys, const uint64_t* offsets, uint64_t m, void* out,
                   void* stream) {
    if (!s) return fail(VF_EINVAL, "vf_query: NULL structure");
    if (m == 0) return VF_OK;
    if (!keys || !out) return fail(VF_EINVAL, "vf_query: NULL keys or out");
    const int key_kind = offsets ? VF_KEYS_BYTES : VF_KEYS_U64;
    for (const auto& pw : {std::make_pair(keys, "keys"), std::make_pair(static_cast<const void*>(offsets), "offsets"),
                           std::make_pair(static_cast<const void*>(out), "out")}) {
        const vf_status cs = vf::check_here(pw.first, pw.second);
        if (cs != VF_OK) return cs;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t ob = s->info.kind == VF_FILTER ? 1 : value_bytes(s->info.b);
    const bool out_dev = on_device(out);
    if (key_kind == VF_KEYS_U64) {
        const bool keys_dev = on_device(keys);
        if (!keys_dev || !out_dev)
            return query_pipelined(s, static_cast<const uint64_t*>(keys), keys_dev, m, out, out_dev, ob, st);
    }
    Staged in_keys;
    vf_status rs = stage_keys(key_kind, keys, offsets, m, st, in_keys);
    if (rs != VF_OK) return rs;
    DevBuf obuf;
    void* dout = out;
    if (!out_dev) {
        VF_CK(obuf.alloc(m * ob, st));
        dout = obuf.p;
    }
    {
        PhaseTimer t(kPhQuery, st);
        VF_CK(vf::launch_query(key_kind, in_keys.keys, in_keys.offs, m, s->geom, s->data, dout, st));
    }
    if (!out_dev) {
        VF_CK(cudaMemcpyAsync(out, dout, m * ob, cudaMemcpyDeviceToHost, st));
        VF_CK(cudaStreamSynchronize(st));
    }
    return VF_OK;
}

vf_status vf_query_batch(const vf_query_req* reqs, uint32_t count, void* stream) {
    if (count > 0 && !reqs) return fail(VF_EINVAL, "vf_query_batch: NULL requests");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<vf::QueryReq> d;
    d.reserve(count);
    uint64_t total = 0;
    for (uint32_t i = 0; i < count; i++) {
        const vf_query_req& r = reqs[i];
        if (!r.s) return fail(VF_EINVAL, "vf_query_batch: NULL structure");
        if (r.m == 0) continue;
        if (!on_device(r.keys) || !on_device(r.out))
            return fail(VF_EINVAL, "vf_query_batch: keys and outputs must be device memory of the current device");
        vf::QueryReq q;
        std::memset(&q, 0, sizeof q);
        q.g = r.s->geom;
        q.data = r.s->data;
        q.keys = r.keys;
        q.out = r.out;
        q.key_off = total;
        q.m = r.m;
        total += r.m;
        d.push_back(q);
    }
    if (d.empty()) return VF_OK;
    DevBuf db;
    vf_status rs = h2d(db, d, st);
    if (rs != VF_OK) return rs;
    {
        PhaseTimer t(kPhQuery, st);
        VF_CK(vf::launch_query_batch(db.as<vf::QueryReq>(), uint32_t(d.size()), total, st));
    }
    return VF_OK;
}

vf_status vf_get_info(const vf_struct* s, vf_info* info) {
    if (!s || !info) return fail(VF_EINVAL, "vf_get_info: NULL argument");
    *info = s->info;
    return VF_OK;
}

vf_status vf_data(const vf_struct* s, const void** dev_ptr, uint64_t* bytes) {
    if (!s || !dev_ptr || !bytes) return fail(VF_EINVAL, "vf_data: NULL argument");
    *dev_ptr = s->data;
    *bytes = s->info.data_bytes;
    return VF_OK;
}

vf_status vf_export(const vf_struct* s, void* host_dst) {
    if (!s || !host_dst) return fail(VF_EINVAL, "vf_export: NULL argument");
    VF_CK(cudaMemcpy(host_dst, s->data, s->info.data_bytes, cudaMemcpyDeviceToHost));
    return VF_OK;
}

vf_status vf_signatures(int key_kind, const void* keys, const uint64_t* offsets, uint64_t n, uint64_t seed,
                        uint64_t* out, void* stream) {
    if (n == 0) return VF_OK;
    if (!keys || !out || (key_kind == VF_KEYS_BYTES && !offsets)) return fail(VF_EINVAL, "vf_signatures: NULL");
    if (key_kind != VF_KEYS_U64 && key_kind != VF_KEYS_BYTES) return fail(VF_EINVAL, "bad key_kind");
    for (const auto& pw : {std::make_pair(keys, "keys"), std::make_pair(static_cast<const void*>(offsets), "offsets"),
                           std::make_pair(static_cast<const void*>(out), "out")}) {
        const vf_status cs = vf::check_here(pw.first, pw.second);
        if (cs != VF_OK) return cs;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Staged in_keys;
    vf_status rs = stage_keys(key_kind, keys, offsets, n, st, in_keys);
    if (rs != VF_OK) return rs;
    const bool out_dev = on_device(out);
    DevBuf obuf;
    void* dout = out;
    if (!out_dev) {
        VF_CK(obuf.alloc(n * 16, st));
        dout = obuf.p;
    }
    VF_CK(vf::launch_sigs(key_kind, in_keys.keys, in_keys.offs, n, vf::mix64(seed ^ vf::kLaneHi),
                          vf::mix64(seed ^ vf::kLaneLo), static_cast<vf::Sig*>(dout), st));
    if (!out_dev) {
        VF_CK(cudaMemcpyAsync(out, dout, n * 16, cudaMemcpyDeviceToHost, st));
        VF_CK(cudaStreamSynchronize(st));
    }
    return VF_OK;
}

vf_status vf_timing_enable(int on) {
    g_timing = on != 0;
    return VF_OK;
}

vf_status vf_debug_faults(int fail_attempts, uint32_t assign_poll_limit, int stall_assign) {
    if (fail_attempts < 0) return fail(VF_EINVAL, "vf_debug_faults: fail_attempts < 0");
    g_debug_fail_attempts = fail_attempts;
    g_debug_assign_limit = assign_poll_limit;
    g_debug_stall_assign = stall_assign != 0;
    return VF_OK;
}

vf_status vf_timing_read(double* ms, uint64_t* launches) {
    if (!ms || !launches) return fail(VF_EINVAL, "vf_timing_read: NULL argument");
    vf_status rs = VF_OK;
    for (auto& t : g_timed) {
        float x = 0.f;
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, t.a, t.b);
        if (e != cudaSuccess) rs = fail(VF_ECUDA, std::string("timing: ") + cudaGetErrorString(e));
        ms[t.phase] += x;
        launches[t.phase] += uint64_t(t.kernels);
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    g_timed.clear();
    return rs;
}

vf_status vf_batch_opts_default(vf_batch_opts* o) {
    if (!o) return fail(VF_EINVAL, "vf_batch_opts_default: NULL");
    std::memset(o, 0, sizeof *o);
    o->lge_threshold = 800000;
    o->lge_target = 16384;
    o->lpt = 1;
    o->use_graph = 1;
    o->small_cta_keys = vf::kLgeSmallTaskKeys;
    return VF_OK;
}

vf_status vf_build_batch(const vf_batch_item* items, uint32_t count, const vf_params* common,
                         const vf_batch_opts* opts, void* stream, vf_struct** out) {
    g_last_error.clear();
    if (!common || !out || (count > 0 && !items)) return fail(VF_EINVAL, "vf_build_batch: NULL argument");
    if (common->mode < VF_MODE_AUTO || common->mode > VF_MODE_MWHC || common->fuse_solver < VF_SOLVER_FLOW ||
        common->fuse_solver > VF_SOLVER_WAVE || (common->arity != 3 && common->arity != 4))
        return fail(VF_EINVAL, "vf_build_batch: bad mode, fuse solver or arity");
    vf_batch_opts o;
    if (opts) o = *opts; else vf_batch_opts_default(&o);
    if (o.lge_target == 0) return fail(VF_EINVAL, "vf_build_batch: lge_target must be positive");
    for (uint32_t i = 0; i < count; i++) {
        out[i] = nullptr;
        const vf_batch_item& it = items[i];
        if (it.b < 1 || it.b > 32 || (it.kind != VF_FUNC && it.kind != VF_FILTER))
            return fail(VF_EINVAL, "vf_build_batch: bad b or kind");
        if (it.n > 0 && !it.keys) return fail(VF_EINVAL, "vf_build_batch: keys is NULL");
        if (it.kind == VF_FUNC && it.n > 0 && !it.values) return fail(VF_EINVAL, "vf_build_batch: a function needs values");
        if (it.n >= (uint64_t(1) << 32)) return fail(VF_ECAPACITY, "vf_build_batch: at most 2^32-1 keys per structure");
        vf_status cs = vf::check_here(it.keys, "vf_build_batch: keys");
        if (cs == VF_OK) cs = vf::check_here(it.values, "vf_build_batch: values");
        if (cs != VF_OK) return cs;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    VF_CK(cudaGetDevice(&dev));
    keep_pool_warm(dev);
    std::vector<Staged> staged(count);
    std::vector<const uint64_t*> kdev(count);
    std::vector<const void*> vdev(count, nullptr);
    for (uint32_t i = 0; i < count; i++) {
        vf_status rs = stage_keys(VF_KEYS_U64, items[i].keys, nullptr, items[i].n, st, staged[i]);
        if (rs != VF_OK) return rs;
        kdev[i] = static_cast<const uint64_t*>(staged[i].keys);
        if (items[i].kind == VF_FUNC && items[i].n > 0) {
            if (on_device(items[i].values)) {
                vdev[i] = items[i].values;
            } else {
                const size_t vb = items[i].n * value_bytes(items[i].b);
                VF_CK(staged[i].vbuf.alloc(vb, st));
                VF_CK(cudaMemcpyAsync(staged[i].vbuf.p, items[i].values, vb, cudaMemcpyHostToDevice, st));
                vdev[i] = staged[i].vbuf.p;
            }
        }
    }
    std::vector<uint32_t> pending(count), attempt(count, 0);
    for (uint32_t i = 0; i < count; i++) pending[i] = i;
    for (int round = 0; round <= common->max_retries && !pending.empty(); round++) {
        std::vector<uint32_t> failed;
        vf_status rs = build_batch_once(items, pending, attempt, *common, o, kdev, vdev, st, dev, out, failed);
        if (rs != VF_OK) {
            for (uint32_t i = 0; i < count; i++) {
                vf_free(out[i]);
                out[i] = nullptr;
            }
            return rs;
        }
        for (uint32_t i : failed) attempt[i]++;
        pending.swap(failed);
    }
    if (!pending.empty()) {
        for (uint32_t i = 0; i < count; i++) {
            vf_free(out[i]);
            out[i] = nullptr;
        }
        return fail(VF_EBUILD, "vf_build_batch: a structure failed every attempt");
    }
    return VF_OK;
}

vf_status vf_tune_batch(const vf_batch_item* items, uint32_t count, const vf_params* common, void* stream,
                        vf_batch_opts* best, double* best_ms) {
    if (!common || !best || (count > 0 && !items)) return fail(VF_EINVAL, "vf_tune_batch: NULL argument");
    uint64_t total = 0, nmax = 0;
    for (uint32_t i = 0; i < count; i++) {
        total += items[i].n;
        nmax = std::max<uint64_t>(nmax, items[i].n);
    }
    const TuneKey key{count, total, nmax};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second;
            if (best_ms) *best_ms = -1.0;
            return VF_OK;
        }
    }
    // sample: every k-th structure, about 5% of the keys and at least 16 structures
    std::vector<vf_batch_item> sample;
    const uint64_t want = std::max<uint64_t>(total / 20, 1);
    const uint32_t stride = uint32_t(std::max<uint64_t>(1, std::min<uint64_t>(count / 16 + 1, total / want)));
    for (uint32_t i = 0; i < count; i += stride) sample.push_back(items[i]);
    std::vector<vf_batch_opts> cands;
    for (uint64_t thr : {common->lge_threshold, ~uint64_t(0)})
        for (uint64_t tgt : {uint64_t(8192), uint64_t(16384)})
            for (int lpt : {1, 0})
                for (uint64_t small : {uint64_t(vf::kLgeSmallTaskKeys), uint64_t(0)}) {
                    vf_batch_opts o;
                    vf_batch_opts_default(&o);
                    o.lge_threshold = thr;
                    o.lge_target = tgt;
                    o.lpt = lpt;
                    o.small_cta_keys = small;
                    cands.push_back(o);
                }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    VF_CK(cudaEventCreate(&e0));
    VF_CK(cudaEventCreate(&e1));
    std::vector<vf_struct*> outs(sample.size(), nullptr);
    double bms = 1e300;
    vf_batch_opts bo = cands[0];
    for (size_t c = 0; c <= cands.size(); c++) {
        const vf_batch_opts& o = cands[c == 0 ? 0 : c - 1];  // the first candidate runs twice (warm-up)
        VF_CK(cudaEventRecord(e0, st));
        vf_status rs = vf_build_batch(sample.data(), uint32_t(sample.size()), common, &o, stream, outs.data());
        VF_CK(cudaEventRecord(e1, st));
        VF_CK(cudaEventSynchronize(e1));
        for (auto*& p : outs) {
            vf_free(p);
            p = nullptr;
        }
        if (rs != VF_OK) continue;
        float ms = 0.f;
        VF_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (c > 0 && ms < bms) {
            bms = ms;
            bo = o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bms >= 1e300) return fail(VF_EBUILD, "vf_tune_batch: no candidate built the sample");
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = bo;
    }
    *best = bo;
    if (best_ms) *best_ms = bms;
    return VF_OK;
}

// ------------------------------------------------------------ serialized form

static vf_status new_struct_from(const vf::StoreHeader& h, const uint8_t* host_or_dev_data, std::FILE* f,
                                 vf_struct** out) {
    int dev = 0;
    VF_CK(cudaGetDevice(&dev));
    uint8_t* d = nullptr;
    VF_CK(cudaMalloc(&d, h.info.data_bytes + 16));
    cudaError_t e = cudaMemset(d, 0, h.info.data_bytes + 16);
    bool io = true;
    if (e == cudaSuccess) {
        if (f) e = vf::file_to_device(f, vf::kStoreHeaderBytes, d, h.info.data_bytes, &io);
        else e = cudaMemcpy(d, host_or_dev_data, h.info.data_bytes, cudaMemcpyDefault);
    }
    if (e != cudaSuccess || !io) {
        cudaFree(d);
        if (!io) return fail(VF_EIO, "reading the data array failed");
        return fail(VF_ECUDA, std::string("loading the data array: ") + cudaGetErrorString(e));
    }
    vf_struct* s = new vf_struct;
    s->info = h.info;
    s->geom = vf::geom_of(h.info);
    s->data = d;
    s->device = dev;
    *out = s;
    return VF_OK;
}

static vf::StoreHeader header_of(const vf_struct* s) {
    vf::StoreHeader h;
    std::memset(&h, 0, sizeof h);
    h.info = s->info;
    h.groups_total = h.groups_done = 1;
    h.dropped = s->info.n - s->info.n_eff;
    h.key_kind = -1;  // queries say which key kind they pass
    return h;
}

vf_status vf_serialize(const vf_struct* s, void* buf, uint64_t capacity, uint64_t* size) {
    if (!s || !size) return fail(VF_EINVAL, "vf_serialize: NULL argument");
    *size = vf::kStoreHeaderBytes + s->info.data_bytes;
    if (!buf) return VF_OK;
    if (capacity < *size) return fail(VF_EINVAL, "vf_serialize: buffer too small");
    vf::store_encode(header_of(s), static_cast<uint8_t*>(buf));
    VF_CK(cudaMemcpy(static_cast<uint8_t*>(buf) + vf::kStoreHeaderBytes, s->data, s->info.data_bytes,
                     cudaMemcpyDeviceToHost));
    return VF_OK;
}

vf_status vf_deserialize(const void* buf, uint64_t size, void* stream, vf_struct** out) {
    (void)stream;
    if (!buf || !out) return fail(VF_EINVAL, "vf_deserialize: NULL argument");
    *out = nullptr;
    vf::StoreHeader h;
    if (!vf::store_decode(static_cast<const uint8_t*>(buf), size, h) || h.groups_done != h.groups_total ||
        size < vf::kStoreHeaderBytes + h.info.data_bytes)
        return fail(VF_EIO, "vf_deserialize: not a complete serialized structure");
    return new_struct_from(h, static_cast<const uint8_t*>(buf) + vf::kStoreHeaderBytes, nullptr, out);
}

vf_status vf_save(const vf_struct* s, const char* path) {
    if (!s || !path) return fail(VF_EINVAL, "vf_save: NULL argument");
    std::FILE* f = std::fopen(path, "wb");
    if (!f) return fail(VF_EIO, std::string("vf_save: cannot create ") + path);
    std::vector<uint8_t> hb(vf::kStoreHeaderBytes);
    vf::store_encode(header_of(s), hb.data());
    bool io = vf::file_write_at(f, 0, hb.data(), hb.size());
    cudaError_t e = cudaSuccess;
    if (io) e = vf::device_to_file(f, vf::kStoreHeaderBytes, s->data, s->info.data_bytes, &io);
    if (std::fclose(f) != 0) io = false;
    if (e != cudaSuccess) return fail(VF_ECUDA, std::string("vf_save: ") + cudaGetErrorString(e));
    if (!io) return fail(VF_EIO, "vf_save: writing failed");
    return VF_OK;
}

vf_status vf_load(const char* path, void* stream, vf_struct** out) {
    (void)stream;
    if (!path || !out) return fail(VF_EINVAL, "vf_load: NULL argument");
    *out = nullptr;
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return fail(VF_EIO, std::string("vf_load: cannot open ") + path);
    std::vector<uint8_t> hb(vf::kStoreHeaderBytes);
    vf::StoreHeader h;
    vf_status rs;
    if (!vf::file_read_at(f, 0, hb.data(), hb.size()) || !vf::store_decode(hb.data(), hb.size(), h) ||
        h.groups_done != h.groups_total)
        rs = fail(VF_EIO, "vf_load: not a complete serialized structure");
    else
        rs = new_struct_from(h, nullptr, f, out);
    std::fclose(f);
    return rs;
}

vf_status vf_free(vf_struct* s) {
    if (!s) return VF_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    cudaError_t e = cudaFree(s->data);
    if (cur != s->device) cudaSetDevice(cur);
    delete s;
    if (e != cudaSuccess) return fail(VF_ECUDA, std::string("cudaFree: ") + cudaGetErrorString(e));
    return VF_OK;
}

}  // extern "C"
