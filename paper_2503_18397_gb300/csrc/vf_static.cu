// Allocation-free build of a small single-shard structure (vf_build_static in
// include/vfunc.h). Every byte of scratch the build needs lives in one
// file-scope device array; the caller provides keys, values and the output
// data array, and nothing here calls cudaMalloc, cudaFree or any other
// allocating routine.
#include <cstring>
#include <mutex>

#include "vf_internal.h"
#include "vfunc.h"

namespace vf {
namespace {

constexpr uint32_t kStaticMaxKeys = 16384;
// cells of a single LGE shard of kStaticMaxKeys keys: ceil(1.12 * M)
constexpr uint32_t kStaticMaxCells = (kStaticMaxKeys * 112u + 99u) / 100u;
constexpr uint64_t kMiscWords = 64;   // [0] error word, [4..] solver statistics
constexpr uint64_t kStartWords = 4;   // shard starts {0, n} as two 64-bit words
constexpr uint64_t kTaskWords = (sizeof(LgeTask) + 15) / 16 * 4;  // the solver's one task
constexpr uint64_t kLocWords = 2ull * kStaticMaxKeys;
constexpr uint64_t kValWords = kStaticMaxKeys;
constexpr uint64_t kSlabWords = lge_offsets(kStaticMaxKeys, kStaticMaxCells).total;
constexpr uint64_t kStaticWords = kMiscWords + kStartWords + kTaskWords + kLocWords + kValWords + kSlabWords;

// The scratch itself: about 4.6 MB, resident on every GPU that loads the
// library for the life of the process. Shared by every call.
static __device__ __align__(256) uint32_t g_static_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
uint32_t* g_static_dev[kMaxDevices] = {};

vf_status fail_static(vf_status st, const char* msg) {
    set_last_error(msg);
    return st;
}

// Device (or managed) memory the current device can use.
bool is_device_pointer(const void* p) { return mem_where(p) == MemWhere::kHere; }

// Device address of g_static_scratch on the current device. In host code the
// array's name is only a stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
vf_status static_scratch(uint32_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail_static(VF_ECUDA, "vf_build_static: no usable current device");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_static_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return fail_static(VF_ECUDA, "vf_build_static: cudaGetSymbolAddress failed");
        g_static_dev[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_static_dev[dev];
    return VF_OK;
}

// Single shard (h = 0): the local signature is the signature's high word.
__global__ void k_static_prep(const uint64_t* __restrict__ keys, const void* __restrict__ values, uint32_t n, int b,
                              uint64_t kh, uint64_t kl, uint64_t* __restrict__ loc, uint32_t* __restrict__ val,
                              unsigned long long* __restrict__ start) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        loc[i] = local_of(sig_u64(__ldg(keys + i), kh, kl), 0);
        if (values) {
            uint32_t v;
            if (b <= 8) v = __ldg(static_cast<const uint8_t*>(values) + i);
            else if (b <= 16) v = __ldg(static_cast<const uint16_t*>(values) + i);
            else v = __ldg(static_cast<const uint32_t*>(values) + i);
            val[i] = b == 32 ? v : (v & ((1u << b) - 1u));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        start[0] = 0;
        start[1] = n;
    }
}

}  // namespace
}  // namespace vf

extern "C" vf_status vf_build_static(const uint64_t* keys, const void* values, uint64_t n, const vf_params* params,
                                     void* data, uint64_t data_capacity, vf_info* info, void* stream) {
    using namespace vf;
    if (!params || !info || !data) return fail_static(VF_EINVAL, "vf_build_static: NULL params, info or data");
    if (n > kStaticMaxKeys) return fail_static(VF_ECAPACITY, "vf_build_static: at most 16384 keys");
    vf_params p = *params;
    if (p.key_kind != VF_KEYS_U64) return fail_static(VF_EINVAL, "vf_build_static: 64-bit integer keys only");
    if (p.b < 1 || p.b > 32 || (p.kind != VF_FUNC && p.kind != VF_FILTER) || p.max_retries < 0)
        return fail_static(VF_EINVAL, "vf_build_static: bad b, kind or max_retries");
    if (n > 0 && !is_device_pointer(keys))
        return fail_static(VF_EINVAL, "vf_build_static: keys must be device memory of the current device");
    if (p.kind == VF_FUNC && n > 0 && !is_device_pointer(values))
        return fail_static(VF_EINVAL, "vf_build_static: values must be device memory of the current device");
    if (!is_device_pointer(data))
        return fail_static(VF_EINVAL, "vf_build_static: data must be device memory of the current device");
    // one shard in the LGE regime
    p.mode = VF_MODE_LGE;
    p.lge_target = kStaticMaxKeys;
    p.lge_max_shard = kStaticMaxKeys;
    vf_info in;
    vf_status rs = vf_plan(&p, n, n, &in);
    if (rs != VF_OK) return rs;
    if (in.h != 0 || in.cells > kStaticMaxCells) return fail_static(VF_ECAPACITY, "vf_build_static: shape out of range");
    if (data_capacity < in.data_bytes) return fail_static(VF_EINVAL, "vf_build_static: data buffer too small");

    uint32_t* base = nullptr;
    rs = static_scratch(&base);
    if (rs != VF_OK) return rs;
    // A launch error left over from the caller's own work would otherwise be
    // reported as this call's failure: drop it before the first launch.
    (void)cudaGetLastError();
    uint32_t* misc = base;
    unsigned long long* start = reinterpret_cast<unsigned long long*>(base + kMiscWords);
    LgeTask* tasks_dev = reinterpret_cast<LgeTask*>(base + kMiscWords + kStartWords);
    uint64_t* loc = reinterpret_cast<uint64_t*>(base + kMiscWords + kStartWords + kTaskWords);
    uint32_t* val = base + kMiscWords + kStartWords + kTaskWords + kLocWords;
    uint32_t* slab = val + kValWords;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    for (int attempt = 0; attempt <= p.max_retries; attempt++) {
        in.seed = p.seed + uint64_t(attempt);
        in.retries = attempt;
        Geom g;
        std::memset(&g, 0, sizeof g);
        g.kh = mix64(in.seed ^ kLaneHi);
        g.kl = mix64(in.seed ^ kLaneLo);
        g.cells = in.cells;
        g.h = 0;
        g.regime = kRegimeLge;
        g.b = in.b;
        g.kind = in.kind;
        // the array keeps the previous call's contents: clear what must start at zero
        if (cudaMemsetAsync(misc, 0, kMiscWords * 4, st) != cudaSuccess ||
            cudaMemsetAsync(data, 0, in.data_bytes, st) != cudaSuccess)
            return fail_static(VF_ECUDA, "vf_build_static: clearing scratch failed");
        k_static_prep<<<32, 256, 0, st>>>(keys, p.kind == VF_FUNC ? values : nullptr, uint32_t(n), in.b, g.kh, g.kl,
                                          loc, val, start);
        LgeTask task;
        std::memset(&task, 0, sizeof task);
        task.loc_off = 0;
        task.cell_base = 0;
        task.data = static_cast<uint8_t*>(data);
        task.m = uint32_t(n);
        task.cells = uint32_t(in.cells);
        task.b = in.b;
        task.kind = in.kind;
        task.item = 0;
        if (cudaMemcpyAsync(tasks_dev, &task, sizeof task, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail_static(VF_ECUDA, "vf_build_static: task upload failed");
        LgeArgs a;
        std::memset(&a, 0, sizeof a);
        a.tasks = tasks_dev;
        a.ntasks = n > 0 ? 1u : 0u;
        a.loc = loc;
        a.val = val;
        a.item_fail = misc;
        a.scratch = slab;
        a.scratch_words_per_cta = kSlabWords;
        a.m_cap = kStaticMaxKeys;
        a.v_cap = kStaticMaxCells;
        a.err = misc;
        a.stats = misc + 4;
        if (cudaGetLastError() != cudaSuccess || launch_lge(a, 1, st) != cudaSuccess)
            return fail_static(VF_ECUDA, "vf_build_static: kernel launch failed");
        uint32_t h[8];
        if (cudaMemcpyAsync(h, misc, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail_static(VF_ECUDA, "vf_build_static: reading the outcome failed");
        if (h[0] & kErrDupKey) return fail_static(VF_EDUP, "vf_build_static: a key was given twice with different values");
        if (h[0] & (kErrCapacity | kErrLgeSize)) return fail_static(VF_ECAPACITY, "vf_build_static: shard exceeds the solver");
        if (h[0] & (kErrUnsolvable | kErrDegOverflow)) continue;
        if (attempt < debug_fail_attempts()) continue;  // test hook of vf_debug_faults, as in vf_build
        in.peeled = h[4];
        in.core = h[5];
        in.rounds = 0;
        in.n_eff = n - h[7];  // a filter drops duplicate local signatures
        *info = in;
        return VF_OK;
    }
    return fail_static(VF_EBUILD, "vf_build_static: all attempts failed (seed .. seed+max_retries)");
}
