// Random-sector read rate of the device (vf_sector_rate in include/vfunc.h):
// the denominator of the query's roofline. A query reads three cells at
// random positions of its structure's data array, each one 32-byte sector;
// how many such sectors the GPU delivers per second depends on whether the
// array fits in L2 and on how DRAM serves scattered sectors, which a copy
// bandwidth does not capture.
#include <algorithm>
#include <string>

#include "vf_internal.h"

namespace vf {
namespace {

constexpr int kPK = 12;  // independent loads per thread per iteration
constexpr int kPThreads = 256;

// Each thread issues kPK loads at positions mulhi(hash, n) < n, n the table's
// words, then folds them into one word so no load is dead.
__global__ void __launch_bounds__(kPThreads) k_sector_probe(const uint32_t* __restrict__ t, uint64_t n, uint32_t iters,
                                                            uint64_t salt, uint32_t* __restrict__ out) {
    const uint64_t tid = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; it++) {
        uint32_t v[kPK];
#pragma unroll
        for (int k = 0; k < kPK; k++) v[k] = __ldg(t + mulhi(mix64(salt ^ (tid * kGolden + uint64_t(it) * kPK + k)), n));
#pragma unroll
        for (int k = 0; k < kPK; k++) acc ^= v[k];
    }
    out[tid] = acc;
}

}  // namespace
}  // namespace vf

extern "C" vf_status vf_sector_rate(uint64_t table_bytes, void* stream, double* sectors_per_s) {
    using namespace vf;
    if (!sectors_per_s || table_bytes < 4096) {
        set_last_error("vf_sector_rate: NULL result or a table below 4096 bytes");
        return VF_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned blocks = unsigned(num_sms()) * 8;
    const uint64_t threads = uint64_t(blocks) * kPThreads;
    uint32_t* t = nullptr;
    uint32_t* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto done = [&](vf_status s, const char* what, cudaError_t e) {
        if (t) cudaFree(t);
        if (out) cudaFree(out);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s != VF_OK) set_last_error((std::string("vf_sector_rate: ") + what + ": " + cudaGetErrorString(e)).c_str());
        return s;
    };
    cudaError_t e = cudaMalloc(&t, table_bytes);
    if (e != cudaSuccess) return done(VF_ENOMEM, "table allocation", e);
    if ((e = cudaMalloc(&out, threads * 4)) != cudaSuccess) return done(VF_ENOMEM, "output allocation", e);
    if ((e = cudaMemsetAsync(t, 1, table_bytes, st)) != cudaSuccess) return done(VF_ECUDA, "memset", e);
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return done(VF_ECUDA, "events", e);
    const uint64_t n = table_bytes / 4;
    double best = 0.0;
    uint32_t iters = 8;
    for (int rep = 0; rep < 8; rep++) {
        cudaEventRecord(e0, st);
        k_sector_probe<<<blocks, kPThreads, 0, st>>>(t, n, iters, 0x5EC7 + uint64_t(rep), out);
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return done(VF_ECUDA, "probe", e);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep >= 2) best = std::max(best, double(threads) * iters * kPK / (double(ms) * 1e-3));
        if (ms < 2.0f && iters < (1u << 16)) iters *= 2;  // grow to a few milliseconds per launch
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return done(VF_ECUDA, "probe launch", e);
    *sectors_per_s = best;
    return done(VF_OK, "", cudaSuccess);
}
