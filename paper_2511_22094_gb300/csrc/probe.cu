// Issue-rate probe of the SM's arithmetic pipes: results per clock per SM of
// the operations the sampler's roofline counts -- FP32 fma (single and
// paired), the special-function unit's ex2, sin, lg2, rsqrt, rcp and sqrt,
// FP64 fma, and the 32-bit high multiply-add and three-input logic of Philox.
// Not part of the method: the roofline's denominators, measured on the device
// instead of taken from a data sheet.
//
// Every thread runs kChains independent dependency chains of one operation,
// so that latency is hidden and only the pipe's issue rate remains.  Each
// block reads the SM's cycle counter around its loop; an SM's rate is its
// blocks' results over the span from the first start to the last end on that
// SM.  The reported rate is the median over SMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "gac.h"
#include "gac_internal.h"

namespace gac {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kChains = 8;
constexpr int kBlocksPerSm = 4;
constexpr int kIters = 4096;

// One operation: the state type, its start value, one dependent step, and
// how many results one step yields per thread.
template <int OP>
struct Op;

template <>
struct Op<GAC_PIPE_FFMA> {
    using T = float;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0.5f + 0.01f * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(x), "f"(0.9999f), "f"(1e-4f));
        return r;
    }
    __device__ static float fold(T x) { return x; }
};
template <>
struct Op<GAC_PIPE_FFMA2> {
    using T = float2;
    static constexpr int kResults = 2;
    __device__ static T init(int j) { return make_float2(0.5f + 0.01f * j, 0.25f + 0.01f * j); }
    __device__ static T step(T x) { return __ffma2_rn(x, make_float2(0.9999f, 0.9999f), make_float2(1e-4f, 1e-4f)); }
    __device__ static float fold(T x) { return x.x + x.y; }
};
// ex2 of -x keeps the chain in (0, 1]
template <>
struct Op<GAC_PIPE_EX2> {
    using T = float;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0.5f + 0.01f * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x));
        return r;
    }
    __device__ static float fold(T x) { return x; }
};
template <>
struct Op<GAC_PIPE_SIN> {
    using T = float;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0.5f + 0.01f * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    __device__ static float fold(T x) { return x; }
};
// lg2(x) + 1.5 keeps the chain in [2, 3]
template <>
struct Op<GAC_PIPE_LG2> {
    using T = float;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 2.0f + 0.01f * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r + 1.5f;
    }
    __device__ static float fold(T x) { return x; }
};
template <>
struct Op<GAC_PIPE_RSQRT> {
    using T = float;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0.75f + 0.01f * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    __device__ static float fold(T x) { return x; }
};
// 1/x + 0.25 (1/(1/x) alone would let the compiler cancel the pair)
template <>
struct Op<GAC_PIPE_RCP> {
    using T = float;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0.75f + 0.01f * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r + 0.25f;
    }
    __device__ static float fold(T x) { return x; }
};
template <>
struct Op<GAC_PIPE_SQRT> {
    using T = float;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0.75f + 0.01f * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    __device__ static float fold(T x) { return x; }
};
template <>
struct Op<GAC_PIPE_DFMA> {
    using T = double;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0.5 + 0.01 * j; }
    __device__ static T step(T x) {
        T r;
        asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(x), "d"(0.9999), "d"(1e-4));
        return r;
    }
    __device__ static float fold(T x) { return static_cast<float>(x); }
};
template <>
struct Op<GAC_PIPE_IMAD_HI> {
    using T = unsigned;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0x9E3779B9u * (j + 1); }
    __device__ static T step(T x) {
        T r;
        asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(0xD2511F53u), "r"(0x1234567u));
        return r;
    }
    __device__ static float fold(T x) { return static_cast<float>(x); }
};
template <>
struct Op<GAC_PIPE_LOP3> {
    using T = unsigned;
    static constexpr int kResults = 1;
    __device__ static T init(int j) { return 0x9E3779B9u * (j + 1); }
    __device__ static T step(T x) {
        T r;
        asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(x), "r"(0xBB67AE85u), "r"(0x3C6EF372u));
        return r;
    }
    __device__ static float fold(T x) { return static_cast<float>(x); }
};

template <int OP>
__global__ void __launch_bounds__(kProbeBlock) pipe_probe_kernel(long long *t0, long long *t1, int *smid, float *sink) {
    using O = Op<OP>;
    typename O::T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = O::init(j + (threadIdx.x & 7));
    __syncthreads();
    const long long c0 = clock64();
#pragma unroll 16
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = O::step(a[j]);
    }
    __syncthreads();
    const long long c1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += O::fold(a[j]);
    if (s == 1234.5f) sink[0] = s;  // keeps the chains live
    if (threadIdx.x == 0) {
        unsigned id;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
        t0[blockIdx.x] = c0;
        t1[blockIdx.x] = c1;
        smid[blockIdx.x] = static_cast<int>(id);
    }
}

template <int OP>
const void *probe_ptr() {
    return reinterpret_cast<const void *>(&pipe_probe_kernel<OP>);
}

const void *probe_kernel(int op) {
    switch (op) {
    case GAC_PIPE_FFMA: return probe_ptr<GAC_PIPE_FFMA>();
    case GAC_PIPE_FFMA2: return probe_ptr<GAC_PIPE_FFMA2>();
    case GAC_PIPE_EX2: return probe_ptr<GAC_PIPE_EX2>();
    case GAC_PIPE_SIN: return probe_ptr<GAC_PIPE_SIN>();
    case GAC_PIPE_LG2: return probe_ptr<GAC_PIPE_LG2>();
    case GAC_PIPE_RSQRT: return probe_ptr<GAC_PIPE_RSQRT>();
    case GAC_PIPE_RCP: return probe_ptr<GAC_PIPE_RCP>();
    case GAC_PIPE_SQRT: return probe_ptr<GAC_PIPE_SQRT>();
    case GAC_PIPE_DFMA: return probe_ptr<GAC_PIPE_DFMA>();
    case GAC_PIPE_IMAD_HI: return probe_ptr<GAC_PIPE_IMAD_HI>();
    case GAC_PIPE_LOP3: return probe_ptr<GAC_PIPE_LOP3>();
    default: return nullptr;
    }
}

int results_per_step(int op) { return op == GAC_PIPE_FFMA2 ? 2 : 1; }

}  // namespace
}  // namespace gac

using namespace gac;

extern "C" gac_status gac_pipe_rate(int op, double *per_clk_sm, void *stream) {
    clear_error();
    const void *fn = probe_kernel(op);
    if (!fn) return fail(GAC_ERR_INVALID_ARG, "unknown pipe probe %d", op);
    if (!per_clk_sm) return fail(GAC_ERR_INVALID_ARG, "per_clk_sm must not be NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device");
    const int grid = sms * kBlocksPerSm;
    void *buf = nullptr;
    const size_t bytes = static_cast<size_t>(grid) * (2 * sizeof(long long) + sizeof(int)) + 16;
    if ((e = cudaMallocAsync(&buf, bytes, s)) != cudaSuccess) return cuda_fail(e, "probe buffer");
    auto *t0 = static_cast<long long *>(buf);
    long long *t1 = t0 + grid;
    int *smid = reinterpret_cast<int *>(t1 + grid);
    float *sink = reinterpret_cast<float *>(smid + grid);
    void *args[] = {&t0, &t1, &smid, &sink};
    // a warm-up launch, then the measured one
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)
        e = cudaLaunchKernel(fn, dim3(grid), dim3(kProbeBlock), args, 0, s);
    std::vector<long long> h0(grid), h1(grid);
    std::vector<int> hs(grid);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h0.data(), t0, grid * sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h1.data(), t1, grid * sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), smid, grid * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(buf, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "pipe probe");
    // per SM: results of its blocks over [first start, last end]
    std::map<int, std::pair<long long, long long>> span;
    std::map<int, int> blocks;
    for (int b = 0; b < grid; ++b) {
        auto it = span.find(hs[b]);
        if (it == span.end()) span[hs[b]] = {h0[b], h1[b]};
        else it->second = {std::min(it->second.first, h0[b]), std::max(it->second.second, h1[b])};
        ++blocks[hs[b]];
    }
    const double per_block =
        static_cast<double>(kProbeBlock) * kChains * kIters * results_per_step(op);
    std::vector<double> rate;
    for (const auto &kv : span) {
        const long long cyc = kv.second.second - kv.second.first;
        if (cyc > 0) rate.push_back(blocks[kv.first] * per_block / static_cast<double>(cyc));
    }
    if (rate.empty()) return fail(GAC_ERR_CUDA, "pipe probe recorded no cycles");
    std::sort(rate.begin(), rate.end());
    *per_clk_sm = rate[rate.size() / 2];
    return GAC_OK;
}
