// gac_mcmc_run_noalloc: the sampler for callers that must not allocate
// device memory (see include/gac.h).  It runs the sliced tile routine that
// the server uses, one launch per slice of iterations, with the chains'
// state between slices in one fixed file-scope device array instead of
// memory allocated per call.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
#include <cuda_runtime.h>

#include <cmath>

#include <algorithm>
#include <cstring>

#include "gac.h"
#include "gac_internal.h"
#include "mh_kernel.cuh"

namespace gac {

// Chain state of one call: theta [P][N*C] f32, L [N*C] f32, accepted and
// non-finite counters [N*C] i32, adaptation state [2][N*C] i32, Welford mean
// and M2 [P][N*C] f64.  Every
// GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_state[GAC_NOALLOC_STATE_BYTES];

template <int KIND>
__global__ void __launch_bounds__(kBlock, mh_min_blocks<KIND, GAC_PREC_MIXED>()) noalloc_kernel(const ModelConst mc, const RunArgs ra,
                                                            const SliceState ss, int t_begin, int t_end) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int64_t tile = blockIdx.x; tile < ra.n_tiles; tile += gridDim.x)
        run_tile<KIND, GAC_PREC_MIXED, false, true>(mc, ra, ss, tile, t_begin, t_end, smem_raw);
}

static const void *noalloc_fn(int kind) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: return reinterpret_cast<const void *>(&noalloc_kernel<GAC_MODEL_MONOEXP>);
    case GAC_MODEL_MWI3: return reinterpret_cast<const void *>(&noalloc_kernel<GAC_MODEL_MWI3>);
    case GAC_MODEL_SMT: return reinterpret_cast<const void *>(&noalloc_kernel<GAC_MODEL_SMT>);
    case GAC_MODEL_AXCAL_SMT: return reinterpret_cast<const void *>(&noalloc_kernel<GAC_MODEL_AXCAL_SMT>);
    default: return reinterpret_cast<const void *>(&noalloc_kernel<GAC_MODEL_LINEAR_TEST>);
    }
}

static void noalloc_launch(int kind, int grid, size_t smem, cudaStream_t s, const ModelConst &mc,
                           const RunArgs &ra, const SliceState &ss, int t0, int t1) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: noalloc_kernel<GAC_MODEL_MONOEXP><<<grid, kBlock, smem, s>>>(mc, ra, ss, t0, t1); break;
    case GAC_MODEL_MWI3: noalloc_kernel<GAC_MODEL_MWI3><<<grid, kBlock, smem, s>>>(mc, ra, ss, t0, t1); break;
    case GAC_MODEL_SMT: noalloc_kernel<GAC_MODEL_SMT><<<grid, kBlock, smem, s>>>(mc, ra, ss, t0, t1); break;
    case GAC_MODEL_AXCAL_SMT: noalloc_kernel<GAC_MODEL_AXCAL_SMT><<<grid, kBlock, smem, s>>>(mc, ra, ss, t0, t1); break;
    default: noalloc_kernel<GAC_MODEL_LINEAR_TEST><<<grid, kBlock, smem, s>>>(mc, ra, ss, t0, t1); break;
    }
}

// Device address of g_noalloc_state in the current context, looked up on
// every call (a host-side query once the module is loaded), so that a new
// context after a device reset gets its own address (host code only sees a
// host-side stand-in under that name).
static gac_status state_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_state);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(chain-state array)");
    *out = p;
    return GAC_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace gac

using namespace gac;

extern "C" gac_status gac_mcmc_run_noalloc(int model_id, const void *data, int64_t n_vox, const float *sigma,
                                           float sigma_scalar, const float *x0, const gac_mcmc_opts *o,
                                           int slice_iterations, gac_result *out, void *stream) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (n_vox < 0) return fail(GAC_ERR_INVALID_ARG, "n_vox must be >= 0");
    if ((st = validate_opts(o, n_vox)) != GAC_OK) return st;
    if (o->precision != GAC_PREC_MIXED) return fail(GAC_ERR_INVALID_ARG, "only the MIXED precision path");
    if (o->trace_n_vox != 0) return fail(GAC_ERR_INVALID_ARG, "no step tracing here");
    if (slice_iterations < 1) return fail(GAC_ERR_INVALID_ARG, "slice_iterations must be >= 1");
    if (!out) return fail(GAC_ERR_INVALID_ARG, "out must not be NULL");
    if (!sigma && !(sigma_scalar > 0.0f && std::isfinite(sigma_scalar)))
        return fail(GAC_ERR_INVALID_ARG, "sigma is NULL and sigma_scalar is not a positive number");
    if (n_vox == 0) return GAC_OK;
    if (!data) return fail(GAC_ERR_INVALID_ARG, "data must not be NULL");

    const size_t P = mc.n_par, NC = static_cast<size_t>(n_vox) * o->n_chains;
    const size_t off_L = up256(P * NC * 4), off_acc = off_L + up256(NC * 4), off_bad = off_acc + up256(NC * 4);
    const size_t off_ad = off_bad + up256(NC * 4);
    const size_t off_wm = off_ad + up256(2 * NC * 4), off_w2 = off_wm + up256(P * NC * 8);
    // all-post-burn-in moments: the block partials of the FP32 accumulation (3P floats per chain)
    const bool blocked = o->moments_mode == GAC_MOMENTS_ALL_POSTBURNIN;
    const size_t off_blk = off_w2 + up256(P * NC * 8);
    const size_t need = off_blk + (blocked ? up256(3 * P * NC * 4) : 0);
    if (need > GAC_NOALLOC_STATE_BYTES)
        return fail(GAC_ERR_INVALID_ARG,
                    "%lld voxels x %d chains need %zu bytes of chain state; this entry point holds at most %zu",
                    static_cast<long long>(n_vox), o->n_chains, need, static_cast<size_t>(GAC_NOALLOC_STATE_BYTES));
    // every array must already be on the device: staging would allocate
    const void *ptrs[] = {data, sigma, x0, out->mean, out->std, out->samples, out->accept_rate, out->nonfinite,
                          out->rhat, out->step_scale};
    const char *names[] = {"data", "sigma", "x0", "mean", "std", "samples", "accept_rate", "nonfinite",
                           "rhat", "step_scale"};
    for (int i = 0; i < 10; ++i)
        if (ptrs[i] && !is_device_ptr(ptrs[i]))
            return fail(GAC_ERR_INVALID_ARG, "%s must be device memory", names[i]);

    void *base = nullptr;
    if ((st = state_address(&base)) != GAC_OK) return st;
    char *b = static_cast<char *>(base);
    SliceState ss;
    ss.theta = b;
    ss.L = b + off_L;
    ss.n_acc = reinterpret_cast<int32_t *>(b + off_acc);
    ss.n_bad = reinterpret_cast<int32_t *>(b + off_bad);
    ss.adapt = reinterpret_cast<int32_t *>(b + off_ad);
    ss.wf_mean = b + off_wm;
    ss.wf_m2 = b + off_w2;
    ss.blk = blocked ? reinterpret_cast<float *>(b + off_blk) : nullptr;

    RunArgs ra;
    std::memset(&ra, 0, sizeof ra);
    ra.data = static_cast<const float *>(data);
    ra.sigma = sigma;
    ra.sigma_scalar = sigma_scalar;
    ra.x0 = x0;
    ra.mean = out->mean;
    ra.std = out->std;
    ra.samples = out->samples;
    ra.accept = out->accept_rate;
    ra.nonfinite = out->nonfinite;
    ra.n_vox = n_vox;
    ra.C = o->n_chains;
    ra.I = o->iterations;
    ra.B = o->burnin;
    ra.T = o->thin;
    ra.S = n_samples(o->iterations, o->burnin, o->thin);
    ra.k0 = static_cast<uint32_t>(o->seed);
    ra.k1 = static_cast<uint32_t>(o->seed >> 32);
    ra.voxel_base = o->voxel_base;
    ra.moments_mode = o->moments_mode;
    ra.vox_per_block = kBlock / ra.C;
    ra.row_stride = row_stride_for(mc.kind, mc.n_meas);
    ra.data_vec4 = (mc.n_meas % 4 == 0) && ((reinterpret_cast<uintptr_t>(data) & 15) == 0);
    ra.n_tiles = (n_vox + ra.vox_per_block - 1) / ra.vox_per_block;
    set_adaptation(ra, o);
    ra.rhat = out->rhat;
    ra.step_scale = out->step_scale;

    const void *fn = noalloc_fn(mc.kind);
    const size_t smem = tile_smem_bytes(mc.n_par, 8, ra.vox_per_block, ra.row_stride, false, blocked);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(carveout)");
    int per_sm = 0, sms = 0, dev = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, smem)) != cudaSuccess)
        return cuda_fail(e, "occupancy");
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    const int64_t grid = std::min<int64_t>(ra.n_tiles, static_cast<int64_t>(std::max(per_sm, 1)) * std::max(sms, 1));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // one launch per slice; the first slice initialises every chain (state
    // and Welford accumulators), so nothing left in the array matters
    int t0 = 0;
    do {
        const int t1 = static_cast<int>(std::min<int64_t>(o->iterations, static_cast<int64_t>(t0) + slice_iterations));
        noalloc_launch(mc.kind, static_cast<int>(grid), smem, s, mc, ra, ss, t0, t1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sampler launch");
        t0 = t1;
    } while (t0 < o->iterations);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sampler");
    return GAC_OK;
}
