// gac_ensemble_run: host side of the affine-invariant ensemble sampler
// (ens_kernel.cuh), with the staging and validation of gac_mcmc_run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ens_kernel.cuh"
#include "gac.h"
#include "gac_internal.h"

namespace gac {

template <int KIND, int PREC, bool TRACE, bool BLOCKED = false>
static const void *ens_ptr() {
    return reinterpret_cast<const void *>(&ens_kernel<KIND, PREC, TRACE, BLOCKED>);
}

template <int KIND, int PREC, bool TRACE, bool BLOCKED = false>
static cudaError_t ens_go(int grid, size_t smem, cudaStream_t s, const ModelConst &mc, const RunArgs &ra,
                          const EnsArgs &ea, const void **fn) {
    if (fn) {
        *fn = ens_ptr<KIND, PREC, TRACE, BLOCKED>();
        return cudaSuccess;
    }
    ens_kernel<KIND, PREC, TRACE, BLOCKED><<<grid, kEnsBlock, smem, s>>>(mc, ra, ea);
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t ens_by_prec(int prec, bool trace, int grid, size_t smem, cudaStream_t s, const ModelConst &mc,
                               const RunArgs &ra, const EnsArgs &ea, const void **fn) {
    switch (prec) {
    case GAC_PREC_MIXED:
        if (ra.moments_mode == GAC_MOMENTS_ALL_POSTBURNIN)
            return trace ? ens_go<KIND, GAC_PREC_MIXED, true, true>(grid, smem, s, mc, ra, ea, fn)
                         : ens_go<KIND, GAC_PREC_MIXED, false, true>(grid, smem, s, mc, ra, ea, fn);
        return trace ? ens_go<KIND, GAC_PREC_MIXED, true>(grid, smem, s, mc, ra, ea, fn)
                     : ens_go<KIND, GAC_PREC_MIXED, false>(grid, smem, s, mc, ra, ea, fn);
    case GAC_PREC_FP32:
        return trace ? ens_go<KIND, GAC_PREC_FP32, true>(grid, smem, s, mc, ra, ea, fn)
                     : ens_go<KIND, GAC_PREC_FP32, false>(grid, smem, s, mc, ra, ea, fn);
    default:
        return trace ? ens_go<KIND, GAC_PREC_FP64, true>(grid, smem, s, mc, ra, ea, fn)
                     : ens_go<KIND, GAC_PREC_FP64, false>(grid, smem, s, mc, ra, ea, fn);
    }
}

// fn != nullptr: only return the kernel's address; otherwise launch it.
static cudaError_t ens_dispatch(int kind, int prec, bool trace, int grid, size_t smem, cudaStream_t s,
                                const ModelConst &mc, const RunArgs &ra, const EnsArgs &ea, const void **fn) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: return ens_by_prec<GAC_MODEL_MONOEXP>(prec, trace, grid, smem, s, mc, ra, ea, fn);
    case GAC_MODEL_MWI3: return ens_by_prec<GAC_MODEL_MWI3>(prec, trace, grid, smem, s, mc, ra, ea, fn);
    case GAC_MODEL_SMT: return ens_by_prec<GAC_MODEL_SMT>(prec, trace, grid, smem, s, mc, ra, ea, fn);
    case GAC_MODEL_AXCAL_SMT: return ens_by_prec<GAC_MODEL_AXCAL_SMT>(prec, trace, grid, smem, s, mc, ra, ea, fn);
    default: return ens_by_prec<GAC_MODEL_LINEAR_TEST>(prec, trace, grid, smem, s, mc, ra, ea, fn);
    }
}

}  // namespace gac

using namespace gac;

extern "C" gac_status gac_ensemble_run(int model_id, const void *data, int64_t n_vox, const float *sigma,
                                       float sigma_scalar, const float *x0, const gac_mcmc_opts *o,
                                       double stretch, gac_result *out, void *stream) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (n_vox < 0) return fail(GAC_ERR_INVALID_ARG, "n_vox must be >= 0");
    if ((st = validate_opts(o, n_vox)) != GAC_OK) return st;
    const int L = o->n_chains;
    if (L < 4 || (L & 1) || L > 128) return fail(GAC_ERR_INVALID_ARG, "walkers (n_chains) must be even, in [4, 128]");
    if (!(stretch > 1.0) || !(stretch < 1e6)) return fail(GAC_ERR_INVALID_ARG, "stretch must be > 1");
    if (!out) return fail(GAC_ERR_INVALID_ARG, "out must not be NULL");
    if (n_vox > 0 && !data) return fail(GAC_ERR_INVALID_ARG, "data must not be NULL");
    if (!sigma && !(sigma_scalar > 0.0f)) return fail(GAC_ERR_INVALID_ARG, "sigma is NULL and sigma_scalar <= 0");
    if (o->trace_n_vox > 0 && !out->trace) return fail(GAC_ERR_INVALID_ARG, "trace_n_vox > 0 needs out->trace");
    if (o->adapt_window != 0 || out->rhat || out->step_scale)
        return fail(GAC_ERR_INVALID_ARG, "step adaptation, rhat and step_scale belong to the MH sampler");
    if (n_vox == 0) return GAC_OK;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    keep_staging_pool();
    const int P = mc.n_par, M = mc.n_meas, H = L / 2;
    const int S = n_samples(o->iterations, o->burnin, o->thin);
    const size_t N = static_cast<size_t>(n_vox);
    DevBuf d_data, d_sigma, d_x0, d_mean, d_std, d_samples, d_acc, d_bad, d_trace;
    if ((st = d_data.make(const_cast<void *>(data), N * M * sizeof(float), true, s, "data")) != GAC_OK) return st;
    if ((st = d_sigma.make(const_cast<float *>(sigma), sigma ? N * sizeof(float) : 0, true, s, "sigma")) != GAC_OK) return st;
    if ((st = d_x0.make(const_cast<float *>(x0), x0 ? N * L * P * sizeof(float) : 0, true, s, "x0")) != GAC_OK) return st;
    if ((st = d_mean.make(out->mean, P * N * sizeof(double), false, s, "mean")) != GAC_OK) return st;
    if ((st = d_std.make(out->std, P * N * sizeof(double), false, s, "std")) != GAC_OK) return st;
    if ((st = d_samples.make(out->samples, static_cast<size_t>(S) * L * P * N * sizeof(float), false, s, "samples")) != GAC_OK) return st;
    if ((st = d_acc.make(out->accept_rate, L * N * sizeof(float), false, s, "accept_rate")) != GAC_OK) return st;
    if ((st = d_bad.make(out->nonfinite, L * N * sizeof(int32_t), false, s, "nonfinite")) != GAC_OK) return st;
    if ((st = d_trace.make(out->trace, static_cast<size_t>(o->trace_n_vox) * L * o->iterations * sizeof(gac_trace_rec), false, s, "trace")) != GAC_OK) return st;

    RunArgs ra;
    std::memset(&ra, 0, sizeof ra);
    ra.data = static_cast<const float *>(d_data.ptr);
    ra.sigma = static_cast<const float *>(d_sigma.ptr);
    ra.sigma_scalar = sigma_scalar;
    ra.x0 = static_cast<const float *>(d_x0.ptr);
    ra.mean = static_cast<double *>(d_mean.ptr);
    ra.std = static_cast<double *>(d_std.ptr);
    ra.samples = static_cast<float *>(d_samples.ptr);
    ra.accept = static_cast<float *>(d_acc.ptr);
    ra.nonfinite = static_cast<int32_t *>(d_bad.ptr);
    ra.trace = static_cast<gac_trace_rec *>(d_trace.ptr);
    ra.n_vox = n_vox;
    ra.C = L;
    ra.I = o->iterations;
    ra.B = o->burnin;
    ra.T = o->thin;
    ra.S = S;
    ra.k0 = static_cast<uint32_t>(o->seed);
    ra.k1 = static_cast<uint32_t>(o->seed >> 32);
    ra.voxel_base = o->voxel_base;
    ra.moments_mode = o->moments_mode;
    ra.trace_n = o->trace_n_vox;
    ra.vox_per_block = kEnsBlock / H;
    ra.row_stride = row_stride_for(mc.kind, M);
    ra.n_tiles = (n_vox + ra.vox_per_block - 1) / ra.vox_per_block;
    EnsArgs ea;
    ea.stretch = static_cast<float>(stretch);
    ea.inv_stretch = static_cast<float>(1.0 / stretch);
    ea.stretch_d = stretch;
    ea.H = H;

    const bool trace = o->trace_n_vox > 0;
    const size_t rb = o->precision == GAC_PREC_FP64 ? 8 : 4, wb = o->precision == GAC_PREC_FP32 ? 4 : 8;
    const size_t smem = ens_smem_bytes(P, rb, wb, ra.vox_per_block, L, ra.row_stride,
                                       o->precision == GAC_PREC_MIXED && o->moments_mode == GAC_MOMENTS_ALL_POSTBURNIN);
    const void *fn = nullptr;
    ens_dispatch(mc.kind, o->precision, trace, 0, 0, s, mc, ra, ea, &fn);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return cuda_fail(e, "ensemble kernel smem");
    // the walkers' positions and Welford accumulators live in shared memory:
    // prefer the largest carveout, so that the register limit (2 blocks) binds
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return cuda_fail(e, "ensemble kernel carveout");
    int per_sm = 0, sms = 0, dev = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEnsBlock, smem)) != cudaSuccess)
        return cuda_fail(e, "occupancy");
    if (per_sm < 1) return fail(GAC_ERR_INVALID_ARG, "ensemble tile does not fit on an SM (%zu bytes)", smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = static_cast<int>(std::min<int64_t>(ra.n_tiles, static_cast<int64_t>(per_sm) * sms));
    e = ens_dispatch(mc.kind, o->precision, trace, grid, smem, s, mc, ra, ea, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "ensemble kernel launch");
    for (DevBuf *b : {&d_mean, &d_std, &d_samples, &d_acc, &d_bad, &d_trace})
        if ((st = b->copy_out()) != GAC_OK) return st;
    e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? GAC_OK : cuda_fail(e, "ensemble kernel");
}
