// Instantiations of the MH kernel for GAC_MODEL_MONOEXP (all precisions, with and
// without step tracing) and of its lane-split form (MIXED, 2 or 4 lanes).
#include "launch.h"
#include "mh_split.cuh"

namespace gac {

template <int PREC, bool TRACE>
static const void *ptr_of() {
    return reinterpret_cast<const void *>(&mh_kernel<GAC_MODEL_MONOEXP, PREC, TRACE>);
}

const void *mh_ptr_monoexp(int prec, bool trace) {
    switch (prec) {
    case GAC_PREC_MIXED: return trace ? ptr_of<GAC_PREC_MIXED, true>() : ptr_of<GAC_PREC_MIXED, false>();
    case GAC_PREC_FP32: return trace ? ptr_of<GAC_PREC_FP32, true>() : ptr_of<GAC_PREC_FP32, false>();
    case GAC_PREC_FP64: return trace ? ptr_of<GAC_PREC_FP64, true>() : ptr_of<GAC_PREC_FP64, false>();
    default: return nullptr;
    }
}

template <int PREC, bool TRACE>
static cudaError_t go(const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg) {
    mh_kernel<GAC_MODEL_MONOEXP, PREC, TRACE><<<cfg.grid, (mh_block<GAC_MODEL_MONOEXP, PREC>()), cfg.smem, cfg.stream>>>(mc, ra);
    return cudaGetLastError();
}

cudaError_t launch_mh_monoexp(int prec, bool trace, const ModelConst &mc, const RunArgs &ra,
                              const LaunchCfg &cfg) {
    switch (prec) {
    case GAC_PREC_MIXED: return trace ? go<GAC_PREC_MIXED, true>(mc, ra, cfg) : go<GAC_PREC_MIXED, false>(mc, ra, cfg);
    case GAC_PREC_FP32: return trace ? go<GAC_PREC_FP32, true>(mc, ra, cfg) : go<GAC_PREC_FP32, false>(mc, ra, cfg);
    case GAC_PREC_FP64: return trace ? go<GAC_PREC_FP64, true>(mc, ra, cfg) : go<GAC_PREC_FP64, false>(mc, ra, cfg);
    default: return cudaErrorInvalidValue;
    }
}

const void *mh_split_ptr_monoexp(int G, bool all) {
    if (G == 2) return all ? reinterpret_cast<const void *>(&mh_split_kernel<GAC_MODEL_MONOEXP, 2, true>)
                           : reinterpret_cast<const void *>(&mh_split_kernel<GAC_MODEL_MONOEXP, 2, false>);
    if (G == 4) return all ? reinterpret_cast<const void *>(&mh_split_kernel<GAC_MODEL_MONOEXP, 4, true>)
                           : reinterpret_cast<const void *>(&mh_split_kernel<GAC_MODEL_MONOEXP, 4, false>);
    return nullptr;
}

cudaError_t launch_mh_split_monoexp(int G, bool all, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg) {
    const dim3 grid(cfg.grid), block(cfg.block);
    if (G == 2 && all) mh_split_kernel<GAC_MODEL_MONOEXP, 2, true><<<grid, block, cfg.smem, cfg.stream>>>(mc, ra);
    else if (G == 2) mh_split_kernel<GAC_MODEL_MONOEXP, 2, false><<<grid, block, cfg.smem, cfg.stream>>>(mc, ra);
    else if (G == 4 && all) mh_split_kernel<GAC_MODEL_MONOEXP, 4, true><<<grid, block, cfg.smem, cfg.stream>>>(mc, ra);
    else if (G == 4) mh_split_kernel<GAC_MODEL_MONOEXP, 4, false><<<grid, block, cfg.smem, cfg.stream>>>(mc, ra);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace gac
