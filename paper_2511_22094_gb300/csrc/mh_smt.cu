// Instantiations of the MH kernel for GAC_MODEL_SMT (all precisions, with and
// without step tracing).
#include "launch.h"

namespace gac {

template <int PREC, bool TRACE>
static const void *ptr_of() {
    return reinterpret_cast<const void *>(&mh_kernel<GAC_MODEL_SMT, PREC, TRACE>);
}

const void *mh_ptr_smt(int prec, bool trace) {
    switch (prec) {
    case GAC_PREC_MIXED: return trace ? ptr_of<GAC_PREC_MIXED, true>() : ptr_of<GAC_PREC_MIXED, false>();
    case GAC_PREC_FP32: return trace ? ptr_of<GAC_PREC_FP32, true>() : ptr_of<GAC_PREC_FP32, false>();
    case GAC_PREC_FP64: return trace ? ptr_of<GAC_PREC_FP64, true>() : ptr_of<GAC_PREC_FP64, false>();
    default: return nullptr;
    }
}

template <int PREC, bool TRACE>
static cudaError_t go(const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg) {
    mh_kernel<GAC_MODEL_SMT, PREC, TRACE><<<cfg.grid, (mh_block<GAC_MODEL_SMT, PREC>()), cfg.smem, cfg.stream>>>(mc, ra);
    return cudaGetLastError();
}

cudaError_t launch_mh_smt(int prec, bool trace, const ModelConst &mc, const RunArgs &ra,
                              const LaunchCfg &cfg) {
    switch (prec) {
    case GAC_PREC_MIXED: return trace ? go<GAC_PREC_MIXED, true>(mc, ra, cfg) : go<GAC_PREC_MIXED, false>(mc, ra, cfg);
    case GAC_PREC_FP32: return trace ? go<GAC_PREC_FP32, true>(mc, ra, cfg) : go<GAC_PREC_FP32, false>(mc, ra, cfg);
    case GAC_PREC_FP64: return trace ? go<GAC_PREC_FP64, true>(mc, ra, cfg) : go<GAC_PREC_FP64, false>(mc, ra, cfg);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gac
