// Host-side launch interface between the C ABI (gac.cu) and the kernel
// translation units (one per model kind, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include "mh_kernel.cuh"

namespace gac {

struct LaunchCfg {
    int grid;
    size_t smem;
    cudaStream_t stream;
    int block = kBlock;  // threads per block (the lane-split kernel sizes its blocks)
};

// Returns the kernel for (kind, precision, trace) or nullptr.
const void *mh_kernel_ptr(int kind, int prec, bool trace);
cudaError_t launch_mh(int kind, int prec, bool trace, const ModelConst &mc, const RunArgs &ra,
                      const LaunchCfg &cfg);

// Per-kind entry points defined in mh_<kind>.cu
const void *mh_ptr_monoexp(int prec, bool trace);
const void *mh_ptr_mwi3(int prec, bool trace);
const void *mh_ptr_smt(int prec, bool trace);
const void *mh_ptr_axcal(int prec, bool trace);
const void *mh_ptr_linear(int prec, bool trace);
// Lane-split kernels (mh_split.cuh): G = 2 or 4 lanes per chain, MIXED; all:
// moments over every post-burn-in state.
const void *mh_split_ptr_monoexp(int G, bool all);
const void *mh_split_ptr_mwi3(int G, bool all);
cudaError_t launch_mh_split_monoexp(int G, bool all, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg);
cudaError_t launch_mh_split_mwi3(int G, bool all, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg);
cudaError_t launch_mh_monoexp(int prec, bool trace, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg);
cudaError_t launch_mh_mwi3(int prec, bool trace, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg);
cudaError_t launch_mh_smt(int prec, bool trace, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg);
cudaError_t launch_mh_axcal(int prec, bool trace, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg);
cudaError_t launch_mh_linear(int prec, bool trace, const ModelConst &mc, const RunArgs &ra, const LaunchCfg &cfg);

}  // namespace gac
