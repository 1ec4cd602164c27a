// Host helpers shared by the translation units of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "gac.h"
#include "models.cuh"

namespace gac {

gac_status fail(gac_status st, const char *fmt, ...);
gac_status cuda_fail(cudaError_t e, const char *what);
void clear_error();
gac_status model_get(int id, ModelConst *out);
bool is_device_ptr(const void *p);
int n_samples(int I, int B, int T);
gac_status validate_opts(const gac_mcmc_opts *o, int64_t n_vox);
int row_stride_for(int kind, int M);
void keep_staging_pool();

// Device view of a caller buffer (see DevBuf::make in gac.cu).
struct DevBuf {
    void *ptr = nullptr;
    void *host = nullptr;
    size_t bytes = 0;
    bool owned = false;
    cudaStream_t stream = nullptr;
    // reread = true: the kernels read the buffer many times (stage page-locked
    // host memory too instead of reading it in place)
    gac_status make(void *user, size_t nbytes, bool in, cudaStream_t s, const char *name, bool reread = false);
    gac_status copy_out();
    ~DevBuf();
};

}  // namespace gac
