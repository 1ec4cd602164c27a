// Test and data-synthesis entry points of the C ABI: the forward model and
// likelihood at given parameters, and the random-number layer.  They run the
// same device functions as the sampler.
#include <cuda_runtime.h>

#include <cstring>

#include "gac.h"
#include "gac_internal.h"
#include "mh_kernel.cuh"

namespace gac {

template <int KIND, int PREC>
__global__ void forward_kernel(const ModelConst mc, const double *theta, int64_t n, double *s) {
    constexpr int P = model_n_par(KIND);
    const int M = mc.n_meas;
    model_smem_load<KIND>(mc);
    __syncthreads();
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double *out = s + i * M;
        if constexpr (PREC == GAC_PREC_FP64) {
            double th[P];
            for (int p = 0; p < P; ++p) th[p] = theta[i * P + p];
            if constexpr (model_complex(KIND))
                eval_d<KIND>(th, mc, [&](int k, double re, double im) { out[2 * k] = re; out[2 * k + 1] = im; });
            else
                eval_d<KIND>(th, mc, [&](int k, double v) { out[k] = v; });
        } else {
            float th[P];
            for (int p = 0; p < P; ++p) th[p] = static_cast<float>(theta[i * P + p]);
            if constexpr (model_complex(KIND))
                eval_f<KIND>(th, mc, [&](int k, float re, float im) { out[2 * k] = re; out[2 * k + 1] = im; });
            else
                eval_f<KIND>(th, mc, [&](int k, float v) { out[k] = v; });
        }
    }
}

template <int KIND, int PREC>
__global__ void loglik_kernel(const ModelConst mc, const double *theta, int64_t n, const float *y,
                              const float *sigma, double *L) {
    constexpr int P = model_n_par(KIND);
    using R = typename PrecTraits<PREC>::R;
    const int M = mc.n_meas;
    model_smem_load<KIND>(mc);
    __syncthreads();
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        R th[P];
        for (int p = 0; p < P; ++p) th[p] = static_cast<R>(theta[i * P + p]);
        const R sg = static_cast<R>(sigma[i]);
        L[i] = static_cast<double>(loglik_any<KIND, PREC>(th, y + i * M, R(1) / (sg * sg), mc));
    }
}

__global__ void philox_kernel(uint32_t k0, uint32_t k1, const uint32_t *t, const uint32_t *v,
                              const uint32_t *c, int64_t n, int nw, uint32_t *out) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        for (int k = 0; 4 * k < nw; ++k) {
            Words4 o = philox4x32_10(t[i], v[i], (c[i] << 8) | static_cast<uint32_t>(k), 0u, k0, k1);
            for (int j = 0; j < 4 && 4 * k + j < nw; ++j) out[i * nw + 4 * k + j] = o.w[j];
        }
    }
}

template <int P, int PREC>
__global__ void normals_kernel(uint32_t k0, uint32_t k1, const uint32_t *t, const uint32_t *v,
                               const uint32_t *c, int64_t n, double *z, uint32_t *w_acc) {
    constexpr int NW = n_words(P);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t w[4 * n_calls(P)];
        draw_words(w, t[i], v[i], c[i], k0, k1);
        for (int j = 0; 2 * j < P; ++j) {
            if constexpr (PREC == GAC_PREC_FP64) {
                double a, b;
                box_muller_d(w[2 * j], w[2 * j + 1], a, b);
                z[i * P + 2 * j] = a;
                if (2 * j + 1 < P) z[i * P + 2 * j + 1] = b;
            } else {
                float a, b;
                box_muller_f(w[2 * j], w[2 * j + 1], a, b);
                z[i * P + 2 * j] = a;
                if (2 * j + 1 < P) z[i * P + 2 * j + 1] = b;
            }
        }
        w_acc[i] = w[NW - 1];
    }
}

static int grid_for(int64_t n) {
    const int64_t blocks = (n + 255) / 256;
    return static_cast<int>(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
}

template <int KIND>
static cudaError_t launch_forward(int prec, const ModelConst &mc, const double *th, int64_t n, double *s,
                                  cudaStream_t st) {
    switch (prec) {
    case GAC_PREC_MIXED: forward_kernel<KIND, GAC_PREC_MIXED><<<grid_for(n), 256, 0, st>>>(mc, th, n, s); break;
    case GAC_PREC_FP32: forward_kernel<KIND, GAC_PREC_FP32><<<grid_for(n), 256, 0, st>>>(mc, th, n, s); break;
    default: forward_kernel<KIND, GAC_PREC_FP64><<<grid_for(n), 256, 0, st>>>(mc, th, n, s); break;
    }
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_loglik(int prec, const ModelConst &mc, const double *th, int64_t n, const float *y,
                                 const float *sg, double *L, cudaStream_t st) {
    switch (prec) {
    case GAC_PREC_MIXED: loglik_kernel<KIND, GAC_PREC_MIXED><<<grid_for(n), 256, 0, st>>>(mc, th, n, y, sg, L); break;
    case GAC_PREC_FP32: loglik_kernel<KIND, GAC_PREC_FP32><<<grid_for(n), 256, 0, st>>>(mc, th, n, y, sg, L); break;
    default: loglik_kernel<KIND, GAC_PREC_FP64><<<grid_for(n), 256, 0, st>>>(mc, th, n, y, sg, L); break;
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_normals_p(int prec, uint64_t seed, const uint32_t *t, const uint32_t *v, const uint32_t *c,
                                   int64_t n, double *z, uint32_t *w, cudaStream_t cs) {
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    if (prec == GAC_PREC_FP64) normals_kernel<P, GAC_PREC_FP64><<<grid_for(n), 256, 0, cs>>>(k0, k1, t, v, c, n, z, w);
    else normals_kernel<P, GAC_PREC_MIXED><<<grid_for(n), 256, 0, cs>>>(k0, k1, t, v, c, n, z, w);
    return cudaGetLastError();
}

}  // namespace gac

using namespace gac;

extern "C" {

gac_status gac_forward(int model_id, const double *theta, int64_t n, int precision, double *s, void *stream) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (n < 0 || (n > 0 && (!theta || !s))) return fail(GAC_ERR_INVALID_ARG, "bad theta/s/n");
    if (precision < GAC_PREC_MIXED || precision > GAC_PREC_FP64)
        return fail(GAC_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (n == 0) return GAC_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    DevBuf dth, ds;
    if ((st = dth.make(const_cast<double *>(theta), n * mc.n_par * sizeof(double), true, cs, "theta")) != GAC_OK) return st;
    if ((st = ds.make(s, n * mc.n_meas * sizeof(double), false, cs, "s")) != GAC_OK) return st;
    const double *th = static_cast<const double *>(dth.ptr);
    double *out = static_cast<double *>(ds.ptr);
    cudaError_t e;
    switch (mc.kind) {
    case GAC_MODEL_MONOEXP: e = launch_forward<GAC_MODEL_MONOEXP>(precision, mc, th, n, out, cs); break;
    case GAC_MODEL_MWI3: e = launch_forward<GAC_MODEL_MWI3>(precision, mc, th, n, out, cs); break;
    case GAC_MODEL_SMT: e = launch_forward<GAC_MODEL_SMT>(precision, mc, th, n, out, cs); break;
    case GAC_MODEL_AXCAL_SMT: e = launch_forward<GAC_MODEL_AXCAL_SMT>(precision, mc, th, n, out, cs); break;
    default: e = launch_forward<GAC_MODEL_LINEAR_TEST>(precision, mc, th, n, out, cs); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "forward kernel launch");
    if ((st = ds.copy_out()) != GAC_OK) return st;
    e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? GAC_OK : cuda_fail(e, "forward kernel");
}

gac_status gac_loglik(int model_id, const double *theta, int64_t n, const float *data, const float *sigma,
                      int precision, double *L, void *stream) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (n < 0 || (n > 0 && (!theta || !data || !sigma || !L))) return fail(GAC_ERR_INVALID_ARG, "bad arguments");
    if (precision < GAC_PREC_MIXED || precision > GAC_PREC_FP64)
        return fail(GAC_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (n == 0) return GAC_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    DevBuf dth, dy, dsg, dl;
    if ((st = dth.make(const_cast<double *>(theta), n * mc.n_par * sizeof(double), true, cs, "theta")) != GAC_OK) return st;
    if ((st = dy.make(const_cast<float *>(data), n * mc.n_meas * sizeof(float), true, cs, "data")) != GAC_OK) return st;
    if ((st = dsg.make(const_cast<float *>(sigma), n * sizeof(float), true, cs, "sigma")) != GAC_OK) return st;
    if ((st = dl.make(L, n * sizeof(double), false, cs, "L")) != GAC_OK) return st;
    const double *th = static_cast<const double *>(dth.ptr);
    const float *y = static_cast<const float *>(dy.ptr);
    const float *sg = static_cast<const float *>(dsg.ptr);
    double *out = static_cast<double *>(dl.ptr);
    cudaError_t e;
    switch (mc.kind) {
    case GAC_MODEL_MONOEXP: e = launch_loglik<GAC_MODEL_MONOEXP>(precision, mc, th, n, y, sg, out, cs); break;
    case GAC_MODEL_MWI3: e = launch_loglik<GAC_MODEL_MWI3>(precision, mc, th, n, y, sg, out, cs); break;
    case GAC_MODEL_SMT: e = launch_loglik<GAC_MODEL_SMT>(precision, mc, th, n, y, sg, out, cs); break;
    case GAC_MODEL_AXCAL_SMT: e = launch_loglik<GAC_MODEL_AXCAL_SMT>(precision, mc, th, n, y, sg, out, cs); break;
    default: e = launch_loglik<GAC_MODEL_LINEAR_TEST>(precision, mc, th, n, y, sg, out, cs); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "loglik kernel launch");
    if ((st = dl.copy_out()) != GAC_OK) return st;
    e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? GAC_OK : cuda_fail(e, "loglik kernel");
}

gac_status gac_philox_words(uint64_t seed, const uint32_t *t, const uint32_t *v, const uint32_t *c, int64_t n,
                            int n_words_, uint32_t *out, void *stream) {
    clear_error();
    if (n < 0 || n_words_ < 1 || n_words_ > 1024 || (n > 0 && (!t || !v || !c || !out)))
        return fail(GAC_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return GAC_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    DevBuf dt, dv, dc, dout;
    gac_status st;
    if ((st = dt.make(const_cast<uint32_t *>(t), n * 4, true, cs, "t")) != GAC_OK) return st;
    if ((st = dv.make(const_cast<uint32_t *>(v), n * 4, true, cs, "v")) != GAC_OK) return st;
    if ((st = dc.make(const_cast<uint32_t *>(c), n * 4, true, cs, "c")) != GAC_OK) return st;
    if ((st = dout.make(out, n * n_words_ * 4, false, cs, "out")) != GAC_OK) return st;
    philox_kernel<<<grid_for(n), 256, 0, cs>>>(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32),
                                              static_cast<const uint32_t *>(dt.ptr), static_cast<const uint32_t *>(dv.ptr),
                                              static_cast<const uint32_t *>(dc.ptr), n, n_words_,
                                              static_cast<uint32_t *>(dout.ptr));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "philox kernel launch");
    if ((st = dout.copy_out()) != GAC_OK) return st;
    e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? GAC_OK : cuda_fail(e, "philox kernel");
}

gac_status gac_normals(uint64_t seed, const uint32_t *t, const uint32_t *v, const uint32_t *c, int64_t n,
                       int n_par, int precision, double *z, uint32_t *w_acc, void *stream) {
    clear_error();
    if (n < 0 || (n > 0 && (!t || !v || !c || !z || !w_acc)))
        return fail(GAC_ERR_INVALID_ARG, "bad arguments");
    if (n_par != 2 && n_par != 4 && n_par != 9)
        return fail(GAC_ERR_INVALID_ARG, "n_par must be 2, 4 or 9 (the registered kinds)");
    if (precision < GAC_PREC_MIXED || precision > GAC_PREC_FP64)
        return fail(GAC_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (n == 0) return GAC_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    DevBuf dt, dv, dc, dz, dw;
    gac_status st;
    if ((st = dt.make(const_cast<uint32_t *>(t), n * 4, true, cs, "t")) != GAC_OK) return st;
    if ((st = dv.make(const_cast<uint32_t *>(v), n * 4, true, cs, "v")) != GAC_OK) return st;
    if ((st = dc.make(const_cast<uint32_t *>(c), n * 4, true, cs, "c")) != GAC_OK) return st;
    if ((st = dz.make(z, n * n_par * sizeof(double), false, cs, "z")) != GAC_OK) return st;
    if ((st = dw.make(w_acc, n * 4, false, cs, "w_acc")) != GAC_OK) return st;
    const uint32_t *pt = static_cast<const uint32_t *>(dt.ptr), *pv = static_cast<const uint32_t *>(dv.ptr),
                   *pc = static_cast<const uint32_t *>(dc.ptr);
    double *pz = static_cast<double *>(dz.ptr);
    uint32_t *pw = static_cast<uint32_t *>(dw.ptr);
    cudaError_t e = n_par == 2 ? launch_normals_p<2>(precision, seed, pt, pv, pc, n, pz, pw, cs)
                  : n_par == 4 ? launch_normals_p<4>(precision, seed, pt, pv, pc, n, pz, pw, cs)
                               : launch_normals_p<9>(precision, seed, pt, pv, pc, n, pz, pw, cs);
    if (e != cudaSuccess) return cuda_fail(e, "normals kernel launch");
    if ((st = dz.copy_out()) != GAC_OK) return st;
    if ((st = dw.copy_out()) != GAC_OK) return st;
    e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? GAC_OK : cuda_fail(e, "normals kernel");
}

}  // extern "C"
