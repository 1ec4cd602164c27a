// C ABI of libgac.so (include/gac.h): model registry, argument validation,
// host/device pointer handling and the launch of the persistent MH kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gac.h"
#include "gac_internal.h"
#include "launch.h"
#include "mh_split.cuh"

namespace gac {

// ------------------------------------------------------------ errors -------
static thread_local std::string g_last_error;

gac_status fail(gac_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

gac_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky launch error state where possible
    if (e == cudaErrorMemoryAllocation)
        return fail(GAC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(GAC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_last_error.clear(); }

// ----------------------------------------------------------- registry ------
static std::mutex g_reg_mu;
static std::vector<ModelConst> g_models;  // id = index + 1

gac_status model_get(int id, ModelConst *out) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    if (id < 1 || id > static_cast<int>(g_models.size()))
        return fail(GAC_ERR_UNKNOWN_MODEL, "unknown model id %d", id);
    *out = g_models[id - 1];
    return GAC_OK;
}

static bool all_finite(const double *a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// ------------------------------------------------------ pointer kinds ------
bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

DevBuf::~DevBuf() {
    if (owned && ptr) cudaFreeAsync(ptr, stream);
}

// Makes a device view of a caller buffer: device pointers are used in place;
// page-locked host memory is mapped into the device's address space, so the
// kernels read and write it in place (over NVLink-C2C on a Grace-Blackwell
// node: the data crosses once, while the kernel runs, with no staging copy);
// pageable host memory gets a stream-ordered device allocation (copied in
// if `in`, out by copy_out).
gac_status DevBuf::make(void *user, size_t nbytes, bool in, cudaStream_t s, const char *name, bool reread) {
    stream = s;
    bytes = nbytes;
    host = user;
    owned = false;
    if (!user || nbytes == 0) {
        ptr = nullptr;
        return GAC_OK;
    }
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, user) == cudaSuccess) {
        if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
            ptr = user;
            return GAC_OK;
        }
        if (a.type == cudaMemoryTypeHost && a.devicePointer && !reread) {
            ptr = a.devicePointer;
            return GAC_OK;
        }
    } else {
        cudaGetLastError();
    }
    cudaError_t e = cudaMallocAsync(&ptr, nbytes, s);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_fail(e, name);
    }
    owned = true;
    if (in) {
        e = cudaMemcpyAsync(ptr, user, nbytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, name);
    }
    return GAC_OK;
}

gac_status DevBuf::copy_out() {
    if (!owned || !ptr || !host) return GAC_OK;
    cudaError_t e = cudaMemcpyAsync(host, ptr, bytes, cudaMemcpyDeviceToHost, stream);
    return e == cudaSuccess ? GAC_OK : cuda_fail(e, "copy result to host");
}

int n_samples(int I, int B, int T) { return (T > 0 && I > B) ? (I - B) / T : 0; }

// Host buffers are staged through the device's default stream-ordered
// memory pool.  Let the pool keep what a call frees (instead of returning it
// to the driver at every synchronisation), so that repeated calls with host
// buffers do not map gigabytes of staging memory anew each time.  Done once
// per device; a caller that needs the memory back can call cudaMemPoolTrimTo
// on the device's default pool.
void keep_staging_pool() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done[dev] = true;
}

// ------------------------------------------------------ SMT g(x) table ----
// g(x) = int_0^1 exp(-x u^2) du by 40-point Gauss-Legendre quadrature: the
// integrand is entire in u, and for -13 <= x <= 17 the rule agrees with
// 40-digit adaptive quadrature to 2e-15 relative.
namespace {
struct GaussLegendre01 {
    static constexpr int n = 40;
    double node[n], weight[n];  // on [0, 1]
    GaussLegendre01() {
        for (int i = 0; i < n; ++i) {
            // Newton's method on the Legendre polynomial P_n from the
            // asymptotic estimate of its i-th root; P_n by the three-term
            // recurrence, P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1)
            double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double pm = 1.0, p = z;
                for (int j = 2; j <= n; ++j) {
                    const double pn = ((2.0 * j - 1.0) * z * p - (j - 1.0) * pm) / j;
                    pm = p;
                    p = pn;
                }
                dp = n * (z * p - pm) / (z * z - 1.0);
                const double dz = p / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-15) break;
            }
            node[i] = 0.5 * (1.0 + z);
            weight[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2 / ((1 - z^2) P_n'^2)) / 2
        }
    }
    double g(double x) const {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += weight[i] * std::exp(-x * node[i] * node[i]);
        return s;
    }
};
}  // namespace

// Monomial coefficients af[0..K-1] (float) in d of the degree-(K-1)
// polynomial that interpolates f(d) at the K Chebyshev points of [-h, h], and
// the largest relative error of that float polynomial, evaluated in double,
// on 65 points of the interval.
template <int K, class F>
static double cheb_fit(F &&f, float af[K], double h) {
    double T[K][K] = {};  // T[n][m]: coefficient of s^m in the Chebyshev polynomial T_n(s)
    T[0][0] = 1.0;
    T[1][1] = 1.0;
    for (int n = 2; n < K; ++n)
        for (int m = 0; m < K; ++m) T[n][m] = (m > 0 ? 2.0 * T[n - 1][m - 1] : 0.0) - T[n - 2][m];
    double fv[K];
    for (int j = 0; j < K; ++j) fv[j] = f(h * std::cos(M_PI * (j + 0.5) / K));
    double a[K] = {};  // monomial coefficients in s = d / h
    for (int n = 0; n < K; ++n) {
        double b = 0.0;  // Chebyshev coefficient b_n
        for (int j = 0; j < K; ++j) b += fv[j] * std::cos(M_PI * n * (j + 0.5) / K);
        b *= (n == 0 ? 1.0 : 2.0) / K;
        for (int m = 0; m < K; ++m) a[m] += b * T[n][m];
    }
    for (int m = 0; m < K; ++m) af[m] = static_cast<float>(a[m] / std::pow(h, m));  // coefficient of d^m
    double worst = 0.0;
    for (int q = 0; q <= 64; ++q) {
        const double dd = -h + 2.0 * h * q / 64.0;
        double p = af[K - 1];
        for (int m = K - 2; m >= 0; --m) p = p * dd + af[m];
        const double ref = f(dd);
        const double rel = std::fabs(p - ref) / std::fabs(ref);
        worst = (rel > worst || rel != rel) ? rel : worst;
    }
    return worst;
}
template <class F>
static double cheb8_fit(F &&f, float af[8]) {
    return cheb_fit<8>(f, af, 0.5);
}

// Fills mc->gtab with, for each centre c = k/2, k = k_lo .. k_hi, the
// monomial coefficients in d of the degree-5 polynomial that interpolates
// g(c + d) at the six Chebyshev points of [-1/4, 1/4], and checks every
// interval on 65 points against the quadrature (relative error of the float
// coefficients evaluated in double at most 2e-7; the interpolation error
// itself is about 1e-8 on quarter-width half-intervals).  k_hi = the centre
// nearest xmax (the largest argument the model's bounds allow) when that fits
// in kGTabMax intervals: then the kernels need no asymptote.  Otherwise the
// table ends at a centre >= 16 and x >= c_hi + 1/4 takes sqrt(pi)/2 x^-1/2.
static gac_status build_g_table(double xmin, double xmax, ModelConst *mc) {
    static const GaussLegendre01 gl;
    const int k_lo = static_cast<int>(std::floor(2.0 * xmin - 0.5));
    if (k_lo < 2 * static_cast<int>(kSmtArgMin) - 2)
        return fail(GAC_ERR_INVALID_ARG, "SMT argument range starts at %g, below %d", xmin,
                    static_cast<int>(kSmtArgMin));
    const double k_need = std::max(std::ceil(2.0 * xmax - 0.5), 2.0 * kGTail);
    const int n_int = static_cast<int>(std::min<double>(kGTabMax, k_need - k_lo + 1));
    const int k_hi = k_lo + n_int - 1;
    if (k_hi < 2 * static_cast<int>(kGTail)) return fail(GAC_ERR_INVALID_ARG, "g(x) table too short");
    for (int i = 0; i < n_int; ++i) {
        const double c = 0.5 * (k_lo + i);
        float af[6];
        const double err = cheb_fit<6>([&](double d) { return gl.g(c + d); }, af, 0.25);
        for (int m = 0; m < 4; ++m) mc->gtab[i * 4 + m] = af[m];
        mc->gtab[(kGTabMax + i) * 4 + 0] = af[4];
        mc->gtab[(kGTabMax + i) * 4 + 1] = af[5];
        mc->gtab[(kGTabMax + i) * 4 + 2] = 0.0f;
        mc->gtab[(kGTabMax + i) * 4 + 3] = 0.0f;
        if (!(err <= 2e-7)) return fail(GAC_ERR_INVALID_ARG, "g(x) table check failed near x = %g", c);
    }
    const int c_lo = k_lo;
    const double c_hi = 0.5 * k_hi;
    mc->gtab_lo = c_lo;
    mc->gtab_n = n_int;
    mc->gtab_tail = c_hi + 0.25 >= xmax ? 0 : 1;
    mc->gtab_tail_x = static_cast<float>(c_hi + 0.25);
    return GAC_OK;
}

// ------------------------------------------------- AxCaliberSMT constants --
// m-th positive zero of J1' (m >= 1): Newton's method on J1'(x) = J0(x) -
// J1(x)/x, with J1''(x) = -J1'(x)/x - (1 - 1/x^2) J1(x) from Bessel's
// equation, from McMahon's estimate (m - 1/4) pi - 7 / (8 (m - 1/4) pi).
static double j1p_zero(int m) {
    const double beta = (m - 0.25) * M_PI;
    double x = beta - 7.0 / (8.0 * beta);
    for (int it = 0; it < 50; ++it) {
        const double j0 = std::cyl_bessel_j(0.0, x), j1 = std::cyl_bessel_j(1.0, x);
        const double d1 = j0 - j1 / x;
        const double d2 = -d1 / x - (1.0 - 1.0 / (x * x)) * j1;
        const double step = d1 / d2;
        x -= step;
        if (std::fabs(step) < 1e-15 * x) break;
    }
    return x;
}

// N_m of the cylinder series in double (see ax_n_series_f for the forms).
static double ax_n_host(double q, double dl, double DL) {
    const double a = q * dl;
    if (a < 1.0) return 2.0 * (std::expm1(-a) + a) - std::exp(-q * DL) * (std::expm1(a) + std::expm1(-a));
    return 2.0 * a - 2.0 + 2.0 * (std::exp(-a) + std::exp(-q * DL)) - std::exp(-q * (DL - dl)) - std::exp(-q * (DL + dl));
}

// Per-measurement constants, distinct timings, series coefficients and the
// number of terms: the FP32 evaluation keeps the terms whose tail stays below
// 2e-8 of the sum for every timing at 64 radii spanning the prior box; the
// FP64 evaluation keeps all kAxMaxTerms.
static gac_status build_axcal(const gac_model_desc *d, ModelConst *mc) {
    AxConst &ax = mc->ax;
    const int K = d->n_acq / 3;
    if (K > kAxMaxMeas) return fail(GAC_ERR_INVALID_ARG, "at most %d AxCaliberSMT measurements", kAxMaxMeas);
    ax.n_timing = 0;
    for (int k = 0; k < K; ++k) {
        const double b = d->acq[3 * k], Delta = d->acq[3 * k + 1], delta = d->acq[3 * k + 2];
        int t = 0;
        while (t < ax.n_timing && !(ax.Delta_d[t] == Delta && ax.delta_d[t] == delta)) ++t;
        if (t == ax.n_timing) {
            if (t == kAxMaxTiming) return fail(GAC_ERR_INVALID_ARG, "at most %d distinct (Delta, delta)", kAxMaxTiming);
            ax.Delta_d[t] = Delta;
            ax.delta_d[t] = delta;
            ax.Delta_f[t] = static_cast<float>(Delta);
            ax.delta_f[t] = static_cast<float>(delta);
            ++ax.n_timing;
        }
        ax.t[k] = t;
        const double g2 = b / (delta * delta * (Delta - delta / 3.0));
        ax.b_d[k] = b;
        ax.g2_d[k] = g2;
        ax.csf_d[k] = std::exp(-b * kAxDcsfD);
        ax.b_f[k] = static_cast<float>(b);
        ax.g2_f[k] = static_cast<float>(g2);
        ax.csf_f[k] = static_cast<float>(ax.csf_d[k]);
    }
    // the FP32 path's measurements in timing order (stable), with their constants
    constexpr double kLog2e = 1.44269504088896340736;
    int pos = 0;
    for (int t = 0; t < ax.n_timing; ++t) {
        ax.first[t] = pos;
        for (int k = 0; k < K; ++k) {
            if (ax.t[k] != t) continue;
            float *m = ax.meas + 8 * pos++;
            m[0] = static_cast<float>(ax.b_d[k] * kAxDaD);
            m[1] = static_cast<float>(ax.g2_d[k]);
            m[2] = static_cast<float>(ax.g2_d[k] * kLog2e);
            m[3] = static_cast<float>(ax.b_d[k] * kLog2e);
            m[4] = static_cast<float>(ax.b_d[k]);
            m[5] = ax.csf_f[k];
            std::memcpy(&m[6], &k, sizeof k);
            m[7] = 0.0f;
        }
    }
    for (int t = ax.n_timing; t <= kAxMaxTiming; ++t) ax.first[t] = pos;
    double x2d[kAxMaxTerms], c[kAxMaxTerms];
    for (int m = 0; m < kAxMaxTerms; ++m) {
        const double x = j1p_zero(m + 1), x2 = x * x;
        x2d[m] = x2 * kAxDaD;
        c[m] = 2.0 / (kAxDaD * kAxDaD * x2 * x2 * x2 * (x2 - 1.0));
        ax.x2d_d[m] = x2d[m];
        ax.c_d[m] = c[m];
        ax.x2d_f[m] = static_cast<float>(x2d[m]);
        ax.c_f[m] = static_cast<float>(c[m]);
    }
    ax.terms_d = kAxMaxTerms;
    const double r_lo = 0.5 * d->lb[0], r_hi = 0.5 * d->ub[0];
    int terms = 1;
    for (int t = 0; t < ax.n_timing; ++t)
        for (int i = 0; i < 64; ++i) {
            const double R = r_lo * std::pow(r_hi / r_lo, i / 63.0), r2 = R * R;
            double term[kAxMaxTerms], total = 0.0;
            for (int m = 0; m < kAxMaxTerms; ++m) total += term[m] = c[m] * ax_n_host(x2d[m] / r2, ax.delta_d[t], ax.Delta_d[t]);
            double tail = total;
            int need = 0;
            while (need < kAxMaxTerms && tail > 2e-8 * total) tail -= term[need++];
            terms = std::max(terms, need);
        }
    ax.terms_f = terms;
    double dmin = ax.delta_d[0];
    for (int t = 1; t < ax.n_timing; ++t) dmin = std::min(dmin, ax.delta_d[t]);
    ax.careful_f = 0;
    while (ax.careful_f < ax.terms_f && x2d[ax.careful_f] / (r_hi * r_hi) * dmin < 1.0) ++ax.careful_f;
    // the FP32 table of phi_j(R) = R^6 sum_m c_m N_m in u = log2 R: intervals
    // of width <= 1/2 over the prior box (at most kAxTabMax, widened if the
    // box is wider), each checked on 65 points; if any check exceeds 3e-7 the
    // kernels sum the series instead
    const double u_lo = std::log2(r_lo), u_hi = std::log2(r_hi);
    const int n_int = std::min(kAxTabMax, std::max(1, static_cast<int>(std::ceil((u_hi - u_lo) / 0.5))));
    const double w = std::max(u_hi - u_lo, 1e-3) / n_int;
    bool ok = true;
    for (int t = 0; t < ax.n_timing && ok; ++t)
        for (int i = 0; i < n_int && ok; ++i) {
            const double uc = u_lo + (i + 0.5) * w;
            auto phi = [&](double dd) {
                const double R = std::exp2(uc + dd * w), r2 = R * R;
                double sum = 0.0;
                for (int m = 0; m < kAxMaxTerms; ++m) sum += c[m] * ax_n_host(x2d[m] / r2, ax.delta_d[t], ax.Delta_d[t]);
                return r2 * r2 * r2 * sum;
            };
            float af[8];
            ok = cheb8_fit(phi, af) <= 3e-7;
            for (int m = 0; m < 8; ++m) ax.tab[((2 * t + (m < 4 ? 0 : 1)) * kAxTabMax + i) * 4 + (m & 3)] = af[m];
        }
    ax.tab_n = ok ? n_int : 0;
    ax.tab_inv_w = static_cast<float>(1.0 / w);
    ax.tab_off = static_cast<float>(-u_lo / w - 0.5);
    return GAC_OK;
}

// ----------------------------------------------------- launch sizing -------
static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int row_stride_for(int kind, int M) {
    // odd stride in the unit the kernel reads (float, or float2 for complex)
    // so that the voxels of a warp fall into distinct shared-memory banks
    if (model_complex(kind)) return 2 * ((M / 2) | 1);
    return M | 1;
}

template <int KIND>
static int block_of(int prec) {
    switch (prec) {
    case GAC_PREC_MIXED: return mh_block<KIND, GAC_PREC_MIXED>();
    case GAC_PREC_FP32: return mh_block<KIND, GAC_PREC_FP32>();
    default: return mh_block<KIND, GAC_PREC_FP64>();
    }
}

// Threads per block of the one-launch kernel for (kind, precision).
int mh_block_size(int kind, int prec) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: return block_of<GAC_MODEL_MONOEXP>(prec);
    case GAC_MODEL_MWI3: return block_of<GAC_MODEL_MWI3>(prec);
    case GAC_MODEL_SMT: return block_of<GAC_MODEL_SMT>(prec);
    case GAC_MODEL_AXCAL_SMT: return block_of<GAC_MODEL_AXCAL_SMT>(prec);
    default: return block_of<GAC_MODEL_LINEAR_TEST>(prec);
    }
}

size_t smem_bytes_for(int kind, int prec, int C, int M, int moments_mode) {
    const size_t w = (prec == GAC_PREC_FP32) ? sizeof(float) : sizeof(double);
    const bool blocked = prec == GAC_PREC_MIXED && moments_mode == GAC_MOMENTS_ALL_POSTBURNIN;
    const int block = mh_block_size(kind, prec);
    return tile_smem_bytes(model_n_par(kind), w, block / C, row_stride_for(kind, M), true, blocked, block);
}

const void *mh_kernel_ptr(int kind, int prec, bool trace) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: return mh_ptr_monoexp(prec, trace);
    case GAC_MODEL_MWI3: return mh_ptr_mwi3(prec, trace);
    case GAC_MODEL_SMT: return mh_ptr_smt(prec, trace);
    case GAC_MODEL_AXCAL_SMT: return mh_ptr_axcal(prec, trace);
    case GAC_MODEL_LINEAR_TEST: return mh_ptr_linear(prec, trace);
    default: return nullptr;
    }
}

cudaError_t launch_mh(int kind, int prec, bool trace, const ModelConst &mc, const RunArgs &ra,
                      const LaunchCfg &cfg) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: return launch_mh_monoexp(prec, trace, mc, ra, cfg);
    case GAC_MODEL_MWI3: return launch_mh_mwi3(prec, trace, mc, ra, cfg);
    case GAC_MODEL_SMT: return launch_mh_smt(prec, trace, mc, ra, cfg);
    case GAC_MODEL_AXCAL_SMT: return launch_mh_axcal(prec, trace, mc, ra, cfg);
    case GAC_MODEL_LINEAR_TEST: return launch_mh_linear(prec, trace, mc, ra, cfg);
    default: return cudaErrorInvalidValue;
    }
}

// Grid: one block per tile of voxels, capped at the number of blocks that
// are resident at once (the kernel strides over the remaining tiles).
gac_status plan_launch(const ModelConst &mc, int prec, bool trace, int C, int64_t n_vox, int moments_mode,
                       LaunchCfg *cfg, int64_t *n_tiles, int *vb) {
    const void *fn = mh_kernel_ptr(mc.kind, prec, trace);
    if (!fn) return fail(GAC_ERR_INVALID_ARG, "no kernel for kind %d precision %d", mc.kind, prec);
    const size_t smem = smem_bytes_for(mc.kind, prec, C, mc.n_meas, moments_mode);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    // prefer the largest shared-memory carveout: the tile and Welford
    // accumulators, not L1, decide how many blocks fit
    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(carveout)");
    int per_sm = 0;
    const int block = mh_block_size(mc.kind, prec);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(GAC_ERR_INVALID_ARG, "kernel does not fit on an SM (smem %zu)", smem);
    // Voxels per tile: a full block's worth, unless the problem is too small
    // to give every resident block a full tile; then tiles shrink (in whole
    // warps of chains) so that the chains spread over all SMs instead of
    // crowding a few -- a small problem is bound by the latency of one
    // iteration, which a warp alone on its SM sub-partition runs fastest.
    // The block's remaining threads stay idle; results do not depend on the
    // tiling (random numbers are keyed by voxel, chain and iteration).
    const int64_t resident = static_cast<int64_t>(per_sm) * sm_count();
    const int64_t chains = n_vox * C;
    int threads = block;
    if (chains < resident * block) {
        const int64_t want = (chains + resident - 1) / resident;  // chains per block
        threads = static_cast<int>(std::min<int64_t>(block, std::max<int64_t>(32, (want + 31) / 32 * 32)));
    }
    *vb = std::max(1, threads / C);
    *n_tiles = (n_vox + *vb - 1) / *vb;
    cfg->grid = static_cast<int>(std::min<int64_t>(*n_tiles, resident));
    cfg->smem = smem;
    return GAC_OK;
}

gac_status validate_opts(const gac_mcmc_opts *o, int64_t n_vox) {
    if (!o) return fail(GAC_ERR_INVALID_ARG, "opts is NULL");
    if (o->iterations < 0 || o->iterations == INT32_MAX)
        return fail(GAC_ERR_INVALID_ARG, "iterations must be in [0, 2^31-2]");
    if (o->burnin < 0) return fail(GAC_ERR_INVALID_ARG, "burnin must be >= 0");
    if (o->thin < 1) return fail(GAC_ERR_INVALID_ARG, "thin must be >= 1");
    if (o->n_chains < 1 || o->n_chains > 64) return fail(GAC_ERR_INVALID_ARG, "n_chains must be in [1, 64]");
    if (o->precision < GAC_PREC_MIXED || o->precision > GAC_PREC_FP64)
        return fail(GAC_ERR_INVALID_ARG, "unknown precision %d", o->precision);
    if (o->moments_mode != GAC_MOMENTS_THINNED && o->moments_mode != GAC_MOMENTS_ALL_POSTBURNIN)
        return fail(GAC_ERR_INVALID_ARG, "unknown moments_mode %d", o->moments_mode);
    if (o->trace_n_vox < 0 || o->trace_n_vox > n_vox)
        return fail(GAC_ERR_INVALID_ARG, "trace_n_vox must be in [0, n_vox]");
    if (o->adapt_window < 0) return fail(GAC_ERR_INVALID_ARG, "adapt_window must be >= 0");
    if (o->adapt_window > 0 && !(o->adapt_target > 0.0 && o->adapt_target < 1.0))
        return fail(GAC_ERR_INVALID_ARG, "adapt_target must be in (0, 1)");
    if (o->voxel_base > (1ull << 32) || static_cast<uint64_t>(n_vox) > (1ull << 32) - o->voxel_base)
        return fail(GAC_ERR_INVALID_ARG, "voxel_base + n_vox must be <= 2^32 (32-bit counter word)");
    if (o->lanes_per_chain != 0 && o->lanes_per_chain != 1 && o->lanes_per_chain != 2 && o->lanes_per_chain != 4)
        return fail(GAC_ERR_INVALID_ARG, "lanes_per_chain must be 0, 1, 2 or 4");
    return GAC_OK;
}

// Lanes per chain of a gac_mcmc_run (1: the one-thread kernel).  The
// lane-split kernel handles MIXED runs without trace of the mono-exponential
// and 3-pool models with evenly spaced echoes in 2..4 blocks of kAnchor; the
// library uses it when the chains would give fewer than one warp per SM
// sub-partition (there it shortens the latency of an iteration; on larger
// problems one thread per chain keeps more chains in flight).
static gac_status choose_lanes(const ModelConst &mc, const gac_mcmc_opts *o, int64_t n_vox, int *lanes) {
    const int nb = (mc.n_acq + kAnchor - 1) / kAnchor;
    const bool eligible = o->precision == GAC_PREC_MIXED && o->trace_n_vox == 0 && mc.even &&
                          (mc.kind == GAC_MODEL_MONOEXP || mc.kind == GAC_MODEL_MWI3) && nb >= 2 && nb <= 4;
    *lanes = 1;
    if (o->lanes_per_chain == 1) return GAC_OK;
    if (o->lanes_per_chain > 1) {
        if (!eligible || nb > o->lanes_per_chain)
            return fail(GAC_ERR_INVALID_ARG,
                        "lanes_per_chain %d needs MIXED precision, no trace and a mono-exponential or 3-pool "
                        "model with evenly spaced echoes in at most %d blocks of %d",
                        o->lanes_per_chain, o->lanes_per_chain, kAnchor);
        *lanes = o->lanes_per_chain;
        return GAC_OK;
    }
    const int64_t one_warp_each = static_cast<int64_t>(sm_count()) * 4 * 32;
    if (eligible && n_vox * o->n_chains < one_warp_each) *lanes = nb <= 2 ? 2 : 4;
    return GAC_OK;
}

// Lane-split launch: blocks just large enough to give every SM the same
// number of warps (whole voxels per block), as many as fit at once.
static gac_status plan_split(const ModelConst &mc, int G, int C, int64_t n_vox, int moments_mode, LaunchCfg *cfg,
                             int64_t *n_tiles, int *vb) {
    const bool all = moments_mode == GAC_MOMENTS_ALL_POSTBURNIN;
    const void *fn = mc.kind == GAC_MODEL_MONOEXP ? mh_split_ptr_monoexp(G, all) : mh_split_ptr_mwi3(G, all);
    if (!fn) return fail(GAC_ERR_INVALID_ARG, "no lane-split kernel for kind %d with %d lanes", mc.kind, G);
    const int sms = sm_count();
    const int64_t warps = (n_vox * C * G + 31) / 32;
    int threads = static_cast<int>(std::min<int64_t>(kBlock, 32 * ((warps + sms - 1) / sms)));
    threads = std::max(threads, 32 * ((C * G + 31) / 32));  // at least one voxel
    *vb = std::max(1, threads / (C * G));
    const size_t smem = split_smem_bytes(mc.n_par, G, threads, *vb, row_stride_for(mc.kind, mc.n_meas), all);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem)) != cudaSuccess)
        return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(GAC_ERR_INVALID_ARG, "lane-split kernel does not fit on an SM (smem %zu)", smem);
    *n_tiles = (n_vox + *vb - 1) / *vb;
    cfg->grid = static_cast<int>(std::min<int64_t>(*n_tiles, static_cast<int64_t>(per_sm) * sms));
    cfg->smem = smem;
    cfg->block = threads;
    return GAC_OK;
}

}  // namespace gac

using namespace gac;

// ===================================================================== ABI ==
extern "C" {

const char *gac_last_error(void) { return g_last_error.c_str(); }

const char *gac_version(void) { return "gac 0.1 (sm_103a)"; }

gac_status gac_model_register(const gac_model_desc *d, int *model_id) {
    clear_error();
    if (!d || !model_id) return fail(GAC_ERR_INVALID_ARG, "desc and model_id must not be NULL");
    const int P = model_n_par(d->kind);
    if (P < 0) return fail(GAC_ERR_UNKNOWN_MODEL, "unknown model kind %d", d->kind);
    if (d->n_par != P) return fail(GAC_ERR_INVALID_ARG, "kind %d has %d parameters, n_par = %d", d->kind, P, d->n_par);
    if (d->n_acq < 1 || d->n_acq > GAC_MAX_ACQ)
        return fail(GAC_ERR_INVALID_ARG, "n_acq must be in [1, %d]", GAC_MAX_ACQ);
    if (!d->acq || !d->lb || !d->ub || !d->step)
        return fail(GAC_ERR_INVALID_ARG, "acq, lb, ub and step must not be NULL");
    if (!all_finite(d->acq, d->n_acq) || !all_finite(d->lb, P) || !all_finite(d->ub, P) ||
        !all_finite(d->step, P))
        return fail(GAC_ERR_INVALID_ARG, "non-finite acquisition, bound or step");
    for (int p = 0; p < P; ++p) {
        if (d->lb[p] > d->ub[p]) return fail(GAC_ERR_INVALID_ARG, "lb[%d] > ub[%d]", p, p);
        if (d->step[p] < 0) return fail(GAC_ERR_INVALID_ARG, "step[%d] < 0", p);
    }
    if (d->kind == GAC_MODEL_MWI3) {
        for (int j = 3; j < 6; ++j)
            if (d->lb[j] <= 0) return fail(GAC_ERR_INVALID_ARG, "T2* lower bounds must be > 0");
        // phase arguments phi0 - 2 pi df t must stay in the range of sincos_cw
        double tmax = 0, dfmax = 0;
        for (int k = 0; k < d->n_acq; ++k) tmax = std::max(tmax, std::fabs(d->acq[k]));
        for (int j = 6; j < 8; ++j) dfmax = std::max({dfmax, std::fabs(d->lb[j]), std::fabs(d->ub[j])});
        const double amax = std::max(std::fabs(d->lb[8]), std::fabs(d->ub[8])) + kTwoPiMilliD * dfmax * tmax * (kAnchor + 1);
        if (amax > kSinCosMaxArg)
            return fail(GAC_ERR_INVALID_ARG, "phase range %.0f rad exceeds %.0f", amax, static_cast<double>(kSinCosMaxArg));
    }
    if (d->kind == GAC_MODEL_SMT) {
        for (int k = 0; k < d->n_acq; ++k) {
            const double b = d->acq[k];
            if (b < 0) return fail(GAC_ERR_INVALID_ARG, "b-values must be >= 0");
            if (b * (d->lb[2] - d->ub[3]) < kSmtArgMin || b * d->lb[1] < kSmtArgMin)
                return fail(GAC_ERR_INVALID_ARG,
                            "SMT bounds outside the validated range: need b*(ub[De_perp]-lb[De_par]) <= 12");
        }
    }

    if (d->kind == GAC_MODEL_AXCAL_SMT) {
        if (d->n_acq % 3 != 0) return fail(GAC_ERR_INVALID_ARG, "AxCaliberSMT takes (b, Delta, delta) triplets");
        for (int k = 0; k < d->n_acq / 3; ++k) {
            const double b = d->acq[3 * k], Delta = d->acq[3 * k + 1], delta = d->acq[3 * k + 2];
            if (b < 0 || !(delta > 0) || !(Delta >= delta))
                return fail(GAC_ERR_INVALID_ARG, "measurement %d: need b >= 0, delta > 0, Delta >= delta", k);
            if (b * (d->ub[3] - kAxDeParD) > -kSmtArgMin)
                return fail(GAC_ERR_INVALID_ARG, "AxCaliberSMT bounds outside the validated range: b*(ub[De_R]-1.7) <= 12");
        }
        if (!(d->lb[0] > 0)) return fail(GAC_ERR_INVALID_ARG, "the axon diameter's lower bound must be > 0");
    }

    ModelConst mc;
    std::memset(&mc, 0, sizeof mc);
    mc.kind = d->kind;
    mc.n_par = P;
    mc.n_acq = d->n_acq;
    mc.n_meas = model_complex(d->kind) ? 2 * d->n_acq : (d->kind == GAC_MODEL_AXCAL_SMT ? d->n_acq / 3 : d->n_acq);
    for (int k = 0; k < d->n_acq; ++k) {
        mc.acq_d[k] = d->acq[k];
        mc.acq_f[k] = static_cast<float>(d->acq[k]);
        mc.acq_l2e_f[k] = static_cast<float>(d->acq[k] * 1.44269504088896340736);
    }
    for (int p = 0; p < P; ++p) {
        mc.lb_d[p] = d->lb[p];
        mc.ub_d[p] = d->ub[p];
        mc.step_d[p] = d->step[p];
        mc.lb_f[p] = static_cast<float>(d->lb[p]);
        mc.ub_f[p] = static_cast<float>(d->ub[p]);
        mc.step_f[p] = static_cast<float>(d->step[p]);
    }
    // evenly spaced acquisitions (to 1e-9 relative) allow the recurrence
    mc.even = 0;
    if (d->n_acq >= 2) {
        const double t0 = d->acq[0];
        const double dt = (d->acq[d->n_acq - 1] - t0) / (d->n_acq - 1);
        bool even = dt > 0;
        for (int k = 0; k < d->n_acq && even; ++k) {
            const double want = t0 + k * dt;
            if (std::fabs(d->acq[k] - want) > 1e-9 * std::max(1.0, std::fabs(want))) even = false;
        }
        if (even) {
            mc.even = 1;
            mc.t0_f = static_cast<float>(t0);
            mc.dt_f = static_cast<float>(dt);
            mc.dtk_f = static_cast<float>(kAnchor * dt);
            auto dd = [](double x) {
                const float hi = static_cast<float>(x);
                return make_float2(hi, static_cast<float>(x - static_cast<double>(hi)));
            };
            mc.dd_t0 = dd(t0);
            mc.dd_dt = dd(dt);
            mc.dd_w0 = dd(kTwoPiMilliD * t0);
            mc.dd_w1 = dd(kTwoPiMilliD * dt);
            mc.dd_wk = dd(kTwoPiMilliD * kAnchor * dt);
            if (d->kind == GAC_MODEL_MWI3) {
                // the 3-pool set-up evaluates e^{-t/T2*} - 1 for t = t0, dt >= 0 only
                if (t0 < 0) mc.even = 0;
                double dfmax = 0;
                for (int j = 6; j < 8; ++j) dfmax = std::max({dfmax, std::fabs(d->lb[j]), std::fabs(d->ub[j])});
                const double bmax = kTwoPiMilliD * dfmax * std::max(std::fabs(t0), dt);
                const double bkh = kTwoPiMilliD * dfmax * 0.5 * kAnchor * dt;
                mc.dd_wkh = dd(kTwoPiMilliD * 0.5 * kAnchor * dt);
                mc.mwi3_flags = (bmax <= 0.78 ? kMwi3SmallB : 0) | (bkh <= 0.78 ? kMwi3SmallBK : 0) |
                                (std::max(t0, dt) / d->lb[5] <= 0.34 ? kMwi3SmallEW : 0);  // pi/4, ln2/2
            }
        }
    }
    if (d->kind == GAC_MODEL_SMT) {
        // the smallest and largest arguments b Da, b (De_par - De_perp) the bounds allow
        double xmin = 0.0, xmax = 0.0;
        for (int k = 0; k < d->n_acq; ++k) {
            xmin = std::min({xmin, d->acq[k] * d->lb[1], d->acq[k] * (d->lb[2] - d->ub[3])});
            xmax = std::max({xmax, d->acq[k] * d->ub[1], d->acq[k] * (d->ub[2] - d->lb[3])});
        }
        const gac_status st = build_g_table(xmin, xmax, &mc);
        if (st != GAC_OK) return st;
    }
    if (d->kind == GAC_MODEL_AXCAL_SMT) {
        gac_status st = build_axcal(d, &mc);
        if (st != GAC_OK) return st;
        // g arguments: 0 <= b Da - kappa <= b Da (up to rounding) and b (1.7 - De_R)
        double xmin = -1.0, xmax = 0.0;
        for (int k = 0; k < mc.n_meas; ++k) {
            const double b = d->acq[3 * k];
            xmin = std::min(xmin, b * (kAxDeParD - d->ub[3]));
            xmax = std::max({xmax, b * kAxDaD, b * (kAxDeParD - d->lb[3])});
        }
        if ((st = build_g_table(xmin, xmax, &mc)) != GAC_OK) return st;
    }
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (size_t i = 0; i < g_models.size(); ++i)  // ModelConst is zero-filled before it is set
        if (std::memcmp(&g_models[i], &mc, sizeof mc) == 0) {
            *model_id = static_cast<int>(i + 1);
            return GAC_OK;
        }
    if (g_models.size() >= GAC_MAX_MODELS)
        return fail(GAC_ERR_INVALID_ARG, "at most %d models can be registered", GAC_MAX_MODELS);
    g_models.push_back(mc);
    *model_id = static_cast<int>(g_models.size());
    return GAC_OK;
}

gac_status gac_model_info(int model_id, int *n_par, int *n_meas) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (n_par) *n_par = mc.n_par;
    if (n_meas) *n_meas = mc.n_meas;
    return GAC_OK;
}

gac_status gac_result_sizes(int model_id, int64_t n_vox, const gac_mcmc_opts *o, size_t bytes[8]) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (!bytes) return fail(GAC_ERR_INVALID_ARG, "bytes must not be NULL");
    if (n_vox < 0) return fail(GAC_ERR_INVALID_ARG, "n_vox must be >= 0");
    if ((st = validate_opts(o, n_vox)) != GAC_OK) return st;
    const size_t N = static_cast<size_t>(n_vox), P = mc.n_par, C = o->n_chains;
    const size_t S = n_samples(o->iterations, o->burnin, o->thin);
    bytes[0] = P * N * sizeof(double);
    bytes[1] = P * N * sizeof(double);
    bytes[2] = S * C * P * N * sizeof(float);
    bytes[3] = C * N * sizeof(float);
    bytes[4] = C * N * sizeof(int32_t);
    bytes[5] = static_cast<size_t>(o->trace_n_vox) * C * o->iterations * sizeof(gac_trace_rec);
    bytes[6] = P * N * sizeof(double);
    bytes[7] = C * N * sizeof(float);
    return GAC_OK;
}

gac_status gac_mcmc_run(int model_id, const void *data, int64_t n_vox, const float *sigma,
                        float sigma_scalar, const float *x0, const gac_mcmc_opts *o,
                        gac_result *out, void *stream) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (n_vox < 0) return fail(GAC_ERR_INVALID_ARG, "n_vox must be >= 0");
    if ((st = validate_opts(o, n_vox)) != GAC_OK) return st;
    if (!out) return fail(GAC_ERR_INVALID_ARG, "out must not be NULL");
    if (n_vox > 0 && !data) return fail(GAC_ERR_INVALID_ARG, "data must not be NULL");
    if (!sigma && !(sigma_scalar > 0.0f && std::isfinite(sigma_scalar)))
        return fail(GAC_ERR_INVALID_ARG, "sigma is NULL and sigma_scalar is not a positive number");
    if (o->trace_n_vox > 0 && !out->trace)
        return fail(GAC_ERR_INVALID_ARG, "trace_n_vox > 0 needs out->trace");
    int lanes = 1;  // lanes per chain: a requested count is checked before anything runs
    if (o->lanes_per_chain > 1 && (st = choose_lanes(mc, o, n_vox, &lanes)) != GAC_OK) return st;
    if (n_vox == 0) return GAC_OK;
    if (o->lanes_per_chain == 0 && (st = choose_lanes(mc, o, n_vox, &lanes)) != GAC_OK) return st;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    keep_staging_pool();
    const int P = mc.n_par, C = o->n_chains, M = mc.n_meas;
    const int S = n_samples(o->iterations, o->burnin, o->thin);
    const size_t N = static_cast<size_t>(n_vox);

    DevBuf d_data, d_sigma, d_x0, d_mean, d_std, d_samples, d_acc, d_bad, d_trace, d_rhat, d_scale;
    if ((st = d_data.make(const_cast<void *>(data), N * M * sizeof(float), true, s, "data")) != GAC_OK) return st;
    if ((st = d_sigma.make(const_cast<float *>(sigma), sigma ? N * sizeof(float) : 0, true, s, "sigma")) != GAC_OK) return st;
    if ((st = d_x0.make(const_cast<float *>(x0), x0 ? N * C * P * sizeof(float) : 0, true, s, "x0")) != GAC_OK) return st;
    if ((st = d_mean.make(out->mean, P * N * sizeof(double), false, s, "mean")) != GAC_OK) return st;
    if ((st = d_std.make(out->std, P * N * sizeof(double), false, s, "std")) != GAC_OK) return st;
    if ((st = d_samples.make(out->samples, static_cast<size_t>(S) * C * P * N * sizeof(float), false, s, "samples")) != GAC_OK) return st;
    if ((st = d_acc.make(out->accept_rate, C * N * sizeof(float), false, s, "accept_rate")) != GAC_OK) return st;
    if ((st = d_bad.make(out->nonfinite, C * N * sizeof(int32_t), false, s, "nonfinite")) != GAC_OK) return st;
    if ((st = d_trace.make(out->trace, static_cast<size_t>(o->trace_n_vox) * C * o->iterations * sizeof(gac_trace_rec), false, s, "trace")) != GAC_OK) return st;
    if ((st = d_rhat.make(out->rhat, P * N * sizeof(double), false, s, "rhat")) != GAC_OK) return st;
    if ((st = d_scale.make(out->step_scale, C * N * sizeof(float), false, s, "step_scale")) != GAC_OK) return st;

    const bool trace = o->trace_n_vox > 0;
    LaunchCfg cfg;
    int64_t n_tiles = 0;
    int vb = 0;
    st = lanes > 1 ? plan_split(mc, lanes, C, n_vox, o->moments_mode, &cfg, &n_tiles, &vb)
                   : plan_launch(mc, o->precision, trace, C, n_vox, o->moments_mode, &cfg, &n_tiles, &vb);
    if (st != GAC_OK) return st;
    cfg.stream = s;

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
    ra.C = C;
    ra.I = o->iterations;
    ra.B = o->burnin;
    ra.T = o->thin;
    ra.S = S;
    ra.k0 = static_cast<uint32_t>(o->seed & 0xFFFFFFFFu);
    ra.k1 = static_cast<uint32_t>(o->seed >> 32);
    ra.voxel_base = o->voxel_base;
    ra.moments_mode = o->moments_mode;
    ra.trace_n = o->trace_n_vox;
    ra.vox_per_block = vb;
    ra.row_stride = row_stride_for(mc.kind, M);
    ra.data_vec4 = (M % 4 == 0) && ((reinterpret_cast<uintptr_t>(ra.data) & 15) == 0);
    ra.n_tiles = n_tiles;
    set_adaptation(ra, o);
    ra.rhat = static_cast<double *>(d_rhat.ptr);
    ra.step_scale = static_cast<float *>(d_scale.ptr);

    cudaError_t e = lanes == 1 ? launch_mh(mc.kind, o->precision, trace, mc, ra, cfg)
                    : mc.kind == GAC_MODEL_MONOEXP
                        ? launch_mh_split_monoexp(lanes, o->moments_mode == GAC_MOMENTS_ALL_POSTBURNIN, mc, ra, cfg)
                        : launch_mh_split_mwi3(lanes, o->moments_mode == GAC_MOMENTS_ALL_POSTBURNIN, mc, ra, cfg);
    if (e != cudaSuccess) return cuda_fail(e, "MH kernel launch");
    for (DevBuf *b : {&d_mean, &d_std, &d_samples, &d_acc, &d_bad, &d_trace, &d_rhat, &d_scale})
        if ((st = b->copy_out()) != GAC_OK) return st;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "MH kernel");
    return GAC_OK;
}

}  // extern "C"
