// Whole-volume gradient fit (askadam.m, Sec. 2.2.1; Eq. 2, 4, 5): Adam on
// the L1 or L2 data loss over a masked voxel grid, with an optional total-
// variation penalty on chosen parameter maps.  One launch per iteration:
//   fit_step_kernel   every voxel (one thread each): forward model and its
//                     analytic Jacobian, the data loss and its gradient, the
//                     total-variation subgradient from the six (or four)
//                     neighbours' current parameters, and the Adam update
//                     into the other parameter buffer; each block writes its
//                     share of the loss, and the last block to finish sums
//                     the shares in a fixed order, records the iteration's
//                     loss and applies the stopping rules; once it sets the
//                     stop flag, later launches return at once.
// Parameters are optimised in normalised form u = (theta - lb) / (ub - lb),
// clamped to [0, 1] after each update, stored [P][N] (structure of arrays).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "gac.h"
#include "gac_internal.h"
#include "mh_kernel.cuh"

namespace gac {

constexpr int kFitBlock = 128;
constexpr int kFitMinBlocks32 = 5;  // FP32: 20 warps an SM (registers <= 102)
constexpr int kFitMaxWindow = 4096;

template <class R>
struct FitArgs {
    const float *data;     // [N][M]
    const uint8_t *mask;   // [N] or nullptr
    const float *weight;   // [N] or nullptr
    int nx, ny, nz;
    int64_t n;
    uint32_t tv_params;
    int tv_dims;
    R scale;               // 1 / (n_mask M)
    R lambda_n;            // lambda / n_mask
    R lr, beta1, beta2, eps;
    int row_stride;        // shared-memory floats per staged measurement row (4 x odd, >= M)
    int vec4;              // rows staged and read as float4 (M % 4 == 0, 16-byte aligned data)
    float inv_m4;          // 1 / (M / 4): row of a tile's float4 number e, exact for e < 2^13
    int fdiv;              // n < 2^24: grid coordinates by float reciprocals (udiv_f)
    float inv_nx, inv_ny;  // 1 / nx, 1 / ny rounded to float
    int *stop;             // set by the last block of the iteration that stops
    int *done;             // updates taken
    unsigned *arrive;      // blocks of the current launch that have finished (reset by the last)
    double *hist;          // [iterations] loss history
    double tol, conv_value;
    int window;
    double *block_loss;    // [gridDim.x]
};

// sign(x) with sign(0) = 0, branch-free (a select and a sign-bit copy)
template <class R>
__device__ __forceinline__ R sgn(R x) {
    return x != R(0) ? copysign(R(1), x) : R(0);
}

// a / b and a % b for a < 2^24 from the float reciprocal inv_b = fl(1 / b):
// the float quotient is within 1 of a / b for b >= 2 (two roundings of
// relative size 2^-24 on a value below 2^23) and exact for b = 1, so one
// correction step gives the integer quotient.
__device__ __forceinline__ unsigned udiv_f(unsigned a, unsigned b, float inv_b, unsigned &rem) {
    unsigned q = __float2uint_rz(__uint2float_rn(a) * inv_b);
    int r = static_cast<int>(a - q * b);
    if (r < 0) {
        --q;
        r += static_cast<int>(b);
    } else if (r >= static_cast<int>(b)) {
        ++q;
        r -= static_cast<int>(b);
    }
    rem = static_cast<unsigned>(r);
    return q;
}

// ------------------------------------------------ models and Jacobians ----
// visit(k, s_k, J_k[P]) per real measurement (complex data: re then im).
template <int KIND, class R, class V>
__device__ __forceinline__ void jacobian(const R *th, const ModelConst &mc, V &&visit) {
    constexpr int P = model_n_par(KIND);
    const int n = mc.n_acq;
    if constexpr (KIND == GAC_MODEL_MONOEXP) {
        for (int k = 0; k < n; ++k) {
            const R t = sizeof(R) == 8 ? R(mc.acq_d[k]) : R(mc.acq_f[k]);
            const R e = exp(-th[1] * t * R(1e-3));
            R J[P] = {e, -th[0] * t * R(1e-3) * e};
            visit(k, th[0] * e, J);
        }
    } else if constexpr (KIND == GAC_MODEL_MWI3) {
        for (int k = 0; k < n; ++k) {
            const R t = sizeof(R) == 8 ? R(mc.acq_d[k]) : R(mc.acq_f[k]);
            R Jr[P], Ji[P];
            R re = R(0), im = R(0);
            const R w2pi = R(6.283185307179586477) * t * R(1e-3);  // d angle / d df
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const R decay = exp(-t / th[3 + j]);
                const R ang = th[8] - ((j < 2) ? th[6 + j] * w2pi : R(0));
                R sn, cs;
                sincos(ang, &sn, &cs);
                const R amp = th[j] * decay;
                re += amp * cs;
                im += amp * sn;
                Jr[j] = decay * cs;
                Ji[j] = decay * sn;
                const R dT = amp * t / (th[3 + j] * th[3 + j]);
                Jr[3 + j] = dT * cs;
                Ji[3 + j] = dT * sn;
                if (j < 2) {
                    Jr[6 + j] = amp * w2pi * sn;
                    Ji[6 + j] = -amp * w2pi * cs;
                }
            }
            Jr[8] = -im;
            Ji[8] = re;
            visit(2 * k, re, Jr);
            visit(2 * k + 1, im, Ji);
        }
    } else if constexpr (KIND == GAC_MODEL_SMT) {
        const R f = th[0], da = th[1], dpar = th[2], dperp = th[3];
        for (int k = 0; k < n; ++k) {
            const R b = sizeof(R) == 8 ? R(mc.acq_d[k]) : R(mc.acq_f[k]);
            R gi, dgi, gx, dgx;
            smt_g_dg(b * da, mc, gi, dgi);
            smt_g_dg(b * (dpar - dperp), mc, gx, dgx);
            const R e = exp(-b * dperp);
            R J[P] = {gi - e * gx, f * b * dgi, (R(1) - f) * e * b * dgx, (R(1) - f) * (-b * e * gx - e * b * dgx)};
            visit(k, f * gi + (R(1) - f) * e * gx, J);
        }
    } else {  // linear test model
        for (int k = 0; k < n; ++k) {
            const R t = sizeof(R) == 8 ? R(mc.acq_d[k]) : R(mc.acq_f[k]);
            R J[P] = {R(1), t};
            visit(k, th[0] + th[1] * t, J);
        }
    }
}

// The 3-pool model's data loss and its gradient in FP32 for evenly spaced
// echoes, from the anchored recurrence of the unit-amplitude pool terms
// u_j(t) = e^{-t/T2*_j} e^{i(phi0 - w_j t)} (the MH kernel's recurrence with
// A_j = 1).  Every entry of the Jacobian is a product,
//   dS/dA_j = u_j,  dS/dT2*_j = A_j t / T2*_j^2 u_j,
//   dS/d df_j = -i 2 pi 1e-3 t A_j u_j,  dS/d phi0 = i S,
// so with d = (d_re, d_im) the loss derivative with respect to (Re S, Im S) at
// an echo, the gradient sums factor into per-pool sums of Re(conj(d) u_j)
// (the amplitudes), of t times them (T2*, scaled by A_j / T2*_j^2 at the end)
// and of t Im(conj(d) u_j) (the frequencies, scaled by A_j 2 pi 1e-3); the
// two offset pools are carried as lane pairs.  rho and its derivative as in
// the visitor of fit_voxel: r = w (y - s), L1 |r| with d = -w sign(r), L2
// r^2 with d = -2 w r (the weight factored out of the sums).  Adds the
// gradient to g[9]; returns the data loss.
template <bool L1>
__device__ __forceinline__ float mwi3_rec_loss_grad_f(const float *th, const ModelConst &mc, const float *yrow,
                                                      float wgt, float *g) {
    const float phi0 = th[8];
    const int n = mc.n_acq;
    // 1 / T2* from the special-function reciprocal and one Newton step (within an ulp)
    auto rcp = [](float x) {
        const float r = rcp_approx(x);
        return fmaf(fmaf(-x, r, 1.0f), r, r);
    };
    const float r0 = rcp(th[3]), r1 = rcp(th[4]), r2 = rcp(th[5]);
    const float2 w = make_float2(kTwoPiMilli * th[6], kTwoPiMilli * th[7]);
    const float2 m0 = make_float2(expf(-mc.t0_f * r0), expf(-mc.t0_f * r1));
    const float2 m1 = make_float2(expf(-mc.dt_f * r0), expf(-mc.dt_f * r1));
    const float2 mk = make_float2(expf(-mc.dtk_f * r0), expf(-mc.dtk_f * r1));
    float2 sn, cs;
    sincos_cw2(__ffma2_rn(make_float2(-w.x, -w.y), f2(mc.t0_f), f2(phi0)), sn, cs);
    float2 X = __fmul2_rn(m0, cs), Y = __fmul2_rn(m0, sn);
    sincos_cw2(__fmul2_rn(make_float2(-w.x, -w.y), f2(mc.dt_f)), sn, cs);
    const float2 RR = __fmul2_rn(m1, cs), RI = __fmul2_rn(m1, sn), NRI = make_float2(-RI.x, -RI.y);
    sincos_cw2(__fmul2_rn(make_float2(-w.x, -w.y), f2(mc.dtk_f)), sn, cs);
    const float2 KR = __fmul2_rn(mk, cs), KI = __fmul2_rn(mk, sn), NKI = make_float2(-KI.x, -KI.y);
    float se, ce;
    sincos_cw(phi0, se, ce);
    const float e2 = expf(-mc.t0_f * r2);
    float2 Z = make_float2(e2 * ce, e2 * se);
    const float2 R2 = f2(expf(-mc.dt_f * r2)), K2 = f2(expf(-mc.dtk_f * r2));
    const float a0 = th[0], a1 = th[1], a2 = th[2];
    // sums over echoes: amplitude terms, t x amplitude terms, t x frequency terms
    float2 G01 = f2(0.0f), T01 = f2(0.0f), C01 = f2(0.0f);
    float G2 = 0.0f, T2 = 0.0f, G8 = 0.0f, loss = 0.0f;
    // rho'(r) w.r.t. s for r = w e, e = y - s: L1 -w sign(w e) = -|w| sign(e)
    // (sign(0) = 0), L2 -2 w r = -2 w^2 e; the loss sums |e| or e^2 and takes
    // the weight's |w| or w^2 once at the end
    const float aw = fabsf(wgt), k2 = -2.0f * wgt * wgt;
    auto deriv = [&](float e) {
        if constexpr (L1) return e != 0.0f ? copysignf(aw, -e) : 0.0f;
        else return k2 * e;
    };
    auto echo = [&](float t, float yr, float yi, float2 x, float2 y, float2 z) {
        const float re = fmaf(a0, x.x, fmaf(a1, x.y, a2 * z.x));
        const float im = fmaf(a0, y.x, fmaf(a1, y.y, a2 * z.y));
        const float er = yr - re, ei = yi - im;
        const float dr = deriv(er), di = deriv(ei);
        if constexpr (L1) loss += fabsf(er) + fabsf(ei);
        else loss = fmaf(er, er, fmaf(ei, ei, loss));
        const float2 D = f2(dr), E = f2(di);
        const float2 inc = __ffma2_rn(E, y, __fmul2_rn(D, x));                       // Re(conj(d) u), pools 0, 1
        const float2 crs = __ffma2_rn(make_float2(-di, -di), x, __fmul2_rn(D, y));  // Im(conj(d) u)
        const float2 tt = f2(t);
        G01 = __fadd2_rn(G01, inc);
        T01 = __ffma2_rn(tt, inc, T01);
        C01 = __ffma2_rn(tt, crs, C01);
        const float inc2 = fmaf(di, z.y, dr * z.x);
        G2 += inc2;
        T2 = fmaf(t, inc2, T2);
        G8 = fmaf(di, re, fmaf(-dr, im, G8));
    };
    // echoes a + i, a + i + 1 (a even) come in one 16-byte load: rows are
    // staged at a multiple of four floats, padded past an odd echo count
    const float4 *q4 = reinterpret_cast<const float4 *>(yrow);
    auto step = [&](float2 &x, float2 &y, float2 &z) {
        const float2 xn = __ffma2_rn(x, RR, __fmul2_rn(y, NRI));
        y = __ffma2_rn(x, RI, __fmul2_rn(y, RR));
        x = xn;
        z = __fmul2_rn(z, R2);
    };
    int a = 0;
    for (; a + kAnchor <= n; a += kAnchor) {  // full blocks: offsets and times fixed
        float2 x = X, y = Y, z = Z;
        const float ta = fmaf(static_cast<float>(a), mc.dt_f, mc.t0_f);
#pragma unroll
        for (int i = 0; i < kAnchor; i += 2) {
            const float4 q = q4[(a + i) >> 1];
            echo(fmaf(static_cast<float>(i), mc.dt_f, ta), q.x, q.y, x, y, z);
            step(x, y, z);
            echo(fmaf(static_cast<float>(i + 1), mc.dt_f, ta), q.z, q.w, x, y, z);
            step(x, y, z);
        }
        const float2 xn = __ffma2_rn(X, KR, __fmul2_rn(Y, NKI));
        Y = __ffma2_rn(X, KI, __fmul2_rn(Y, KR));
        X = xn;
        Z = __fmul2_rn(Z, K2);
    }
    // the last, partial block (not unrolled: it runs once)
    float2 x = X, y = Y, z = Z;
#pragma unroll 1
    for (int k = a; k < n; ++k) {
        const float4 q = q4[k >> 1];
        echo(fmaf(static_cast<float>(k), mc.dt_f, mc.t0_f), (k & 1) ? q.z : q.x, (k & 1) ? q.w : q.y, x, y, z);
        step(x, y, z);
    }
    g[0] += G01.x;
    g[1] += G01.y;
    g[2] += G2;
    g[3] += a0 * r0 * r0 * T01.x;
    g[4] += a1 * r1 * r1 * T01.y;
    g[5] += a2 * r2 * r2 * T2;
    g[6] += a0 * kTwoPiMilli * C01.x;
    g[7] += a1 * kTwoPiMilli * C01.y;
    g[8] += G8;
    return L1 ? aw * loss : wgt * wgt * loss;
}

// One voxel's update: forward model and Jacobian against its staged data row
// y, the loss gradient, the total-variation subgradient, Adam and the box.
// Returns the voxel's share of the loss (0 outside the mask).
// One voxel's update in two phases around the warp's staging points (the
// kernel below): phase A issues the loads of the total-variation neighbours
// and evaluates the model and its Jacobian against the staged data row y
// (loss and gradient into loss, g); phase B adds the total-variation
// subgradient and takes the Adam step and the box, with the voxel's Adam
// moments from shared memory (mo: m1 at [p * 32], m2 at [(P + p) * 32]).
template <int KIND, class R>
struct FitTv {
    unsigned grid_bit = 0, nbit = 0;  // neighbours inside the grid; inside the grid and the mask
    int p0 = model_n_par(KIND);       // first penalised map (P: none)
    R nb0[6];                         // its neighbours' values
    uint8_t nmask[6];                 // the neighbours' mask bytes
};

template <int KIND, class R>
__device__ __forceinline__ int fit_offset(const FitTv<KIND, R> &tv, int j, const int (&step)[3]) {
    return ((tv.grid_bit >> j) & 1u) ? ((j & 1) ? -step[j >> 1] : step[j >> 1]) : 0;
}

// Phase A.  The neighbours' mask bytes and values load first and are used in
// phase B, so nothing waits on them before the model.
template <int KIND, int PREC, bool L1>
__device__ __forceinline__ void fit_phase_a(const ModelConst &mc, const FitArgs<typename PrecTraits<PREC>::R> &fa, int v,
                                            const float *y, const typename PrecTraits<PREC>::R (&u)[model_n_par(KIND)],
                                            bool inside, typename PrecTraits<PREC>::R w,
                                            const typename PrecTraits<PREC>::R *u_in, FitTv<KIND, typename PrecTraits<PREC>::R> &tv,
                                            typename PrecTraits<PREC>::R &loss, typename PrecTraits<PREC>::R (&g)[model_n_par(KIND)]) {
    using R = typename PrecTraits<PREC>::R;
    constexpr int P = model_n_par(KIND);
    const int n = static_cast<int>(fa.n);
    const int step[3] = {1, fa.nx, fa.nx * fa.ny};
    if (fa.tv_params && fa.lambda_n != R(0)) {
        const unsigned vu = static_cast<unsigned>(v), nxu = static_cast<unsigned>(fa.nx), nyu = static_cast<unsigned>(fa.ny);
        unsigned cx, cy, q, cz;
        if (fa.fdiv) {  // the same for every thread
            q = udiv_f(vu, nxu, fa.inv_nx, cx);
            cz = udiv_f(q, nyu, fa.inv_ny, cy);
        } else {
            q = vu / nxu;
            cx = vu - q * nxu;
            cz = q / nyu;
            cy = q - cz * nyu;
        }
        const int coord[3] = {static_cast<int>(cx), static_cast<int>(cy), static_cast<int>(cz)};
        const int ext[3] = {fa.nx, fa.ny, fa.nz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const bool use = d < fa.tv_dims;
            tv.grid_bit |= static_cast<unsigned>(use && coord[d] + 1 < ext[d]) << (2 * d) |
                           static_cast<unsigned>(use && coord[d] > 0) << (2 * d + 1);
        }
        tv.nbit = tv.grid_bit;
        if (fa.mask) {
#pragma unroll
            for (int j = 0; j < 6; ++j) tv.nmask[j] = fa.mask[v + fit_offset(tv, j, step)];
        }
        tv.p0 = __ffs(fa.tv_params) - 1;
        if (tv.p0 < P) {
#pragma unroll
            for (int j = 0; j < 6; ++j) tv.nb0[j] = u_in[tv.p0 * n + v + fit_offset(tv, j, step)];
        }
    }
    loss = R(0);
#pragma unroll
    for (int p = 0; p < P; ++p) g[p] = R(0);
    if (!inside) return;
    R th[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const R lo = sizeof(R) == 8 ? R(mc.lb_d[p]) : R(mc.lb_f[p]);
        const R hi = sizeof(R) == 8 ? R(mc.ub_d[p]) : R(mc.ub_f[p]);
        th[p] = lo + u[p] * (hi - lo);
    }
    // data term: rho(w (y - s)), drho/ds = -w sign(r) (L1) or -2 w r (L2)
    auto visit = [&](int k, R s, const R *J) {
        const R r = w * (R(y[k]) - s);
        R d;
        if constexpr (L1) {
            d = -w * sgn(r);
            loss += fabs(r);
        } else {
            d = R(-2) * w * r;
            loss += r * r;
        }
#pragma unroll
        for (int p = 0; p < P; ++p) g[p] = fma(d, J[p], g[p]);
    };
    if constexpr (KIND == GAC_MODEL_MWI3 && PREC == GAC_PREC_FP32) {
        if (mc.even) loss = mwi3_rec_loss_grad_f<L1>(th, mc, y, w, g);  // same branch for every thread
        else jacobian<KIND, R>(th, mc, visit);
    } else {
        jacobian<KIND, R>(th, mc, visit);
    }
}

// Phase B; returns the voxel's share of the loss (0 outside the mask).
template <int KIND, int PREC>
__device__ __forceinline__ typename PrecTraits<PREC>::R fit_phase_b(
    const ModelConst &mc, const FitArgs<typename PrecTraits<PREC>::R> &fa, int v,
    const typename PrecTraits<PREC>::R (&u)[model_n_par(KIND)], bool inside, const FitTv<KIND, typename PrecTraits<PREC>::R> &tv_in,
    typename PrecTraits<PREC>::R loss, typename PrecTraits<PREC>::R (&g)[model_n_par(KIND)],
    const typename PrecTraits<PREC>::R *mo, const typename PrecTraits<PREC>::R *u_in, typename PrecTraits<PREC>::R *u_out,
    typename PrecTraits<PREC>::R *m1, typename PrecTraits<PREC>::R *m2, typename PrecTraits<PREC>::R c1,
    typename PrecTraits<PREC>::R c2) {
    using R = typename PrecTraits<PREC>::R;
    constexpr int P = model_n_par(KIND);
    const int n = static_cast<int>(fa.n);
    if (!inside) {
#pragma unroll
        for (int p = 0; p < P; ++p) u_out[p * n + v] = u[p];
        return R(0);
    }
    R vl = loss * fa.scale;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const R range = sizeof(R) == 8 ? R(mc.ub_d[p] - mc.lb_d[p]) : R(mc.ub_f[p] - mc.lb_f[p]);
        g[p] *= fa.scale * range;
    }
    // total variation: pairs (v - e_d, v) and (v, v + e_d) of masked neighbours
    if (fa.tv_params && fa.lambda_n != R(0)) {
        const int step[3] = {1, fa.nx, fa.nx * fa.ny};
        unsigned nbit = tv_in.nbit;
        if (fa.mask) {
#pragma unroll
            for (int j = 0; j < 6; ++j) nbit &= ~(static_cast<unsigned>(tv_in.nmask[j] == 0) << j);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (!((fa.tv_params >> p) & 1u)) continue;
            R nb[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) nb[j] = p == tv_in.p0 ? tv_in.nb0[j] : u_in[p * n + v + fit_offset(tv_in, j, step)];
            R tv = R(0), tv_loss = R(0);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if ((nbit >> (2 * d)) & 1u) {
                    const R diff = nb[2 * d] - u[p];
                    tv -= sgn(diff);
                    tv_loss += fabs(diff);
                }
                if ((nbit >> (2 * d + 1)) & 1u) tv += sgn(u[p] - nb[2 * d + 1]);
            }
            g[p] = fma(fa.lambda_n, tv, g[p]);
            vl += fa.lambda_n * tv_loss;
        }
    }
    // Adam (bias-corrected moments), then the box.  FP32: the corrections as
    // the reciprocals c1, c2 carry (1 / (1 - beta^t)), the step's square root
    // and quotient on the special-function unit (a few ulp); FP64: divided,
    // as the oracle does
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const R a = fa.beta1 * mo[p * 32] + (R(1) - fa.beta1) * g[p];
        const R b = fa.beta2 * mo[(P + p) * 32] + (R(1) - fa.beta2) * g[p] * g[p];
        m1[p * n + v] = a;
        m2[p * n + v] = b;
        R stepu;
        if constexpr (sizeof(R) == 8) {
            stepu = fa.lr * (a / c1) / (sqrt(b / c2) + fa.eps);
        } else {
            float sq;
            asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq) : "f"(b * c2));
            stepu = __fdividef(fa.lr * (a * c1), sq + fa.eps);
        }
        u_out[p * n + v] = fmin(fmax(u[p] - stepu, R(0)), R(1));
    }
    return vl;
}

// 4-byte asynchronous global -> shared copies (no register round trip), in
// commit groups; wait<N> returns when at most N groups are still in flight.
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
template <class T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Persistent warps over tiles of 32 voxels (warp tile w, w + all warps, ...).
// Each warp stages its own tile's measurement rows and Adam moments in its
// own part of shared memory (fit_warp_smem) with cp.async copies, and only
// the warp waits for them, so warps drift apart and hide each other's memory
// latency instead of meeting at a block barrier.  The copies are placed where
// their buffers fall free: the next tile's rows as soon as the model has read
// the current ones (before phase B), the next tile's moments after phase B;
// each lane's next parameters, mask flag and weight load into registers
// during phase B.  So neither the moments nor the next parameters occupy
// registers during the model, and more warps fit on an SM.  Rows sit at an
// odd number of float4s, so that a warp's 16-byte reads of one echo pair hit
// distinct banks.
constexpr int kFitWarps = kFitBlock / 32;
constexpr int fit_min_blocks(int prec) { return prec == GAC_PREC_FP32 ? kFitMinBlocks32 : 1; }

// Shared memory of one warp: 32 staged rows, then the tile's moments
// [2][P][32] (m1, m2).
__host__ __device__ constexpr size_t fit_warp_smem(int row_stride, int P, size_t rbytes) {
    return 32 * static_cast<size_t>(row_stride) * sizeof(float) + 2 * static_cast<size_t>(P) * 32 * rbytes;
}

template <int KIND, int PREC, bool L1>
__global__ void __launch_bounds__(kFitBlock, fit_min_blocks(PREC)) fit_step_kernel(const ModelConst mc, const FitArgs<typename PrecTraits<PREC>::R> fa,
                                                             const typename PrecTraits<PREC>::R *u_in,
                                                             typename PrecTraits<PREC>::R *u_out,
                                                             typename PrecTraits<PREC>::R *m1,
                                                             typename PrecTraits<PREC>::R *m2,
                                                             typename PrecTraits<PREC>::R c1,
                                                             typename PrecTraits<PREC>::R c2, int t_iter) {
    using R = typename PrecTraits<PREC>::R;
    constexpr int P = model_n_par(KIND);
    __shared__ double red[kFitBlock];
    __shared__ bool last;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // launched as a programmatic dependent of the previous update: its blocks
    // become resident while that launch drains, and wait here until it has
    // completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (*fa.stop) return;  // the same for every thread
    model_smem_load<KIND>(mc);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int M = mc.n_meas;
    const int n = static_cast<int>(fa.n);
    const int n_tiles = (n + 31) / 32;
    unsigned char *wmem = smem_raw + warp * fit_warp_smem(fa.row_stride, P, sizeof(R));
    float *rows_s = reinterpret_cast<float *>(wmem);
    R *mo_s = reinterpret_cast<R *>(wmem + 32 * static_cast<size_t>(fa.row_stride) * sizeof(float));
    auto stage_rows = [&](int tile) {
        const int base = tile * 32;
        const int rows = min(32, n - base);
        const float *src = fa.data + static_cast<int64_t>(base) * M;
        if (fa.vec4) {  // 16-byte copies; row = floor((e + 1/2) / (M/4)) by one float multiply
            const int M4 = M >> 2, S4 = fa.row_stride >> 2, total4 = rows * M4;
#pragma unroll 4
            for (int e = lane; e < total4; e += 32) {
                const int row = static_cast<int>((static_cast<float>(e) + 0.5f) * fa.inv_m4);
                cp_async16(rows_s + 4 * (row * S4 + (e - row * M4)), src + 4 * e);
            }
        } else {
            const int total = rows * M;
            for (int e = lane; e < total; e += 32) {
                const int row = e / M;
                cp_async4(rows_s + row * fa.row_stride + (e - row * M), src + e);
            }
        }
    };
    auto stage_moments = [&](int tile) {
        const int e = tile * 32 + lane;
        if (e < n) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                cp_async_elem(mo_s + p * 32 + lane, m1 + p * n + e);
                cp_async_elem(mo_s + (P + p) * 32 + lane, m2 + p * n + e);
            }
        }
    };
    // the lane's next voxel: parameters, mask flag and weight
    R un[P];
    bool in_n = true;
    R w_n = R(1);
    auto load_next = [&](int vv) {
        if (vv < n) {
#pragma unroll
            for (int p = 0; p < P; ++p) un[p] = u_in[p * n + vv];
            in_n = !fa.mask || fa.mask[vv];
            w_n = fa.weight ? R(fa.weight[vv]) : R(1);
        }
    };
    R my_loss = R(0);
    const int stride = gridDim.x * kFitWarps;
    int tile = blockIdx.x * kFitWarps + warp;
    if (tile < n_tiles) {
        stage_rows(tile);
        stage_moments(tile);
    }
    cp_async_commit();
    load_next(tile * 32 + lane);
    for (; tile < n_tiles; tile += stride) {
        cp_async_wait<0>();
        __syncwarp();
        const int v = tile * 32 + lane;
        const bool active = v < n;
        R u[P];
#pragma unroll
        for (int p = 0; p < P; ++p) u[p] = un[p];
        const bool inside = active && in_n;
        const R w = w_n;
        FitTv<KIND, R> tv;
        R loss, g[P];
        if (active) fit_phase_a<KIND, PREC, L1>(mc, fa, v, rows_s + lane * fa.row_stride, u, inside, w, u_in, tv, loss, g);
        __syncwarp();  // the model has read every row: the buffer takes the next tile's
        const int next = tile + stride;
        if (next < n_tiles) stage_rows(next);
        cp_async_commit();
        load_next(next * 32 + lane);
        if (active) my_loss += fit_phase_b<KIND, PREC>(mc, fa, v, u, inside, tv, loss, g, mo_s + lane, u_in, u_out, m1, m2, c1, c2);
        __syncwarp();  // phase B has read every moment
        if (next < n_tiles) stage_moments(next);
        cp_async_commit();
    }
    cp_async_wait<0>();
    // the block's share of the loss, summed in a fixed order: lanes by
    // shuffles within each warp, then the warps
    double sum = static_cast<double>(my_loss);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if (lane == 0) red[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < kFitWarps; ++i) t += red[i];
        fa.block_loss[blockIdx.x] = t;
        __threadfence();  // the share is visible before the count says so
        last = atomicAdd(fa.arrive, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {  // every other block's share has landed
        __threadfence();
        fit_check(fa, gridDim.x, t_iter, red);
        if (threadIdx.x == 0) *fa.arrive = 0u;  // for the next launch, which starts after this one ends
    }
}

// Run by the last block of iteration t: sums the block shares (fixed order:
// thread i the shares i, i + 256, ..., then a tree), records loss t and
// applies the stopping rules: loss < tol, or |least-squares slope of the
// last `window` losses| < conv_value.
template <class FA>
__device__ void fit_check(const FA &fa, int n_blocks, int t, double *red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) s += __ldcg(fa.block_loss + i);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = kFitBlock / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double loss = red[0];
    fa.hist[t - 1] = loss;
    *fa.done = t;
    bool halt = fa.tol > 0.0 && loss < fa.tol;
    const int window = fa.window;
    if (!halt && fa.conv_value > 0.0 && window > 1 && t >= window) {
        const double *yv = fa.hist + t - window;
        const double xm = 0.5 * (window - 1);
        double ym = 0.0, sxy = 0.0, sxx = 0.0;
        for (int i = 0; i < window; ++i) ym += yv[i];
        ym /= window;
        for (int i = 0; i < window; ++i) {
            sxy += (i - xm) * (yv[i] - ym);
            sxx += (i - xm) * (i - xm);
        }
        halt = fabs(sxy / sxx) < fa.conv_value;
    }
    if (halt) *fa.stop = 1;
}

// The number of non-zero mask bytes (one atomic add per block).
__global__ void count_mask_kernel(const uint8_t *mask, int64_t n, unsigned long long *count) {
    __shared__ unsigned part[8];
    unsigned c = 0;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        c += mask[i] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(count, t);
    }
}

// theta [N][P] (double) <-> u [P][N]; outside the mask theta is left alone.
template <class R>
__global__ void theta_to_u_kernel(const ModelConst mc, const double *theta, int64_t n, R *u) {
    const int P = mc.n_par;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n * P;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t v = i / P;
        const int p = static_cast<int>(i - v * P);
        const double range = mc.ub_d[p] - mc.lb_d[p];
        const double x = range > 0 ? (theta[i] - mc.lb_d[p]) / range : 0.0;
        u[p * n + v] = static_cast<R>(fmin(fmax(x, 0.0), 1.0));
    }
}
template <class R>
__global__ void u_to_theta_kernel(const ModelConst mc, const R *u, const uint8_t *mask, int64_t n, double *theta) {
    const int P = mc.n_par;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n * P;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t v = i / P;
        const int p = static_cast<int>(i - v * P);
        if (mask && !mask[v]) continue;
        theta[i] = mc.lb_d[p] + static_cast<double>(u[p * n + v]) * (mc.ub_d[p] - mc.lb_d[p]);
    }
}

template <int PREC, bool L1>
static const void *step_ptr(int kind) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: return reinterpret_cast<const void *>(&fit_step_kernel<GAC_MODEL_MONOEXP, PREC, L1>);
    case GAC_MODEL_MWI3: return reinterpret_cast<const void *>(&fit_step_kernel<GAC_MODEL_MWI3, PREC, L1>);
    case GAC_MODEL_SMT: return reinterpret_cast<const void *>(&fit_step_kernel<GAC_MODEL_SMT, PREC, L1>);
    default: return reinterpret_cast<const void *>(&fit_step_kernel<GAC_MODEL_LINEAR_TEST, PREC, L1>);
    }
}

template <int KIND, int PREC>
static cudaError_t launch_step(bool l1, int grid, size_t smem, cudaStream_t s, const ModelConst &mc,
                               const FitArgs<typename PrecTraits<PREC>::R> &fa, const void *u_in, void *u_out,
                               void *m1, void *m2, double c1, double c2, int t) {
    using R = typename PrecTraits<PREC>::R;
    auto *ui = static_cast<const R *>(u_in);
    auto *uo = static_cast<R *>(u_out);
    // programmatic stream serialization: the launch may begin while the
    // previous kernel in the stream drains (the kernel waits for it first)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kFitBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto *m1r = static_cast<R *>(m1);
    auto *m2r = static_cast<R *>(m2);
    if (l1) return cudaLaunchKernelEx(&cfg, fit_step_kernel<KIND, PREC, true>, mc, fa, ui, uo, m1r, m2r, R(c1), R(c2), t);
    return cudaLaunchKernelEx(&cfg, fit_step_kernel<KIND, PREC, false>, mc, fa, ui, uo, m1r, m2r, R(c1), R(c2), t);
}

template <int PREC>
static cudaError_t launch_step_kind(int kind, bool l1, int grid, size_t smem, cudaStream_t s, const ModelConst &mc,
                                    const FitArgs<typename PrecTraits<PREC>::R> &fa, const void *u_in, void *u_out,
                                    void *m1, void *m2, double c1, double c2, int t) {
    switch (kind) {
    case GAC_MODEL_MONOEXP: return launch_step<GAC_MODEL_MONOEXP, PREC>(l1, grid, smem, s, mc, fa, u_in, u_out, m1, m2, c1, c2, t);
    case GAC_MODEL_MWI3: return launch_step<GAC_MODEL_MWI3, PREC>(l1, grid, smem, s, mc, fa, u_in, u_out, m1, m2, c1, c2, t);
    case GAC_MODEL_SMT: return launch_step<GAC_MODEL_SMT, PREC>(l1, grid, smem, s, mc, fa, u_in, u_out, m1, m2, c1, c2, t);
    default: return launch_step<GAC_MODEL_LINEAR_TEST, PREC>(l1, grid, smem, s, mc, fa, u_in, u_out, m1, m2, c1, c2, t);
    }
}

template <int PREC>
static gac_status fit_run_prec(const ModelConst &mc, const gac_fit_opts *o, const float *d_data, const uint8_t *d_mask,
                               const float *d_weight, int64_t n_mask, double *theta, double *loss_history,
                               int *iterations_done, cudaStream_t s) {
    using R = typename PrecTraits<PREC>::R;
    const int P = mc.n_par;
    const int64_t N = static_cast<int64_t>(o->nx) * o->ny * o->nz;
    const size_t RB = sizeof(R);
    DevBuf d_theta;
    gac_status st = d_theta.make(theta, static_cast<size_t>(N) * P * sizeof(double), true, s, "theta");
    if (st != GAC_OK) return st;
    int sms = 0, dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // rows at an odd number of float4s (padded up), so that a warp's 16-byte
    // reads of one column fall into distinct banks; staged by 16-byte copies
    // when rows are whole float4s and the data is aligned, else by 4-byte ones
    const bool vec4 = mc.n_meas % 4 == 0 && (reinterpret_cast<uintptr_t>(d_data) & 15) == 0;
    const int row_stride = 4 * (((mc.n_meas + 3) / 4) | 1);
    const size_t smem = kFitWarps * fit_warp_smem(row_stride, P, sizeof(R));
    if (smem > static_cast<size_t>(smem_max))
        return fail(GAC_ERR_INVALID_ARG, "fit: %d measurements per voxel need %zu bytes of staging, more than the %d a block has",
                    mc.n_meas, smem, smem_max);
    const bool l1 = o->loss == GAC_FIT_L1;
    const void *fn = l1 ? step_ptr<PREC, true>(mc.kind) : step_ptr<PREC, false>(mc.kind);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFitBlock, smem);
    if (e != cudaSuccess) return cuda_fail(e, "fit kernel attributes");
    // persistent warps, each given the same number of 32-voxel tiles (+-1)
    const int64_t tiles = (N + 31) / 32;
    const int64_t slots = static_cast<int64_t>(sms) * std::max(per_sm, 1) * kFitWarps;
    const int64_t per_warp = (tiles + slots - 1) / slots;
    const int grid = static_cast<int>((tiles + per_warp * kFitWarps - 1) / (per_warp * kFitWarps));
    // work arrays: u (two buffers), Adam moments, block losses, history, flags
    const int I = o->iterations;
    const size_t bytes_u = static_cast<size_t>(N) * P * RB;
    const size_t total = 4 * bytes_u + grid * sizeof(double) + static_cast<size_t>(std::max(I, 1)) * sizeof(double) + 3 * sizeof(int);
    void *base = nullptr;
    e = cudaMallocAsync(&base, total, s);
    if (e != cudaSuccess) return cuda_fail(e, "fit work arrays");
    struct Free {
        void *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } guard{base, s};
    char *b = static_cast<char *>(base);
    void *u0 = b, *u1 = b + bytes_u, *m1 = b + 2 * bytes_u, *m2 = b + 3 * bytes_u;
    double *block_loss = reinterpret_cast<double *>(b + 4 * bytes_u);
    double *hist = block_loss + grid;
    int *flags = reinterpret_cast<int *>(hist + std::max(I, 1));  // stop, done, arrival count
    if ((e = cudaMemsetAsync(m1, 0, 2 * bytes_u, s)) != cudaSuccess) return cuda_fail(e, "fit memset");
    if ((e = cudaMemsetAsync(flags, 0, 3 * sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "fit memset");
    const int conv_grid = static_cast<int>(std::min<int64_t>((N * P + 255) / 256, static_cast<int64_t>(sms) * 8));
    theta_to_u_kernel<R><<<conv_grid, 256, 0, s>>>(mc, static_cast<const double *>(d_theta.ptr), N, static_cast<R *>(u0));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "theta to u");
    FitArgs<R> fa;
    std::memset(&fa, 0, sizeof fa);
    fa.data = d_data;
    fa.mask = d_mask;
    fa.weight = d_weight;
    fa.nx = o->nx;
    fa.ny = o->ny;
    fa.nz = o->nz;
    fa.n = N;
    fa.tv_params = o->tv_params;
    fa.tv_dims = o->tv_dims;
    fa.scale = static_cast<R>(1.0 / (static_cast<double>(n_mask) * mc.n_meas));
    fa.lambda_n = static_cast<R>(o->tv_lambda / static_cast<double>(n_mask));
    fa.lr = static_cast<R>(o->learning_rate);
    fa.beta1 = static_cast<R>(o->beta1);
    fa.beta2 = static_cast<R>(o->beta2);
    fa.eps = static_cast<R>(o->epsilon);
    fa.stop = flags;
    fa.done = flags + 1;
    fa.arrive = reinterpret_cast<unsigned *>(flags + 2);
    fa.hist = hist;
    fa.tol = o->tol;
    fa.conv_value = o->convergence_value;
    fa.window = o->convergence_window;
    fa.block_loss = block_loss;
    fa.row_stride = row_stride;
    fa.vec4 = vec4;
    fa.inv_m4 = vec4 ? 1.0f / static_cast<float>(mc.n_meas / 4) : 0.0f;
    fa.fdiv = N < (int64_t(1) << 24);
    fa.inv_nx = 1.0f / static_cast<float>(o->nx);
    fa.inv_ny = 1.0f / static_cast<float>(o->ny);
    // iterations in chunks; the stop flag is read between chunks
    constexpr int kChunk = 128;
    int t = 1;
    while (t <= I) {
        const int t_end = std::min(I, t + kChunk - 1);
        for (; t <= t_end; ++t) {
            double c1 = 1.0 - std::pow(o->beta1, t), c2 = 1.0 - std::pow(o->beta2, t);
            if (PREC == GAC_PREC_FP32) {  // the FP32 kernel multiplies by the reciprocals
                c1 = 1.0 / c1;
                c2 = 1.0 / c2;
            }
            const void *ui = (t & 1) ? u0 : u1;
            void *uo = (t & 1) ? u1 : u0;
            if ((e = launch_step_kind<PREC>(mc.kind, l1, grid, smem, s, mc, fa, ui, uo, m1, m2, c1, c2, t)) != cudaSuccess)
                return cuda_fail(e, "fit step");
        }
        int stop = 0;
        if ((e = cudaMemcpyAsync(&stop, flags, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_fail(e, "fit flag");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "fit");
        if (stop) break;
    }
    int done = 0;
    if ((e = cudaMemcpyAsync(&done, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "fit done");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "fit");
    if (iterations_done) *iterations_done = done;
    if (loss_history && done > 0) {
        if ((e = cudaMemcpyAsync(loss_history, hist, done * sizeof(double), cudaMemcpyDefault, s)) != cudaSuccess)
            return cuda_fail(e, "loss history");
    }
    // u of the last update (iteration `done` wrote buffer (done & 1) ? u1 : u0) -> theta
    const void *u_fin = done == 0 ? u0 : ((done & 1) ? u1 : u0);
    u_to_theta_kernel<R><<<conv_grid, 256, 0, s>>>(mc, static_cast<const R *>(u_fin), d_mask, N,
                                                   static_cast<double *>(d_theta.ptr));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "u to theta");
    if ((st = d_theta.copy_out()) != GAC_OK) return st;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "fit");
    return GAC_OK;
}

}  // namespace gac

using namespace gac;

extern "C" gac_status gac_fit_run(int model_id, const void *data, const uint8_t *mask, const float *weight,
                                  const gac_fit_opts *o, double *theta, double *loss_history, int *iterations_done,
                                  void *stream) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (!o || !theta || !data) return fail(GAC_ERR_INVALID_ARG, "opts, theta and data must not be NULL");
    if (mc.kind == GAC_MODEL_AXCAL_SMT) return fail(GAC_ERR_INVALID_ARG, "no analytic gradient for AxCaliberSMT");
    if (o->nx < 1 || o->ny < 1 || o->nz < 1) return fail(GAC_ERR_INVALID_ARG, "grid extents must be >= 1");
    if (o->loss != GAC_FIT_L1 && o->loss != GAC_FIT_L2) return fail(GAC_ERR_INVALID_ARG, "unknown loss %d", o->loss);
    if (o->iterations < 0) return fail(GAC_ERR_INVALID_ARG, "iterations must be >= 0");
    if (!(o->learning_rate > 0) || !(o->beta1 >= 0 && o->beta1 < 1) || !(o->beta2 >= 0 && o->beta2 < 1) || !(o->epsilon > 0))
        return fail(GAC_ERR_INVALID_ARG, "Adam needs learning_rate > 0, beta in [0, 1), epsilon > 0");
    if (o->tv_dims != 2 && o->tv_dims != 3) return fail(GAC_ERR_INVALID_ARG, "tv_dims must be 2 or 3");
    if (!(o->tv_lambda >= 0) || !(o->tol >= 0) || !(o->convergence_value >= 0))
        return fail(GAC_ERR_INVALID_ARG, "tv_lambda, tol and convergence_value must be >= 0");
    if (o->convergence_value > 0 && (o->convergence_window < 2 || o->convergence_window > kFitMaxWindow))
        return fail(GAC_ERR_INVALID_ARG, "convergence_window must be in [2, %d]", kFitMaxWindow);
    if (o->precision != GAC_PREC_FP32 && o->precision != GAC_PREC_FP64)
        return fail(GAC_ERR_INVALID_ARG, "precision must be FP32 or FP64");
    const int64_t N = static_cast<int64_t>(o->nx) * o->ny * o->nz;
    const int M = mc.n_meas;
    if (N * mc.n_par >= (int64_t(1) << 31))
        return fail(GAC_ERR_INVALID_ARG, "the fit takes fewer than 2^31 / %d voxels (32-bit indexing)", mc.n_par);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    keep_staging_pool();
    if (o->iterations == 0) {
        if (iterations_done) *iterations_done = 0;
        return GAC_OK;
    }
    // the mask count, from the caller's buffer: counted in place (host), or
    // on the device with only the count read back
    int64_t n_mask = N;
    if (mask) {
        if (is_device_ptr(mask)) {
            unsigned long long *d_count = nullptr, h_count = 0;
            cudaError_t e = cudaMallocAsync(&d_count, sizeof *d_count, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, sizeof *d_count, s);
            if (e == cudaSuccess) {
                int dev = 0, sms = 0;
                e = cudaGetDevice(&dev);
                if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (e == cudaSuccess) {
                    const int g = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, int64_t(sms) * 4)));
                    count_mask_kernel<<<g, 256, 0, s>>>(mask, N, d_count);
                    e = cudaGetLastError();
                }
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h_count, d_count, sizeof h_count, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (d_count) cudaFreeAsync(d_count, s);
            if (e != cudaSuccess) return cuda_fail(e, "mask count");
            n_mask = static_cast<int64_t>(h_count);
        } else {
            n_mask = 0;
            for (int64_t i = 0; i < N; ++i) n_mask += mask[i] != 0;
        }
    }
    if (n_mask == 0) {
        if (iterations_done) *iterations_done = 0;
        return GAC_OK;
    }
    DevBuf d_data, d_mask, d_weight;
    // every iteration rereads the data, mask and weights: stage them in device memory
    if ((st = d_data.make(const_cast<void *>(data), static_cast<size_t>(N) * M * sizeof(float), true, s, "data", true)) != GAC_OK)
        return st;
    if ((st = d_mask.make(const_cast<uint8_t *>(mask), mask ? static_cast<size_t>(N) : 0, true, s, "mask", true)) != GAC_OK)
        return st;
    if ((st = d_weight.make(const_cast<float *>(weight), weight ? static_cast<size_t>(N) * sizeof(float) : 0, true, s, "weight",
                            true)) != GAC_OK)
        return st;
    const auto *dd = static_cast<const float *>(d_data.ptr);
    const auto *dm = static_cast<const uint8_t *>(d_mask.ptr);
    const auto *dw = static_cast<const float *>(d_weight.ptr);
    return o->precision == GAC_PREC_FP64
               ? fit_run_prec<GAC_PREC_FP64>(mc, o, dd, dm, dw, n_mask, theta, loss_history, iterations_done, s)
               : fit_run_prec<GAC_PREC_FP32>(mc, o, dd, dm, dw, n_mask, theta, loss_history, iterations_done, s);
}
