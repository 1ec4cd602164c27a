// Forward signal models on the device, in FP32 (MIXED and FP32 paths) and
// FP64, each written as `eval(theta, mc, visit)` that calls visit(k, s_k) or
// visit(k, re_k, im_k) for every acquisition k.  The sampler's likelihood and
// the gac_forward test entry point both go through eval, so they share one
// arithmetic.
//
//  MONOEXP (Eq. 3): s_k = S0 exp(-R2* TE_k), TE in ms, R2* in 1/s.
//  MWI3:  S(t) = exp(i phi0) sum_j A_j exp(-t/T2*_j) exp(-i 2 pi df_j t), df_EW = 0.
//  SMT:   s(b) = f g(b Da) + (1-f) exp(-b De_perp) g(b (De_par - De_perp)),
//         g(x) = integral_0^1 exp(-x u^2) du.
//  LINEAR_TEST: s_k = a + c t_k.
//
// FP32 evaluation of evenly spaced echoes (MONOEXP, MWI3) uses an anchored
// geometric recurrence: with t_k = t_0 + k dt, each pool's term is
// E_k = E_0 R^k with R = exp(-dt (rate + i w)).  Inside a block of K = 6
// echoes the term advances by one complex multiply, and each block starts
// from the previous anchor times R^K.  This replaces 3 transcendental calls
// per echo and pool by one multiply.  MONOEXP takes E_0, R and R^K from expf.
// MWI3, whose log-likelihood at high SNR needs the forward model to a few
// 1e-7, carries R and R^K as d = R - 1 (small for the slowly decaying pools,
// so their rounding is far below an ulp of R and does not compound along a
// block) and computes E_0, d and d_K from double-float arguments with an own
// expm1 and sincos (details at eval_mwi3_f).
// Unevenly spaced echoes, and the FP64 path, evaluate every echo directly.
#pragma once
#include <cstdint>
#include <type_traits>

#include "gac.h"

namespace gac {

constexpr int kAnchor = 6;
constexpr float kSinCosMaxArg = 6000.0f;  // |x| bound of sincos_cw (registration checks it)
constexpr float kSmtArgMin = -12.0f;  // registration keeps b (De_par - De_perp), b Da >= -12
constexpr int kGTabMax = 96;          // half-unit intervals of the g(x) table, centres c_lo/2 .. c_hi/2
constexpr float kGTail = 16.0f;       // x >= 16: g(x) = sqrt(pi)/2 x^-1/2 within erfc(4) = 1.5e-8

// AxCaliberSMT (Sec. 2.5, after Fan et al. 2020): measurements are
// (b, Delta, delta) triplets; the cylinder series runs over the zeros of J1'.
constexpr int kAxMaxMeas = GAC_MAX_ACQ / 3;
constexpr int kAxMaxTiming = 4;   // distinct (Delta, delta) pairs
constexpr int kAxMaxTerms = 64;   // zeros of J1' in the series
constexpr int kAxTabMax = 16;     // intervals of the FP32 table of the series in log2 R
constexpr float kAxDa = 1.7f, kAxDePar = 1.7f, kAxDcsf = 3.0f;  // um^2/ms (fixed, Sec. 2.5)
constexpr double kAxDaD = 1.7, kAxDeParD = 1.7, kAxDcsfD = 3.0;

struct AxConst {
    int n_timing;       // distinct (Delta, delta)
    int terms_f;        // series terms of the FP32 evaluation (tail < 2e-8 on the prior box)
    int terms_d;        // of the FP64 evaluation
    int careful_f;      // leading terms whose q delta can fall below 1 on the prior box
    int t[kAxMaxMeas];  // timing of measurement k
    float b_f[kAxMaxMeas], g2_f[kAxMaxMeas], csf_f[kAxMaxMeas];  // b, gamma^2 G^2, e^{-b D_csf}
    double b_d[kAxMaxMeas], g2_d[kAxMaxMeas], csf_d[kAxMaxMeas];
    float delta_f[kAxMaxTiming], Delta_f[kAxMaxTiming];
    double delta_d[kAxMaxTiming], Delta_d[kAxMaxTiming];
    // term m: c_m = 2 / (Da^2 x_m^6 (x_m^2 - 1)), x_m^2 Da (q = x_m^2 Da / R^2)
    float c_f[kAxMaxTerms], x2d_f[kAxMaxTerms];
    double c_d[kAxMaxTerms], x2d_d[kAxMaxTerms];
    // FP32 path: phi_j(R) = R^6 sum_m c_m N_m per timing j as a piecewise
    // degree-7 polynomial in log2 R (intervals of width 1/tab_inv_w from
    // log2 of the smallest radius; centred coordinate in [-1/2, 1/2]), used
    // when tab_n > 0 (registration checks it against the series).  Layout
    // [timing][2][kAxTabMax][4]: a_0..a_3 of every interval, then a_4..a_7.
    int tab_n;
    float tab_off, tab_inv_w;  // t = log2 R * tab_inv_w + tab_off; interval rint(t), d = t - rint(t)
    alignas(16) float tab[kAxMaxTiming * 2 * kAxTabMax * 4];
    // FP32 path, measurements in timing order: timing j owns positions
    // first[j] .. first[j+1]-1; position i holds (b Da, g2, g2 log2 e,
    // b log2 e) and (b, e^{-b D_csf}, the measurement's index as int bits, 0).
    int first[kAxMaxTiming + 1];
    alignas(16) float meas[kAxMaxMeas * 2 * 4];
};

struct ModelConst {
    int kind;
    int n_par;
    int n_acq;
    int n_meas;
    int even;       // acquisitions evenly spaced (recurrence allowed)
    float t0_f, dt_f, dtk_f;  // first acquisition, spacing, kAnchor * spacing
    // the same as double-float pairs (x = hi + lo), and 2 pi 1e-3 t for t =
    // t0, dt, kAnchor dt (the phase per Hz, in rad), for the 3-pool recurrence
    float2 dd_t0, dd_dt, dd_w0, dd_w1, dd_wk;
    // 3-pool set-up shortcuts that registration proved safe for every
    // parameter the bounds allow: kMwi3SmallB |2 pi 1e-3 df t| <= pi/4 for
    // t = t0, dt; kMwi3SmallBK the same for t = kAnchor dt / 2;
    // kMwi3SmallEW t / T2*_EW <= ln2/2 for t = t0, dt
    int mwi3_flags;
    float2 dd_wkh;  // dd_wk / 2
    float acq_f[GAC_MAX_ACQ];
    float acq_l2e_f[GAC_MAX_ACQ];  // acquisition x log2 e (exponentials as 2^x)
    double acq_d[GAC_MAX_ACQ];
    float lb_f[GAC_MAX_PAR], ub_f[GAC_MAX_PAR], step_f[GAC_MAX_PAR];
    double lb_d[GAC_MAX_PAR], ub_d[GAC_MAX_PAR], step_d[GAC_MAX_PAR];
    // g(x) = int_0^1 exp(-x u^2) du on half-unit intervals centred at the
    // half-integers c = k/2, k = gtab_lo .. gtab_lo + gtab_n - 1:
    // g(c + d) = sum_{n<=5} a_n d^n for |d| <= 1/4 (the Chebyshev interpolant
    // of degree 5).  Layout [2][kGTabMax][4]: a_0..a_3 of every interval, then
    // a_4, a_5 (and two zeros), so one interval is two 16-byte loads.  When
    // the table covers every argument the model's bounds allow, gtab_tail =
    // 0; otherwise x >= gtab_tail_x (>= 16.25) takes the asymptote
    // sqrt(pi)/2 x^-1/2.
    alignas(16) float gtab[2 * kGTabMax * 4];
    int gtab_lo;
    int gtab_n;
    int gtab_tail;
    float gtab_tail_x;
    AxConst ax;  // GAC_MODEL_AXCAL_SMT only
};

__host__ __device__ constexpr int model_n_par(int kind) {
    return kind == GAC_MODEL_MONOEXP ? 2
         : kind == GAC_MODEL_MWI3 ? 9
         : kind == GAC_MODEL_SMT ? 4
         : kind == GAC_MODEL_AXCAL_SMT ? 4
         : kind == GAC_MODEL_LINEAR_TEST ? 2 : -1;
}
__host__ __device__ constexpr bool model_complex(int kind) { return kind == GAC_MODEL_MWI3; }

constexpr int kMwi3SmallB = 1, kMwi3SmallBK = 2, kMwi3SmallEW = 4;
constexpr float kTwoPiMilli = 6.28318530717958648e-3f;  // 2 pi * 1e-3: Hz * ms -> rad
constexpr double kTwoPiMilliD = 6.28318530717958648e-3;
constexpr float kSqrtPiHalf = 0.886226925452758014f;
constexpr double kSqrtPiHalfD = 0.886226925452758014;

// ---------------------------------------------------------------- g(x) ----
// The g(x) table of the block's model, copied from ModelConst by
// model_smem_load before the first evaluation (the lookups of a warp go to
// different intervals, which the constant bank would serialise).
static __shared__ float4 smt_gtab_s[2 * kGTabMax];

// The AxCaliberSMT series table and per-measurement constants of the
// block's model (FP32 path).
static __shared__ float4 ax_tab_s[kAxMaxTiming * 2 * kAxTabMax];
static __shared__ float4 ax_meas_s[kAxMaxMeas * 2];

template <int KIND>
__device__ __forceinline__ void model_smem_load(const ModelConst &mc) {
    if constexpr (KIND == GAC_MODEL_SMT || KIND == GAC_MODEL_AXCAL_SMT) {
        float *dst = reinterpret_cast<float *>(smt_gtab_s);
        for (int e = threadIdx.x; e < 2 * kGTabMax * 4; e += blockDim.x) dst[e] = mc.gtab[e];
    }
    if constexpr (KIND == GAC_MODEL_AXCAL_SMT) {
        float *dst = reinterpret_cast<float *>(ax_tab_s);
        for (int e = threadIdx.x; e < kAxMaxTiming * 2 * kAxTabMax * 4; e += blockDim.x) dst[e] = mc.ax.tab[e];
        float *dm = reinterpret_cast<float *>(ax_meas_s);
        for (int e = threadIdx.x; e < kAxMaxMeas * 2 * 4; e += blockDim.x) dm[e] = mc.ax.meas[e];
    }
}

// 2^x on the special-function unit (ex2.approx; the callers fold log2 e into
// their constants).
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// g(x) in FP32 without branches: the interval is k = rint(2x), taken from
// the bits of 2x + 1.5 * 2^23 (exact for |x| < 2^21), and d = x - k/2 is
// exact; Horner in d over the interval's six coefficients.  With TAIL, x >=
// gtab_tail_x takes the asymptote sqrt(pi)/2 x^-1/2 instead (relative error
// below erfc(4)); without it the table covers every argument the bounds
// allow.  The clamped index keeps every load inside the table for any x.
template <bool TAIL>
__device__ __forceinline__ float smt_g_f(float x, const ModelConst &mc) {
    constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
    const float t = fmaf(x, 2.0f, kRound);
    const float d = fmaf(t - kRound, -0.5f, x);
    // one unsigned min keeps the index in the table (a negative index wraps
    // to a large unsigned value)
    const int i = static_cast<int>(min(static_cast<unsigned>(__float_as_int(t) - __float_as_int(kRound) - mc.gtab_lo),
                                       static_cast<unsigned>(mc.gtab_n - 1)));
    const float4 lo = smt_gtab_s[i];
    const float4 hi = smt_gtab_s[kGTabMax + i];
    float p = fmaf(hi.y, d, hi.x);
    p = fmaf(p, d, lo.w);
    p = fmaf(p, d, lo.z);
    p = fmaf(p, d, lo.y);
    p = fmaf(p, d, lo.x);
    if constexpr (TAIL) {
        const float tail = kSqrtPiHalf * rsqrtf(x);
        return x >= mc.gtab_tail_x ? tail : p;
    } else {
        return p;
    }
}

__device__ __forceinline__ double smt_g_d(double x) {
    if (x > 0.0) {
        if (x < 1e-300) return 1.0;
        const double s = sqrt(x);
        return kSqrtPiHalfD * erf(s) / s;
    }
    const double y = -x;
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 200; ++n) {
        term *= y / n;
        const double add = term / (2 * n + 1);
        sum += add;
        if (add <= 1e-17 * sum) break;
    }
    return sum;
}

// g(x) and g'(x) in FP32 from the same table: the interval polynomial and its
// derivative (d/dx = d/dd); g' = -g / (2x) on the tail.
__device__ __forceinline__ void smt_g_dg(float x, const ModelConst &mc, float &g, float &dg) {
    constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
    const float t = fmaf(x, 2.0f, kRound);
    const float d = fmaf(t - kRound, -0.5f, x);
    int i = __float_as_int(t) - __float_as_int(kRound) - mc.gtab_lo;
    i = min(max(i, 0), mc.gtab_n - 1);
    const float4 lo = smt_gtab_s[i];
    const float4 hi = smt_gtab_s[kGTabMax + i];
    float p = fmaf(hi.y, d, hi.x), q = fmaf(5.0f * hi.y, d, 4.0f * hi.x);
    p = fmaf(p, d, lo.w);
    q = fmaf(q, d, 3.0f * lo.w);
    p = fmaf(p, d, lo.z);
    q = fmaf(q, d, 2.0f * lo.z);
    p = fmaf(p, d, lo.y);
    q = fmaf(q, d, lo.y);
    p = fmaf(p, d, lo.x);
    if (mc.gtab_tail && x >= mc.gtab_tail_x) {
        const float tail = kSqrtPiHalf * rsqrtf(x);
        g = tail;
        dg = -0.5f * tail / x;
    } else {
        g = p;
        dg = q;
    }
}

// g(x) and g'(x) in FP64: g' = (e^{-x} - g(x)) / (2x) (integration by parts of
// -int u^2 e^{-x u^2} du), and near 0, where that form cancels, its Taylor
// series sum_{n>=1} (-1)^n x^(n-1) / ((n-1)! (2n+1)).
__device__ __forceinline__ void smt_g_dg(double x, const ModelConst &, double &g, double &dg) {
    g = smt_g_d(x);
    if (fabs(x) > 0.5) {
        dg = (exp(-x) - g) / (2.0 * x);
        return;
    }
    double term = -1.0, sum = 0.0;  // term = (-1)^n x^(n-1) / (n-1)!
    for (int n = 1; n < 40; ++n) {
        const double add = term / (2.0 * n + 1.0);  // (-1)^n n x^(n-1) / (n! (2n+1))
        sum += add;
        if (fabs(add) <= 1e-17 * fabs(sum)) break;
        term *= -x / n;
    }
    dg = sum;
}

// sin and cos of x in FP32 for |x| <= kSinCosMaxArg.  Cody & Waite's
// additive range reduction by pi/2 ("Software Manual for the Elementary
// Functions", 1980) with a three-part constant whose first two parts have
// 12 trailing zero bits, so that q * part is exact for |q| < 2^12; then the
// Taylor polynomials of sin (degree 9) and cos (degree 10) on |r| <= pi/4,
// whose truncation errors are below 3e-9 and 2e-10.  No branches.
__device__ __forceinline__ void sincos_cw(float x, float &sn, float &cs) {
    const float q = rintf(x * 0.636619772367581343f);  // round(x * 2/pi)
    float r = fmaf(q, -1.5703125f, x);                   // pi/2 = 1.5703125
    r = fmaf(q, -4.837512969970703125e-4f, r);           //     + 4.8375129699707e-4
    r = fmaf(q, -7.549790126404332e-8f, r);              //     + 7.5497901264e-8
    const float r2 = r * r;
    float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);  //  1/9!, -1/7!
    ps = fmaf(ps, r2, 8.33333333e-3f);                     //  1/5!
    ps = fmaf(ps, r2, -1.66666667e-1f);                    // -1/3!
    const float sr = fmaf(ps * r2, r, r);
    float pc = fmaf(r2, -2.75573192e-7f, 2.48015873e-5f);  // -1/10!, 1/8!
    pc = fmaf(pc, r2, -1.38888889e-3f);                    // -1/6!
    pc = fmaf(pc, r2, 4.16666667e-2f);                     //  1/4!
    pc = fmaf(pc, r2, -0.5f);                              // -1/2!
    const float cr = fmaf(pc, r2, 1.0f);
    const int n = static_cast<int>(q);  // quadrant: x = n pi/2 + r
    const float a = (n & 1) ? cr : sr;
    const float b = (n & 1) ? sr : cr;
    sn = (n & 2) ? -a : a;
    cs = ((n + 1) & 2) ? -b : b;
}

// Paired FP32 arithmetic (Blackwell's two-lane FFMA2/FADD2/FMUL2): each lane
// performs exactly the operation of the scalar code, so results are
// bit-identical while two values take one instruction.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// sincos_cw on both lanes of x.
__device__ __forceinline__ void sincos_cw2(float2 x, float2 &sn, float2 &cs) {
    const float2 qx = __fmul2_rn(x, f2(0.636619772367581343f));
    const float2 q = make_float2(rintf(qx.x), rintf(qx.y));
    float2 r = __ffma2_rn(q, f2(-1.5703125f), x);
    r = __ffma2_rn(q, f2(-4.837512969970703125e-4f), r);
    r = __ffma2_rn(q, f2(-7.549790126404332e-8f), r);
    const float2 r2 = __fmul2_rn(r, r);
    float2 ps = __ffma2_rn(r2, f2(2.75573192e-6f), f2(-1.98412698e-4f));
    ps = __ffma2_rn(ps, r2, f2(8.33333333e-3f));
    ps = __ffma2_rn(ps, r2, f2(-1.66666667e-1f));
    const float2 sr = __ffma2_rn(__fmul2_rn(ps, r2), r, r);
    float2 pc = __ffma2_rn(r2, f2(-2.75573192e-7f), f2(2.48015873e-5f));
    pc = __ffma2_rn(pc, r2, f2(-1.38888889e-3f));
    pc = __ffma2_rn(pc, r2, f2(4.16666667e-2f));
    pc = __ffma2_rn(pc, r2, f2(-0.5f));
    const float2 cr = __ffma2_rn(pc, r2, f2(1.0f));
    const int n0 = static_cast<int>(q.x), n1 = static_cast<int>(q.y);
    const float a0 = (n0 & 1) ? cr.x : sr.x, b0 = (n0 & 1) ? sr.x : cr.x;
    const float a1 = (n1 & 1) ? cr.y : sr.y, b1 = (n1 & 1) ? sr.y : cr.y;
    sn = make_float2((n0 & 2) ? -a0 : a0, (n1 & 2) ? -a1 : a1);
    cs = make_float2(((n0 + 1) & 2) ? -b0 : b0, ((n1 + 1) & 2) ? -b1 : b1);
}

// sincos_cw on both lanes, also returning cm = cos x - 1.  For |x| <= pi/4
// (no quadrant shift) cm is the polynomial's own cos r - 1 = r^2 pc, so it
// keeps its relative accuracy however small x is; otherwise cos x is far from
// 1 and cm = cos x - 1 loses nothing.
__device__ __forceinline__ void sincos_cm2(float2 x, float2 &sn, float2 &cs, float2 &cm) {
    const float2 qx = __fmul2_rn(x, f2(0.636619772367581343f));
    const float2 q = make_float2(rintf(qx.x), rintf(qx.y));
    float2 r = __ffma2_rn(q, f2(-1.5703125f), x);
    r = __ffma2_rn(q, f2(-4.837512969970703125e-4f), r);
    r = __ffma2_rn(q, f2(-7.549790126404332e-8f), r);
    const float2 r2 = __fmul2_rn(r, r);
    float2 ps = __ffma2_rn(r2, f2(2.75573192e-6f), f2(-1.98412698e-4f));
    ps = __ffma2_rn(ps, r2, f2(8.33333333e-3f));
    ps = __ffma2_rn(ps, r2, f2(-1.66666667e-1f));
    const float2 sr = __ffma2_rn(__fmul2_rn(ps, r2), r, r);
    float2 pc = __ffma2_rn(r2, f2(-2.75573192e-7f), f2(2.48015873e-5f));
    pc = __ffma2_rn(pc, r2, f2(-1.38888889e-3f));
    pc = __ffma2_rn(pc, r2, f2(4.16666667e-2f));
    pc = __ffma2_rn(pc, r2, f2(-0.5f));
    const float2 cm0 = __fmul2_rn(pc, r2);  // cos r - 1
    const float2 cr = __fadd2_rn(cm0, f2(1.0f));
    const int n0 = static_cast<int>(q.x), n1 = static_cast<int>(q.y);
    const float a0 = (n0 & 1) ? cr.x : sr.x, b0 = (n0 & 1) ? sr.x : cr.x;
    const float a1 = (n1 & 1) ? cr.y : sr.y, b1 = (n1 & 1) ? sr.y : cr.y;
    sn = make_float2((n0 & 2) ? -a0 : a0, (n1 & 2) ? -a1 : a1);
    cs = make_float2(((n0 + 1) & 2) ? -b0 : b0, ((n1 + 1) & 2) ? -b1 : b1);
    cm = make_float2(n0 == 0 ? cm0.x : cs.x - 1.0f, n1 == 0 ? cm0.y : cs.y - 1.0f);
}

// e^x - 1 on both lanes, FP32, relative accuracy kept for small |x|.  With
// k = rint(x log2 e) and r = x - k ln 2 (ln 2 split Cody-Waite style, the
// high part with 9 trailing zero bits so that k * hi is exact for |k| < 2^9),
// e^r - 1 is its Taylor series to r^8/8! (|r| <= ln2/2: the rest is below
// 6e-10 of the value) and e^x - 1 = 2^k (e^r - 1) + (2^k - 1).  For |x| <
// ln2/2 (k = 0) the result is the polynomial itself.  x >= -80 after a clamp
// (e^-80 - 1 = -1 in FP32); callers keep x <= 80, so 2^k stays a normal float.
// SMALL: the caller guarantees |x| <= ln2/2, so k = 0 and r = x.
template <bool SMALL = false>
__device__ __forceinline__ float2 expm1_f2(float2 x) {
    constexpr float kRound = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer
    float2 t, r;
    if constexpr (SMALL) {
        r = x;
    } else {
        x = make_float2(fmaxf(x.x, -80.0f), fmaxf(x.y, -80.0f));
        t = __ffma2_rn(x, f2(1.44269504088896341f), f2(kRound));
        const float2 k = __fadd2_rn(t, f2(-kRound));
        r = __ffma2_rn(k, f2(-0.693145751953125f), x);
        r = __ffma2_rn(k, f2(-1.42860682030941723e-6f), r);
    }
    float2 p = __ffma2_rn(r, f2(2.48015873015873016e-5f), f2(1.98412698412698413e-4f));  // 1/8!, 1/7!
    p = __ffma2_rn(p, r, f2(1.38888888888888889e-3f));                                   // 1/6!
    p = __ffma2_rn(p, r, f2(8.33333333333333333e-3f));                                   // 1/5!
    p = __ffma2_rn(p, r, f2(4.16666666666666667e-2f));                                   // 1/4!
    p = __ffma2_rn(p, r, f2(1.66666666666666667e-1f));                                   // 1/3!
    p = __ffma2_rn(p, r, f2(0.5f));                                                      // 1/2!
    const float2 em = __ffma2_rn(__fmul2_rn(r, r), p, r);
    if constexpr (SMALL) return em;
    // 2^k from the low bits of t (k + 127 is the biased exponent)
    const float2 p2k = make_float2(__int_as_float((__float_as_int(t.x) << 23) + 0x3f800000),
                                   __int_as_float((__float_as_int(t.y) << 23) + 0x3f800000));
    return __ffma2_rn(p2k, em, __fadd2_rn(p2k, f2(-1.0f)));
}

// sin x and cos x - 1 on both lanes for |x| <= pi/4: the Taylor polynomials of
// sincos_cw without its range reduction (cos x - 1 = x^2 pc keeps its
// relative accuracy for small x).
__device__ __forceinline__ void sincos_small2(float2 x, float2 &sn, float2 &cm) {
    const float2 r2 = __fmul2_rn(x, x);
    float2 ps = __ffma2_rn(r2, f2(2.75573192e-6f), f2(-1.98412698e-4f));
    ps = __ffma2_rn(ps, r2, f2(8.33333333e-3f));
    ps = __ffma2_rn(ps, r2, f2(-1.66666667e-1f));
    sn = __ffma2_rn(__fmul2_rn(ps, r2), x, x);
    float2 pc = __ffma2_rn(r2, f2(-2.75573192e-7f), f2(2.48015873e-5f));
    pc = __ffma2_rn(pc, r2, f2(-1.38888889e-3f));
    pc = __ffma2_rn(pc, r2, f2(4.16666667e-2f));
    pc = __ffma2_rn(pc, r2, f2(-0.5f));
    cm = __fmul2_rn(pc, r2);
}

// 1/x on the special-function unit (rcp.approx, ~1 ulp); callers that need
// the exact reciprocal add the Newton residual r (1 - r x) as a low part.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ----------------------------------------------------------- FP32 models --
// Tells a visitor that a block of echoes of a recurrence is complete, if it
// wants to know (visitors without block_end() ignore it).
template <class V>
__device__ __forceinline__ auto end_block(V &v, int) -> decltype(v.block_end(), void()) {
    v.block_end();
}
template <class V>
__device__ __forceinline__ void end_block(V &, long) {}

// The mono-exponential recurrence for evenly spaced echoes: the first
// anchor S0 e^{-t0 R2*} and the per-echo and per-block ratios.
struct MonoRec {
    float anchor, r1, rk;
};
__device__ __forceinline__ MonoRec monoexp_setup_f(const float *th, const ModelConst &mc) {
    const float rate = th[1] * 1e-3f;  // 1/s -> 1/ms
    return {th[0] * expf(-mc.t0_f * rate), expf(-mc.dt_f * rate), expf(-mc.dtk_f * rate)};
}

// Echoes a .. a+cnt-1 (FULL: cnt = kAnchor) from the block's anchor.
template <bool FULL, class V>
__device__ __forceinline__ void monoexp_block_f(float e, float r1, int a, int cnt, V &visit) {
#pragma unroll
    for (int i = 0; i < kAnchor; ++i) {
        if (FULL || i < cnt) visit(a + i, e);
        e = __fmul_rn(e, r1);
    }
}

template <class V>
__device__ __forceinline__ void eval_monoexp_f(const float *th, const ModelConst &mc, V &&visit) {
    const float s0 = th[0];
    const float rate = th[1] * 1e-3f;  // 1/s -> 1/ms
    const int n = mc.n_acq;
    if (mc.even) {
        const MonoRec mr = monoexp_setup_f(th, mc);
        float anchor = mr.anchor;
        const float r1 = mr.r1;
        const float rk = mr.rk;
        // products rounded explicitly (never contracted into the residual's
        // subtraction), so that every caller of this recurrence -- the
        // one-thread and the lane-split samplers -- gets the same bits
        int a = 0;
        for (; a + kAnchor <= n; a += kAnchor) {
            monoexp_block_f<true>(anchor, r1, a, kAnchor, visit);
            end_block(visit, 0);
            anchor = __fmul_rn(anchor, rk);
        }
        if (a < n) monoexp_block_f<false>(anchor, r1, a, n - a, visit);  // last, partial block
    } else {
        for (int k0 = 0; k0 < n; k0 += kAnchor) {
            const int k1 = min(k0 + kAnchor, n);
            for (int k = k0; k < k1; ++k) visit(k, s0 * expf(-mc.acq_f[k] * rate));
            end_block(visit, 0);
        }
    }
}

// The 3-pool recurrence for evenly spaced echoes: its set-up (anchors of the
// first block and the ratios in delta form), one block of echoes, and the
// step from one block's anchors to the next.  eval_mwi3_f strings them
// together; the lane-split sampler gives the blocks to different lanes,
// each lane stepping its anchors the same way, so both give the same bits.
struct Mwi3Rec {
    float2 X, Y, Z;              // anchors of block 0: (Re MW, Re IW), (Im MW, Im IW), (Re EW, Im EW)
    float2 DR, DI, NDI;          // per-echo ratio - 1 of MW, IW (real, imaginary, -imaginary)
    float2 KR, KI, NKI;          // per-block ratio - 1 of MW, IW
    float dE, dKE;               // per-echo and per-block ratio - 1 of EW (real)
};

__device__ __forceinline__ Mwi3Rec mwi3_setup_f(const float *th, const ModelConst &mc) {
    const float phi0 = th[8];
    // Per pool j: E_0 = A_j e^{-t0/T2*_j} e^{i(phi0 - w_j t0)} and the ratios
    // R = e^{-dt (1/T2*_j + i w_j)} and R^K, the ratios in delta form
    // d = R - 1.  The slow pools have |d| << 1, so rounding d costs far
    // less than an ulp of R, and E <- E + E d advances a term without
    // compounding R's own rounding over the block.  The set-up, in FP32:
    //  - a = t / T2* for t = t0, dt as a double-float (t and 1/T2* as
    //    hi + lo pairs), e^{-a} - 1 = expm1_f2(-a_hi) - a_lo e^{-a};
    //  - (1 + em_dt)^K - 1 by squaring in delta form;
    //  - the phases b = w t = df (2 pi 1e-3 t) as double-floats, the
    //    phasor e^{-ib} - 1 = (cos b - 1, -sin b) of the high part,
    //    corrected to first order by the low part;
    //  - d = (1 + em)(1 + cm + i sn) - 1 = em + cm + em cm + i (sn + em sn);
    //  - E_0 = A (1 + em_0) e^{i phi0} e^{-i b0}, the last factor applied
    //    in delta form to e^{i phi0} (which the extra-cellular pool uses
    //    as it is), and A (1 + em_0) c = A c + (A em_0 c + err(A c)).
    // The myelin- and intra-axonal pools (frequency offsets) are carried as
    // lane pairs: X = (Re E_MW, Re E_IW), Y = (Im E_MW, Im E_IW); the
    // extra-cellular pool, whose ratio is real, as Z = (Re E_EW, Im E_EW).
    static_assert(kAnchor == 6, "R^K is formed as ((1 + d)^2 (1 + d))^2");
    const float2 T2 = make_float2(th[3], th[4]);
    const float2 rh = make_float2(rcp_approx(th[3]), rcp_approx(th[4]));
    const float2 rl = __fmul2_rn(rh, __ffma2_rn(neg2(rh), T2, f2(1.0f)));
    const float rh2 = rcp_approx(th[5]);
    const float rl2 = rh2 * fmaf(-rh2, th[5], 1.0f);
    // e^{-t r} - 1 per lane, t = th + tl, r = rh + rl
    auto em_of = [](float2 rh_, float2 rl_, float2 th_, float2 tl_, auto small) {
        const float2 ah = __fmul2_rn(rh_, th_);
        float2 al = __ffma2_rn(rh_, th_, neg2(ah));
        al = __ffma2_rn(rl_, th_, al);
        al = __ffma2_rn(rh_, tl_, al);
        const float2 em = expm1_f2<decltype(small)::value>(neg2(ah));
        return __ffma2_rn(neg2(al), em, __fadd2_rn(em, neg2(al)));
    };
    using Full = std::false_type;
    const float2 em0 = em_of(rh, rl, f2(mc.dd_t0.x), f2(mc.dd_t0.y), Full{});  // MW, IW over t0
    const float2 em1 = em_of(rh, rl, f2(mc.dd_dt.x), f2(mc.dd_dt.y), Full{});  // MW, IW over dt
    const float2 tE = make_float2(mc.dd_t0.x, mc.dd_dt.x), tlE = make_float2(mc.dd_t0.y, mc.dd_dt.y);
    const float2 emE = (mc.mwi3_flags & kMwi3SmallEW) ? em_of(f2(rh2), f2(rl2), tE, tlE, std::true_type{})
                                                      : em_of(f2(rh2), f2(rl2), tE, tlE, Full{});  // EW over t0, dt
    // (1 + e)^6 - 1: e2 = e (2 + e), e3 = e2 + e + e2 e, e6 = e3 (2 + e3)
    const float2 e2 = __ffma2_rn(em1, em1, __fadd2_rn(em1, em1));
    const float2 e3 = __ffma2_rn(e2, em1, __fadd2_rn(e2, em1));
    const float2 emK = __ffma2_rn(e3, e3, __fadd2_rn(e3, e3));
    const float dE = emE.y;
    const float dE2 = fmaf(dE, dE, dE + dE), dE3 = fmaf(dE2, dE, dE2 + dE);
    const float dKE = fmaf(dE3, dE3, dE3 + dE3);
    // phases b = df (2 pi 1e-3 t) as hi + lo
    const float2 df = make_float2(th[6], th[7]);
    auto phase = [&df](float2 c, float2 &lo) {
        const float2 bh = __fmul2_rn(df, f2(c.x));
        lo = __ffma2_rn(df, f2(c.y), __ffma2_rn(df, f2(c.x), neg2(bh)));
        return bh;
    };
    // e^{-i(bh + bl)} - 1 as (cos - 1, sin); SMALL: |bh| <= pi/4
    auto phasor = [](float2 bh, float2 bl, bool small, float2 &cm1, float2 &sn1) {
        float2 sn, cs, cm;
        if (small) {
            sincos_small2(neg2(bh), sn, cm);
            cs = __fadd2_rn(cm, f2(1.0f));
        } else {
            sincos_cm2(neg2(bh), sn, cs, cm);
        }
        sn1 = __ffma2_rn(cs, neg2(bl), sn);
        cm1 = __ffma2_rn(sn, bl, cm);
    };
    const bool small = (mc.mwi3_flags & kMwi3SmallB) != 0;  // the same for every thread
    float2 b0l, b1l;
    const float2 b0h = phase(mc.dd_w0, b0l), b1h = phase(mc.dd_w1, b1l);
    float2 DR, DI, KR, KI, cmb, snb;
    phasor(b1h, b1l, small, cmb, snb);
    DR = __ffma2_rn(em1, cmb, __fadd2_rn(em1, cmb));
    DI = __ffma2_rn(em1, snb, snb);
    if (mc.mwi3_flags & kMwi3SmallBK) {
        // e^{-i bK} - 1 = u (2 + u) from u = e^{-i bK/2} - 1
        float2 bkl;
        const float2 bkh = phase(mc.dd_wkh, bkl);
        float2 ur, ui;
        phasor(bkh, bkl, true, ur, ui);
        const float2 ur2 = __fadd2_rn(ur, ur);
        cmb = __ffma2_rn(ur, ur, __ffma2_rn(neg2(ui), ui, ur2));
        snb = __ffma2_rn(ur2, ui, __fadd2_rn(ui, ui));
    } else {
        float2 bkl;
        const float2 bkh = phase(mc.dd_wk, bkl);
        phasor(bkh, bkl, false, cmb, snb);
    }
    KR = __ffma2_rn(emK, cmb, __fadd2_rn(emK, cmb));
    KI = __ffma2_rn(emK, snb, snb);
    // E_0: e^{i phi0} (1 + cm + i sn) = e^{i phi0} + (ce cm - se sn, se cm + ce sn)
    float se, ce;
    sincos_cw(phi0, se, ce);
    phasor(b0h, b0l, small, cmb, snb);
    const float2 c0 = __fadd2_rn(f2(ce), __ffma2_rn(f2(ce), cmb, __fmul2_rn(f2(-se), snb)));
    const float2 s0 = __fadd2_rn(f2(se), __ffma2_rn(f2(se), cmb, __fmul2_rn(f2(ce), snb)));
    auto amp = [](float2 a, float2 aem, float2 c) {
        const float2 p = __fmul2_rn(a, c);
        return __fadd2_rn(p, __ffma2_rn(aem, c, __ffma2_rn(a, c, neg2(p))));
    };
    const float2 A = make_float2(th[0], th[1]);
    const float2 Aem = __fmul2_rn(A, em0);
    float2 X = amp(A, Aem, c0), Y = amp(A, Aem, s0);
    float2 Z = amp(f2(th[2]), f2(th[2] * emE.x), make_float2(ce, se));
    return {X, Y, Z, DR, DI, neg2(DI), KR, KI, neg2(KI), dE, dKE};
}

__device__ __forceinline__ void mwi3_next_anchor(const Mwi3Rec &r, float2 &X, float2 &Y, float2 &Z) {
    const float2 xn = __ffma2_rn(X, r.KR, __ffma2_rn(Y, r.NKI, X));
    Y = __ffma2_rn(Y, r.KR, __ffma2_rn(X, r.KI, Y));
    X = xn;
    Z = __ffma2_rn(Z, f2(r.dKE), Z);
}

// Echoes a .. a+cnt-1 (FULL: cnt = kAnchor) from the block's anchors.
template <bool FULL, class V>
__device__ __forceinline__ void mwi3_block_f(const Mwi3Rec &r, float2 x, float2 y, float2 z, int a, int cnt,
                                             V &visit) {
#pragma unroll
    for (int i = 0; i < kAnchor; ++i) {
        if (FULL || i < cnt) visit(a + i, x.x + x.y + z.x, y.x + y.y + z.y);
        const float2 xn = __ffma2_rn(x, r.DR, __ffma2_rn(y, r.NDI, x));
        y = __ffma2_rn(y, r.DR, __ffma2_rn(x, r.DI, y));
        x = xn;
        z = __ffma2_rn(z, f2(r.dE), z);
    }
}

template <class V>
__device__ __forceinline__ void eval_mwi3_f(const float *th, const ModelConst &mc, V &&visit) {
    const float phi0 = th[8];
    const int n = mc.n_acq;
    if (mc.even) {
        const Mwi3Rec r = mwi3_setup_f(th, mc);
        float2 X = r.X, Y = r.Y, Z = r.Z;
        int a = 0;
        for (; a + kAnchor <= n; a += kAnchor) {
            mwi3_block_f<true>(r, X, Y, Z, a, kAnchor, visit);
            end_block(visit, 0);
            mwi3_next_anchor(r, X, Y, Z);
        }
        if (a < n) mwi3_block_f<false>(r, X, Y, Z, a, n - a, visit);
    } else {
        float rate[3], w[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rate[j] = 1.0f / th[3 + j];
            w[j] = (j < 2) ? kTwoPiMilli * th[6 + j] : 0.0f;
        }
        for (int k0 = 0; k0 < n; k0 += kAnchor) {
            const int k1 = min(k0 + kAnchor, n);
            for (int k = k0; k < k1; ++k) {
                const float t = mc.acq_f[k];
                float re = 0.0f, im = 0.0f;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float m = th[j] * expf(-t * rate[j]);
                    float s, c;
                    sincos_cw(fmaf(-w[j], t, phi0), s, c);
                    re = fmaf(m, c, re);
                    im = fmaf(m, s, im);
                }
                visit(k, re, im);
            }
            end_block(visit, 0);
        }
    }
}

template <bool TAIL, class V>
__device__ __forceinline__ void eval_smt_f(const float *th, const ModelConst &mc, V &&visit) {
    const float f = th[0], da = th[1], dpar = th[2], dperp = th[3];
    const float ddiff = dpar - dperp;
    const int n = mc.n_acq;
    // S(b = 0) = S0 = 1 exactly, by a select (no branch); blocks of kAnchor
    // b-values unrolled, and a protocol of at most kAnchor b-values (one
    // block, the same for every thread) reads them at fixed offsets
    auto one = [&](int k) {
        const float b = mc.acq_f[k];
        const float intra = smt_g_f<TAIL>(b * da, mc);
        const float extra = ex2_approx(-mc.acq_l2e_f[k] * dperp) * smt_g_f<TAIL>(b * ddiff, mc);
        visit(k, b == 0.0f ? 1.0f : fmaf(f, intra, (1.0f - f) * extra));
    };
    if (n <= kAnchor) {
#pragma unroll
        for (int k = 0; k < kAnchor; ++k)
            if (k < n) one(k);
        end_block(visit, 0);
        return;
    }
    for (int k0 = 0; k0 < n; k0 += kAnchor) {
#pragma unroll
        for (int i = 0; i < kAnchor; ++i)
            if (k0 + i < n) one(k0 + i);
        end_block(visit, 0);
    }
}

// The cylinder's Gaussian-phase attenuation (Neuman 1974; van Gelderen et al.
// 1994) is kappa = gamma^2 G^2 R^6 sum_m c_m N_m with
//   N_m = 2 delta q - 2 + 2 e^{-q delta} + 2 e^{-q Delta} - e^{-q (Delta - delta)}
//         - e^{-q (Delta + delta)},   q = x_m^2 Da / R^2,
// which also equals 2 E(a) - e^{-q Delta} H(a) with a = q delta,
// E(a) = e^{-a} - 1 + a and H(a) = e^{a} + e^{-a} - 2.  For a >= 1 the direct
// form loses at most ~3 bits; for a < 1 (wide cylinders, leading terms only)
// E and H come from their Taylor series, whose leading orders would cancel in
// the direct form.
__device__ __forceinline__ float ax_n_direct_f(float q, float dl, float DL) {
    const float A = __expf(-q * dl), B = __expf(-q * DL), C = __expf(-q * (DL - dl));
    return fmaf(2.0f * dl, q, -2.0f) + 2.0f * (A + B) - C - A * B;
}
__device__ __forceinline__ float ax_n_series_f(float q, float dl, float DL) {
    const float a = q * dl, a2 = a * a;
    // E(a) / a^2 = sum_k (-a)^k / (k+2)!, k <= 9 (next term < 3e-9 of the sum)
    float e = fmaf(a, 2.50521084e-8f, -2.75573192e-7f);
    e = fmaf(e, a, 2.75573192e-6f);
    e = fmaf(e, a, -2.48015873e-5f);
    e = fmaf(e, a, 1.98412698e-4f);
    e = fmaf(e, a, -1.38888889e-3f);
    e = fmaf(e, a, 8.33333333e-3f);
    e = fmaf(e, a, -4.16666667e-2f);
    e = fmaf(e, a, 1.66666667e-1f);
    e = fmaf(e, -a, 0.5f);
    // H(a) / a^2 = sum_k 2 a^(2k) / (2k+2)!, k <= 4 (next term < 5e-9)
    float h = fmaf(a2, 5.51146384e-7f, 4.96031746e-5f);
    h = fmaf(h, a2, 2.77777778e-3f);
    h = fmaf(h, a2, 8.33333333e-2f);
    h = fmaf(h, a2, 1.0f);
    return a2 * fmaf(2.0f, e, -__expf(-q * DL) * h);
}

// phi_j(R) = R^6 sum_m c_m N_m for every timing j, summed term by term.
__device__ __forceinline__ void ax_phi_series_f(float R, const AxConst &ax, float (&phi)[kAxMaxTiming]) {
    const float R2 = R * R, inv_r2 = 1.0f / R2, r6 = R2 * R2 * R2;
#pragma unroll
    for (int j = 0; j < kAxMaxTiming; ++j) {
        phi[j] = 0.0f;
        if (j < ax.n_timing) {  // the same for every thread
            const float dl = ax.delta_f[j], DL = ax.Delta_f[j];
            float acc = 0.0f;
            int m = 0;
            for (; m < ax.careful_f; ++m) {
                const float q = ax.x2d_f[m] * inv_r2;
                const float n = (q * dl < 1.0f) ? ax_n_series_f(q, dl, DL) : ax_n_direct_f(q, dl, DL);
                acc = fmaf(ax.c_f[m], n, acc);
            }
            for (; m < ax.terms_f; ++m) acc = fmaf(ax.c_f[m], ax_n_direct_f(ax.x2d_f[m] * inv_r2, dl, DL), acc);
            phi[j] = acc * r6;
        }
    }
}

// The same from the shared-memory table: interval rint(t) of t = log2 R *
// tab_inv_w + tab_off (clamped, so every load stays in the table), Horner in
// d = t - interval.
__device__ __forceinline__ void ax_phi_table_f(float R, const AxConst &ax, float (&phi)[kAxMaxTiming]) {
    constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
    const float t = fmaf(log2f(R), ax.tab_inv_w, ax.tab_off);  // once per evaluation: the accurate log2
    int i = static_cast<int>((t + kRound) - kRound);
    i = min(max(i, 0), ax.tab_n - 1);
    const float d = t - static_cast<float>(i);
#pragma unroll
    for (int j = 0; j < kAxMaxTiming; ++j) {
        phi[j] = 0.0f;
        if (j < ax.n_timing) {
            const float4 lo = ax_tab_s[(2 * j) * kAxTabMax + i];
            const float4 hi = ax_tab_s[(2 * j + 1) * kAxTabMax + i];
            float p = fmaf(hi.w, d, hi.z);
            p = fmaf(p, d, hi.y);
            p = fmaf(p, d, hi.x);
            p = fmaf(p, d, lo.w);
            p = fmaf(p, d, lo.z);
            p = fmaf(p, d, lo.y);
            phi[j] = fmaf(p, d, lo.x);
        }
    }
}

// Measurements in timing order, so that the timing's attenuation phi_j is a
// loop constant; per measurement two 16-byte shared-memory loads bring
// b Da, g2, g2 log2 e, b log2 e, b, e^{-b D_csf} and the measurement's index.
template <bool TAIL, class V>
__device__ __forceinline__ void eval_axcal_f(const float *th, const ModelConst &mc, V &&visit) {
    const AxConst &ax = mc.ax;
    const float R = 0.5f * th[0], fn = th[1], fcsf = th[2], der = th[3];
    float phi[kAxMaxTiming];
    if (ax.tab_n > 0) ax_phi_table_f(R, ax, phi);  // the same branch for every thread
    else ax_phi_series_f(R, ax, phi);
    const float w_r = (1.0f - fcsf) * fn, w_h = (1.0f - fcsf) * (1.0f - fn), dh = kAxDePar - der;
    for (int j = 0; j < ax.n_timing; ++j) {
        const float nph = -(j == 0 ? phi[0] : (j == 1 ? phi[1] : (j == 2 ? phi[2] : phi[3])));
        const int end = ax.first[j + 1];
        for (int i0 = ax.first[j]; i0 < end; i0 += kAnchor) {
            const int i1 = min(i0 + kAnchor, end);
            for (int i = i0; i < i1; ++i) {
                const float4 A = ax_meas_s[2 * i], B = ax_meas_s[2 * i + 1];
                // restricted: e^{-kappa} g(b Da - kappa), kappa = g2 phi_j
                const float sr = ex2_approx(A.z * nph) * smt_g_f<TAIL>(fmaf(A.y, nph, A.x), mc);
                // hindered: e^{-b De_R} g(b (De_par - De_R))
                const float sh = ex2_approx(-A.w * der) * smt_g_f<TAIL>(B.x * dh, mc);
                visit(__float_as_int(B.z), fmaf(w_r, sr, fmaf(w_h, sh, fcsf * B.y)));
            }
            end_block(visit, 0);
        }
    }
}

template <class V>
__device__ __forceinline__ void eval_linear_f(const float *th, const ModelConst &mc, V &&visit) {
    for (int k = 0; k < mc.n_acq; ++k) visit(k, fmaf(th[1], mc.acq_f[k], th[0]));
}

// ----------------------------------------------------------- FP64 models --
template <class V>
__device__ __forceinline__ void eval_monoexp_d(const double *th, const ModelConst &mc, V &&visit) {
    for (int k = 0; k < mc.n_acq; ++k) visit(k, th[0] * exp(-th[1] * mc.acq_d[k] * 1e-3));
}

template <class V>
__device__ __forceinline__ void eval_mwi3_d(const double *th, const ModelConst &mc, V &&visit) {
    for (int k = 0; k < mc.n_acq; ++k) {
        const double t = mc.acq_d[k];
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double m = th[j] * exp(-t / th[3 + j]);
            const double df = (j < 2) ? th[6 + j] : 0.0;
            double s, c;
            sincos(th[8] - kTwoPiMilliD * df * t, &s, &c);
            re += m * c;
            im += m * s;
        }
        visit(k, re, im);
    }
}

template <class V>
__device__ __forceinline__ void eval_smt_d(const double *th, const ModelConst &mc, V &&visit) {
    for (int k = 0; k < mc.n_acq; ++k) {
        const double b = mc.acq_d[k];
        const double intra = smt_g_d(b * th[1]);
        const double extra = exp(-b * th[3]) * smt_g_d(b * (th[2] - th[3]));
        visit(k, th[0] * intra + (1.0 - th[0]) * extra);
    }
}

template <class V>
__device__ __forceinline__ void eval_axcal_d(const double *th, const ModelConst &mc, V &&visit) {
    const AxConst &ax = mc.ax;
    const double R = 0.5 * th[0], fn = th[1], fcsf = th[2], der = th[3];
    const double R2 = R * R, r6 = R2 * R2 * R2;
    double phi[kAxMaxTiming];
#pragma unroll
    for (int j = 0; j < kAxMaxTiming; ++j) {
        phi[j] = 0.0;
        if (j < ax.n_timing) {
            const double dl = ax.delta_d[j], DL = ax.Delta_d[j];
            double acc = 0.0;
            for (int m = 0; m < ax.terms_d; ++m) {
                const double q = ax.x2d_d[m] / R2, a = q * dl;
                double n;
                if (a < 1.0) {  // 2 E(a) - e^{-q Delta} H(a) (see ax_n_series_f)
                    const double em = expm1(-a), ep = expm1(a);
                    n = 2.0 * (em + a) - exp(-q * DL) * (ep + em);
                } else {
                    const double A = exp(-a), B = exp(-q * DL), C = exp(-q * (DL - dl));
                    n = 2.0 * a - 2.0 + 2.0 * (A + B) - C - A * B;
                }
                acc += ax.c_d[m] * n;
            }
            phi[j] = acc * r6;
        }
    }
    for (int k = 0; k < mc.n_meas; ++k) {
        const double b = ax.b_d[k];
        const int t = ax.t[k];
        const double ph = t == 0 ? phi[0] : (t == 1 ? phi[1] : (t == 2 ? phi[2] : phi[3]));
        const double kap = ax.g2_d[k] * ph;
        const double sr = exp(-kap) * smt_g_d(b * kAxDaD - kap);
        const double sh = exp(-b * der) * smt_g_d(b * (kAxDeParD - der));
        visit(k, (1.0 - fcsf) * (fn * sr + (1.0 - fn) * sh) + fcsf * ax.csf_d[k]);
    }
}

template <class V>
__device__ __forceinline__ void eval_linear_d(const double *th, const ModelConst &mc, V &&visit) {
    for (int k = 0; k < mc.n_acq; ++k) visit(k, th[0] + th[1] * mc.acq_d[k]);
}

// --------------------------------------------------------- dispatch by kind
template <int KIND, class V>
__device__ __forceinline__ void eval_f(const float *th, const ModelConst &mc, V &&visit) {
    if constexpr (KIND == GAC_MODEL_MONOEXP) eval_monoexp_f(th, mc, visit);
    else if constexpr (KIND == GAC_MODEL_MWI3) eval_mwi3_f(th, mc, visit);
    else if constexpr (KIND == GAC_MODEL_SMT) {
        if (mc.gtab_tail) eval_smt_f<true>(th, mc, visit);  // the same branch for every thread
        else eval_smt_f<false>(th, mc, visit);
    } else if constexpr (KIND == GAC_MODEL_AXCAL_SMT) {
        if (mc.gtab_tail) eval_axcal_f<true>(th, mc, visit);
        else eval_axcal_f<false>(th, mc, visit);
    }
    else eval_linear_f(th, mc, visit);
}

template <int KIND, class V>
__device__ __forceinline__ void eval_d(const double *th, const ModelConst &mc, V &&visit) {
    if constexpr (KIND == GAC_MODEL_MONOEXP) eval_monoexp_d(th, mc, visit);
    else if constexpr (KIND == GAC_MODEL_MWI3) eval_mwi3_d(th, mc, visit);
    else if constexpr (KIND == GAC_MODEL_SMT) eval_smt_d(th, mc, visit);
    else if constexpr (KIND == GAC_MODEL_AXCAL_SMT) eval_axcal_d(th, mc, visit);
    else eval_linear_d(th, mc, visit);
}

// ----------------------------------------------------- likelihood sums -----
// Kahan-compensated FP32 sum (MIXED path).
// Sums of squared residuals.  Complex rows feed (d_re, d_im) pairs, squared
// and accumulated lane-wise by one paired FMA; real rows feed single
// residuals.  The models call block_end() after each block of echoes of
// their recurrences (end_block below).
//
// MIXED: plain FP32 inside a block of kAnchor acquisitions (at most
// 2 kAnchor terms), the block sums added with Kahan's compensation.
struct KahanSum {
    float2 p = make_float2(0.0f, 0.0f);
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add2(float2 d) { p = __ffma2_rn(d, d, p); }
    __device__ __forceinline__ void add(float d) { p.x = fmaf(d, d, p.x); }
    __device__ __forceinline__ void block_end() {
        const float y = (p.x + p.y) - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
        p = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ float value() {
        block_end();
        return s;
    }
};
// FP32: one plain FP32 sum per lane.
struct PlainSumF {
    float2 p = make_float2(0.0f, 0.0f);
    __device__ __forceinline__ void add2(float2 d) { p = __ffma2_rn(d, d, p); }
    __device__ __forceinline__ void add(float d) { p.x = fmaf(d, d, p.x); }
    __device__ __forceinline__ void block_end() {}
    __device__ __forceinline__ float value() const { return p.x + p.y; }
};
struct PlainSumD {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// -1/2 * sum_m (y_m - s_m)^2 / sigma^2, with y read from `y` (row of the
// voxel; complex rows as re, im pairs).  ACC = KahanSum or PlainSumF.
template <class ACC>
struct ResidualVisitor {
    ACC &acc;
    const float *y;
    __device__ __forceinline__ void operator()(int k, float sr, float si) const {
        const float2 yk = reinterpret_cast<const float2 *>(y)[k];
        acc.add2(__ffma2_rn(make_float2(sr, si), f2(-1.0f), yk));  // y - s, both parts
    }
    __device__ __forceinline__ void operator()(int k, float s) const { acc.add(__fsub_rn(y[k], s)); }
    __device__ __forceinline__ void block_end() const { acc.block_end(); }
};

template <int KIND, class ACC>
__device__ __forceinline__ float loglik_f(const float *th, const float *y, float inv_s2,
                                          const ModelConst &mc) {
    ACC acc;
    eval_f<KIND>(th, mc, ResidualVisitor<ACC>{acc, y});
    return -0.5f * acc.value() * inv_s2;
}

template <int KIND>
__device__ __forceinline__ double loglik_d(const double *th, const float *y, double inv_s2,
                                           const ModelConst &mc) {
    PlainSumD acc;
    if constexpr (model_complex(KIND)) {
        eval_d<KIND>(th, mc, [&](int k, double sr, double si) {
            const double dr = static_cast<double>(y[2 * k]) - sr;
            const double di = static_cast<double>(y[2 * k + 1]) - si;
            acc.add(dr * dr + di * di);
        });
    } else {
        eval_d<KIND>(th, mc, [&](int k, double s) {
            const double d = static_cast<double>(y[k]) - s;
            acc.add(d * d);
        });
    }
    return -0.5 * acc.value() * inv_s2;
}

}  // namespace gac
