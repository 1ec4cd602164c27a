// Persistent Metropolis-Hastings kernels (mcmc.m hot path, Sec. 2.2.2).
//
// One thread owns one (voxel, chain): a block holds VB = floor(256 / C)
// voxels x C chains (chain fastest).  For a tile of voxels and an iteration
// range (t_begin, t_end] the block
//   a1  stages the voxels' measurements in shared memory (coalesced 16-byte
//       global loads, odd row stride so that the lanes of a warp hit
//       distinct banks), then every thread
//   a2  draws or loads its initial state and evaluates its likelihood
//       (or, when resuming a slice, reloads theta, L and its counters),
//   a3  per iteration draws Philox words for (t, voxel, chain),
//   a4  proposes theta' = clamp(theta + step * z, lb, ub) (step scaled by
//       2^(e/4) when burn-in adaptation is on; e changes at window ends),
//   a5  evaluates the forward model at every acquisition and
//   a6  accumulates the Gaussian log-likelihood in registers,
//   a7  accepts iff log u < L' - L,
//   a8  on the thinning grid stores the state (coalesced over voxels) and
//       updates Welford accumulators,
// and after the last iteration
//   a9  pools the C chains' accumulators of each voxel (Chan et al.'s
//       update for equal counts, one parameter per thread) and writes mean, SD, R-hat,
//       acceptance rate, the non-finite count and the step multiplier.
// Nothing but thinned samples touches HBM inside the iteration loop.
//
// Two drivers share this tile routine: mh_kernel runs one job in one launch
// (t in (0, I], Welford accumulators in shared memory, nothing saved), and
// the serving kernel runs slices of many jobs (chain state and Welford
// accumulators in HBM between slices; resuming from them reproduces an
// uninterrupted run, because the random numbers depend only on (seed, t,
// voxel, chain)).
//
// Precision variants (template PREC):
//   MIXED  FP32 model and residuals, FP32 block sums of six acquisitions
//          added with Kahan's compensation, acceptance with
//          FP64 semantics (an FP32 test with a proven error margin decides
//          almost every step; steps inside the margin are decided in FP64
//          from the same L, L' and acceptance word), FP64 Welford.
//   FP32   FP32 everywhere (plain sum, FP32 decision, FP32 Welford).
//   FP64   FP64 everywhere.
#pragma once
#include <climits>
#include <cmath>
#include <cstdint>

#include "gac.h"
#include "models.cuh"
#include "philox.cuh"

namespace gac {

constexpr int kBlock = 256;
// Blocks per SM each kernel is compiled for (a register cap): the 3-pool
// model needs ~118 registers (2 blocks of 256); AxCaliberSMT spills under the
// 3-block cap of 80 registers and runs 8% faster at 2 blocks; SMT and the
// lighter models fit 3 blocks; FP64 paths are left uncapped.
template <int KIND, int PREC>
constexpr int mh_min_blocks() {
    return PREC == GAC_PREC_FP64 ? 1 : ((KIND == GAC_MODEL_MWI3 || KIND == GAC_MODEL_AXCAL_SMT) ? 2 : 3);
}

// The one-launch kernel's own block size and blocks per SM (the serving and
// allocation-free kernels always run blocks of kBlock).  Measured on the
// 3-pool MIXED kernel: blocks of 128 threads, 5 or 6 per SM (20 or 24 warps),
// ran 3% slower than 2 blocks of 256, so every kind keeps kBlock.
template <int KIND, int PREC>
__host__ __device__ constexpr int mh_block() {
    return kBlock;
}
template <int KIND, int PREC>
constexpr int mh_launch_min_blocks() {
    return mh_block<KIND, PREC>() == kBlock ? mh_min_blocks<KIND, PREC>() : 5;
}

struct RunArgs {
    const float *data;   // [N][M]
    const float *sigma;  // [N] or nullptr
    float sigma_scalar;
    const float *x0;     // [N][C][P] or nullptr
    double *mean;        // [P][N]
    double *std;         // [P][N]
    float *samples;      // [S][C][P][N]
    float *accept;       // [C][N]
    int32_t *nonfinite;  // [C][N]
    gac_trace_rec *trace;  // [trace_n][C][I]
    int64_t n_vox;
    int C, I, B, T, S;
    uint32_t k0, k1;     // Philox key (seed lo, hi)
    uint64_t voxel_base;
    int moments_mode;
    int trace_n;
    int vox_per_block;   // VB
    int row_stride;      // shared-memory floats per voxel row (padded)
    int data_vec4;       // rows are whole float4s and data is 16-byte aligned
    int64_t n_tiles;
    // burn-in step adaptation: window W (0 = off); e rises when a window's
    // acceptances a > adapt_hi (= floor(target W)), falls when a < adapt_lo
    // (= ceil(target W))
    int adapt_window, adapt_lo, adapt_hi;
    double *rhat;        // [P][N] or nullptr
    float *step_scale;   // [C][N] or nullptr
};

// Chain state kept in HBM between slices, structure of arrays over the
// N*C chains (index v*C + c, so a warp's accesses are contiguous).
struct SliceState {
    void *theta;     // [P][N*C] of R
    void *L;         // [N*C] of R
    int32_t *n_acc;  // [N*C]
    int32_t *n_bad;  // [N*C]
    void *wf_mean;   // [P][N*C] of W
    void *wf_m2;     // [P][N*C] of W
    int32_t *adapt;  // [2][N*C]: adaptation exponent e, accepted count at the window start
    float *blk;      // [3P][N*C]: MIXED all-post-burn-in block partials (sum d, sum d^2, reference)
};

// 1/n for the FP64 Welford updates, n < kInvN: a load (one address per warp,
// through the read-only cache) instead of an FP64 division, whose several
// FP64 instructions each hold a GB300 sub-partition's FP64 pipe for ~76
// cycles (1.68 FP64 results per SM clock).  The table is computed at compile
// time with IEEE division, so it holds exactly what the division returns; it
// lives in global memory (in the constant bank its 32 KB crowded out the
// kernel parameters the iteration loop reads: 1.5% slower).
constexpr int kInvN = 4096;
struct InvTable {
    double v[kInvN];
};
constexpr InvTable make_inv_table() {
    InvTable t{};
    for (int i = 1; i < kInvN; ++i) t.v[i] = 1.0 / static_cast<double>(i);
    return t;
}
static __device__ InvTable g_inv_n = make_inv_table();

// The Welford update's multiply-adds, written as explicit FMAs so that every
// kernel that accumulates moments rounds them the same way.
__device__ __forceinline__ double welford_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float welford_fma(float a, float b, float c) { return fmaf(a, b, c); }

// TABLE: from g_inv_n (the lane-split kernel, where the division's FP64
// latency is exposed); otherwise the division itself (the one-thread kernel,
// whose loop measured 1.5% faster without the table's load).  Equal values.
template <class W, bool TABLE = false>
__device__ __forceinline__ W inv_count(int n) {
    if constexpr (sizeof(W) == 8 && TABLE) return n < kInvN ? __ldg(&g_inv_n.v[n]) : 1.0 / static_cast<double>(n);
    else return W(1) / W(n);
}

// MIXED path, moments over every post-burn-in state: the states of blocks of
// kMomBlock consecutive post-burn-in iterations (aligned to t - B = 0, so the
// blocks do not depend on slicing) are summed in FP32 as deviations d = x -
// x_ref from the block's first state; each full block, and the last partial
// one, is merged into the FP64 Welford state with Chan et al.'s pairwise
// formula.  One FP64 merge per block instead of an FP64 update per iteration:
// FP64 issues at 1/73 of the FP32 rate on this part.
constexpr int kMomBlock = 64;

// Host: the adaptation fields of RunArgs.  a > target W <=> a > floor(target W)
// and a < target W <=> a < ceil(target W) for integer a.
inline void set_adaptation(RunArgs &ra, const gac_mcmc_opts *o) {
    ra.adapt_window = o->adapt_window;
    const double x = o->adapt_target * static_cast<double>(o->adapt_window);
    ra.adapt_lo = o->adapt_window > 0 ? static_cast<int>(std::ceil(x)) : 0;
    ra.adapt_hi = o->adapt_window > 0 ? static_cast<int>(std::floor(x)) : 0;
}

// Step multiplier s = 2^(e/4) of the adaptation, as the Box-Muller radius
// factor k: -2 s^2 = -2^(e/2 + 1) against ln u (FP64), times ln 2 against
// log2 u (FP32).
template <class R>
__device__ __forceinline__ R adapt_bm_scale(int e) {
    if constexpr (sizeof(R) == 8) return -exp2(0.5 * e + 1.0);
    else return exp2f(0.5f * static_cast<float>(e)) * kNeg2Ln2;
}

template <int PREC>
struct PrecTraits;
template <>
struct PrecTraits<GAC_PREC_MIXED> {
    using R = float;   // state, model
    using W = double;  // Welford accumulators
    using Acc = KahanSum;
};
template <>
struct PrecTraits<GAC_PREC_FP32> {
    using R = float;
    using W = float;
    using Acc = PlainSumF;
};
template <>
struct PrecTraits<GAC_PREC_FP64> {
    using R = double;
    using W = double;
    using Acc = PlainSumD;
};

template <int KIND, int PREC>
__device__ __forceinline__ typename PrecTraits<PREC>::R loglik_any(
    const typename PrecTraits<PREC>::R *th, const float *y, typename PrecTraits<PREC>::R inv_s2,
    const ModelConst &mc) {
    if constexpr (PREC == GAC_PREC_FP64) return loglik_d<KIND>(th, y, inv_s2, mc);
    else return loglik_f<KIND, typename PrecTraits<PREC>::Acc>(th, y, inv_s2, mc);
}

// MIXED acceptance, FP64 semantics at FP32 cost, from lu32 = __logf(u01_f(w)).
// Error of the FP32 quantities against their FP64 counterparts:
//   d32 = Lp - L:        one rounding of the exact difference of two floats,
//                        <= 2^-24 |Lp - L|;
//   lu32 = __logf(u32):  <= 2^-21.41 absolute on [0.5, 2], 3 ulp otherwise
//                        (|ln u| <= 22.2 -> < 6e-6), plus 2^-24 from
//                        rounding u to float.
// A margin of 1e-5 + 2^-22 |d32| covers both (with room for the rounding of
// the gap itself); inside it the decision is recomputed in FP64 from the same
// L, Lp and word.  NaN lands in the FP64 branch and rejects.  The wider
// margin 1e-5 + 2^-20 (|L| + |Lp|) (WIDE) is valid too, as |d32| <= |L| +
// |Lp|; it grows far from the posterior, where both are large and their
// difference is not, so the lane-split kernel, whose FP64 latency nothing
// hides, takes the tight one, and the one-thread kernel the wide one (its
// loop measured 1.2% faster so).  The decision is the FP64 one either way.
template <bool WIDE = false>
__device__ __forceinline__ bool accept_mixed(float Lp, float L, float lu32, uint32_t w) {
    const float d32 = Lp - L;
    const float margin = WIDE ? 1e-5f + 0x1p-20f * (fabsf(L) + fabsf(Lp)) : fmaf(0x1p-22f, fabsf(d32), 1e-5f);
    const float gap = d32 - lu32;
    if (fabsf(gap) > margin) return gap > 0.0f;
    return log(u01_d(w)) < static_cast<double>(Lp) - static_cast<double>(L);
}

// Acceptance: log u < Lp - L.
template <int PREC>
__device__ __forceinline__ bool accept_step(typename PrecTraits<PREC>::R Lp,
                                            typename PrecTraits<PREC>::R L, uint32_t w) {
    if constexpr (PREC == GAC_PREC_FP64) {
        return log(u01_d(w)) < Lp - L;
    } else if constexpr (PREC == GAC_PREC_FP32) {
        return logf(u01_f(w)) < Lp - L;
    } else {
        // FP64 semantics at FP32 cost (accept_mixed).
        return accept_mixed<true>(Lp, L, __logf(u01_f(w)), w);
    }
}

// Shared-memory bytes of one block: Welford accumulators (one-launch driver
// only) + the measurement tile + the MIXED all-post-burn-in block partials
// ([3P][block] floats, when blocked_moments), for blocks of `block` threads.
__host__ __device__ inline size_t tile_smem_bytes(int P, size_t w_bytes, int VB, int row_stride,
                                                  bool welford_in_smem, bool blocked_moments = false,
                                                  int block = kBlock) {
    return (welford_in_smem ? 2 * static_cast<size_t>(P) * block * w_bytes : 0) +
           static_cast<size_t>(VB) * row_stride * sizeof(float) +
           (blocked_moments ? 3 * static_cast<size_t>(P) * block * sizeof(float) : 0);
}

// Pools one parameter of C chains that each hold n values, from their
// Welford means and sums of squared deviations (mean_k[k], m2_k[k]): with
// equal counts the pooled mean is the mean of the chain means, and the pooled
// sum of squares is sum_k M2_k + n sum_k (mean_k - mean)^2 (Chan et al.'s
// update, applied to all chains at once).  Writes the mean and the SD (n-1
// divisor; NaN for no values, 0 for one) and R-hat: W = mean within-chain
// variance, B/n = variance of the chain means, R-hat = sqrt(((n-1)/n W +
// B/n) / W), NaN for C < 2 or n < 2.  Any output may be nullptr.  FP64.
template <class W>
__device__ __forceinline__ void pool_chains(const W *mean_k, const W *m2_k, int C, int n, double *mean_out,
                                            double *sd_out, double *rhat_out) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    double mu = 0.0;
    for (int k = 0; k < C; ++k) mu += static_cast<double>(mean_k[k]);
    mu /= C;
    double ss_within = 0.0, ss_between = 0.0;
    for (int k = 0; k < C; ++k) {
        const double d = static_cast<double>(mean_k[k]) - mu;
        ss_within += static_cast<double>(m2_k[k]);
        ss_between += d * d;
    }
    const double n_all = static_cast<double>(C) * n;
    if (mean_out) *mean_out = n > 0 ? mu : nan;
    if (sd_out) *sd_out = n_all > 1 ? sqrt((ss_within + n * ss_between) / (n_all - 1.0)) : (n_all == 1 ? 0.0 : nan);
    if (rhat_out) {
        double r = nan;
        if (C >= 2 && n >= 2) {
            const double w_in = ss_within / (static_cast<double>(C) * (n - 1));
            const double b_n = ss_between / (C - 1);
            r = sqrt(((n - 1.0) / n * w_in + b_n) / w_in);
        }
        *rhat_out = r;
    }
}

// Runs iterations t_begin+1 .. t_end of the chains of one tile of voxels.
// SLICED = false: t_begin = 0, t_end = I, Welford accumulators in shared
// memory at the start of `smem`; SLICED = true: chain state and accumulators
// in `ss` (HBM).
template <int KIND, int PREC, bool TRACE, bool SLICED, int BLK = kBlock>
__device__ __forceinline__ void run_tile(const ModelConst &mc, const RunArgs &ra,
                                         const SliceState &ss, int64_t tile, int t_begin,
                                         int t_end, unsigned char *smem) {
    using R = typename PrecTraits<PREC>::R;
    using W = typename PrecTraits<PREC>::W;
    constexpr int P = model_n_par(KIND);
    constexpr int NW = n_words(P);
    constexpr int NWA = 4 * n_calls(P);

    const int tid = threadIdx.x;
    const int C = ra.C;
    const int VB = ra.vox_per_block;
    const int M = mc.n_meas;
    const int lv = tid / C;
    const int c = tid - lv * C;
    const bool lane_used = tid < VB * C;

    const int64_t v0 = tile * VB;
    const int64_t nchains = ra.n_vox * C;
    W *wf_mean;
    W *wf_m2;
    int64_t wf_stride, wf_idx;
    float *ytile;
    if constexpr (SLICED) {
        wf_mean = static_cast<W *>(ss.wf_mean);
        wf_m2 = static_cast<W *>(ss.wf_m2);
        wf_stride = nchains;
        wf_idx = v0 * C + tid;
        ytile = reinterpret_cast<float *>(smem);
    } else {
        wf_mean = reinterpret_cast<W *>(smem);
        wf_m2 = wf_mean + P * BLK;
        wf_stride = BLK;
        wf_idx = tid;
        ytile = reinterpret_cast<float *>(wf_m2 + P * BLK);
    }

    const int64_t left = ra.n_vox - v0;
    const int nv = left < VB ? static_cast<int>(left) : VB;
    // MIXED all-post-burn-in block partials: s1 [P][BLK], s2, reference
    float *const bs = ytile + VB * ra.row_stride;

    // a1: stage measurements of voxels [v0, v0 + nv) (and the model's
    // table) in shared memory
    __syncthreads();
    model_smem_load<KIND>(mc);
    {
        const float *src = ra.data + v0 * M;
        const int total = nv * M;
        if (ra.data_vec4) {
            const float4 *src4 = reinterpret_cast<const float4 *>(src);
            for (int i = tid; i < total / 4; i += BLK) {
                const float4 q = __ldg(src4 + i);
                const int e = 4 * i, row = e / M, col = e - row * M;
                float *dst = ytile + row * ra.row_stride + col;
                dst[0] = q.x;
                dst[1] = q.y;
                dst[2] = q.z;
                dst[3] = q.w;
            }
        } else {
            for (int i = tid; i < total; i += BLK) {
                const int row = i / M, col = i - row * M;
                ytile[row * ra.row_stride + col] = __ldg(src + i);
            }
        }
    }
    __syncthreads();

    const bool active = lane_used && lv < nv;
    const int64_t v = v0 + lv;
    const int64_t ch = v * C + c;  // chain index in [0, N*C)
    if (active) {
        const float *y = ytile + lv * ra.row_stride;
        const float sig = ra.sigma ? __ldg(ra.sigma + v) : ra.sigma_scalar;
        const R inv_s2 = R(1) / (R(sig) * R(sig));
        const uint32_t vg = static_cast<uint32_t>(ra.voxel_base + static_cast<uint64_t>(v));
        const uint32_t cu = static_cast<uint32_t>(c);

        // a2: initial state, or the state saved by the previous slice
        R th[P];
        R L;
        int n_acc = 0, n_bad = 0;
        int ad_e = 0, ad_acc0 = 0;  // adaptation exponent, n_acc at the window start
        if (SLICED && t_begin > 0) {
#pragma unroll
            for (int p = 0; p < P; ++p) th[p] = static_cast<const R *>(ss.theta)[p * nchains + ch];
            L = static_cast<const R *>(ss.L)[ch];
            n_acc = ss.n_acc[ch];
            n_bad = ss.n_bad[ch];
            ad_e = ss.adapt[ch];
            ad_acc0 = ss.adapt[nchains + ch];
        } else {
            if (ra.x0) {
                const float *x0 = ra.x0 + ch * P;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if constexpr (PREC == GAC_PREC_FP64)
                        th[p] = fmin(fmax(static_cast<double>(x0[p]), mc.lb_d[p]), mc.ub_d[p]);
                    else
                        th[p] = fminf(fmaxf(x0[p], mc.lb_f[p]), mc.ub_f[p]);
                }
            } else {
                uint32_t w0[4 * ((P + 3) / 4)];
                draw_words(w0, kInitIteration, vg, cu, ra.k0, ra.k1);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    if constexpr (PREC == GAC_PREC_FP64)
                        th[p] = mc.lb_d[p] + (mc.ub_d[p] - mc.lb_d[p]) * u01_d(w0[p]);
                    else
                        th[p] = fmaf(mc.ub_f[p] - mc.lb_f[p], u01_f(w0[p]), mc.lb_f[p]);
                }
            }
            L = loglik_any<KIND, PREC>(th, y, inv_s2, mc);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                wf_mean[p * wf_stride + wf_idx] = W(0);
                wf_m2[p * wf_stride + wf_idx] = W(0);
            }
        }

        // moments taken so far, and the next iteration on the thinning grid
        const bool all_mode = ra.moments_mode == GAC_MOMENTS_ALL_POSTBURNIN;
        int n_mom = all_mode ? max(t_begin - ra.B, 0) : (t_begin > ra.B ? (t_begin - ra.B) / ra.T : 0);
        // blocked accumulation (MIXED, all states): states in the open block,
        // n_mom = states already merged into the FP64 Welford state
        constexpr bool kBlocked = PREC == GAC_PREC_MIXED;
        int blk_n = 0;
        if constexpr (kBlocked) {
            if (all_mode) {
                blk_n = n_mom % kMomBlock;
                n_mom -= blk_n;
                if constexpr (SLICED) {
                    if (blk_n > 0)
                        for (int k = 0; k < 3 * P; ++k) bs[k * BLK + tid] = ss.blk[k * nchains + ch];
                }
            }
        }
        int to_thin = t_begin < ra.B ? ra.B + ra.T : ra.B + ((t_begin - ra.B) / ra.T + 1) * ra.T;
        // next window end of the burn-in adaptation (INT_MAX: none left)
        const int W_ad = ra.adapt_window;
        int to_adapt = INT_MAX;
        if (W_ad > 0 && (t_begin / W_ad + 1) <= ra.B / W_ad) to_adapt = (t_begin / W_ad + 1) * W_ad;
        R bm_k = adapt_bm_scale<R>(ad_e);

        // iterations run in segments that end at the adaptation windows, so
        // the loop itself carries no adaptation test
        for (int t_seg = t_begin; t_seg < t_end;) {
            const int seg_end = to_adapt < t_end ? to_adapt : t_end;
            for (int t = t_seg + 1; t <= seg_end; ++t) {
                // a3: random words for (t, voxel, chain)
                uint32_t w[NWA];
                draw_words(w, static_cast<uint32_t>(t), vg, cu, ra.k0, ra.k1);
                // a4: proposal
                R prop[P];
#pragma unroll
                for (int j = 0; 2 * j < P; ++j) {
                    R z0, z1;
                    if constexpr (PREC == GAC_PREC_FP64) box_muller_d(w[2 * j], w[2 * j + 1], z0, z1, bm_k);
                    else box_muller_f(w[2 * j], w[2 * j + 1], z0, z1, bm_k);
                    if constexpr (PREC == GAC_PREC_FP64) {
                        prop[2 * j] = fmin(fmax(fma(mc.step_d[2 * j], z0, th[2 * j]), mc.lb_d[2 * j]),
                                           mc.ub_d[2 * j]);
                        if (2 * j + 1 < P)
                            prop[2 * j + 1] = fmin(fmax(fma(mc.step_d[2 * j + 1], z1, th[2 * j + 1]),
                                                        mc.lb_d[2 * j + 1]), mc.ub_d[2 * j + 1]);
                    } else {
                        prop[2 * j] = fminf(fmaxf(fmaf(mc.step_f[2 * j], z0, th[2 * j]), mc.lb_f[2 * j]),
                                            mc.ub_f[2 * j]);
                        if (2 * j + 1 < P)
                            prop[2 * j + 1] = fminf(fmaxf(fmaf(mc.step_f[2 * j + 1], z1, th[2 * j + 1]),
                                                          mc.lb_f[2 * j + 1]), mc.ub_f[2 * j + 1]);
                    }
                }
                // a5 + a6: forward model and likelihood
                const R Lp = loglik_any<KIND, PREC>(prop, y, inv_s2, mc);
                // a7: accept / reject
                const uint32_t w_acc = w[NW - 1];
                const bool acc = accept_step<PREC>(Lp, L, w_acc);
                n_bad += !isfinite(Lp);
                if constexpr (TRACE) {
                    if (v < ra.trace_n) {
                        gac_trace_rec *rec = ra.trace + ch * static_cast<int64_t>(ra.I) + (t - 1);
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            rec->theta[p] = static_cast<double>(th[p]);
                            rec->prop[p] = static_cast<double>(prop[p]);
                        }
                        rec->L = static_cast<double>(L);
                        rec->Lp = static_cast<double>(Lp);
                        rec->w_acc = w_acc;
                        rec->accepted = acc ? 1 : 0;
                    }
                }
                if (acc) {
#pragma unroll
                    for (int p = 0; p < P; ++p) th[p] = prop[p];
                    L = Lp;
                    ++n_acc;
                }
                // a8: thinning grid t = B + T, B + 2T, ... and moments
                const bool on_grid = (t == to_thin);
                if (on_grid) {
                    to_thin += ra.T;
                    if (ra.samples) {
                        const int s = (t - ra.B) / ra.T - 1;
                        float *dst = ra.samples + ((static_cast<int64_t>(s) * C + c) * P) * ra.n_vox + v;
#pragma unroll
                        for (int p = 0; p < P; ++p) dst[p * ra.n_vox] = static_cast<float>(th[p]);
                    }
                }
                if (kBlocked && all_mode) {
                    if (t > ra.B) {
                        float *s1 = bs + tid, *s2 = bs + P * BLK + tid, *ref = bs + 2 * P * BLK + tid;
                        if (blk_n == 0) {  // a block's first state is its reference (the same t for every thread)
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                ref[p * BLK] = static_cast<float>(th[p]);
                                s1[p * BLK] = 0.0f;
                                s2[p * BLK] = 0.0f;
                            }
                        } else {
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                const float d = static_cast<float>(th[p]) - ref[p * BLK];
                                s1[p * BLK] += d;
                                s2[p * BLK] = fmaf(d, d, s2[p * BLK]);
                            }
                        }
                        if (++blk_n == kMomBlock || t == ra.I) {
                            // merge the block (n_b states, mean ref + s1/n_b, M2 = s2 - s1^2/n_b)
                            // into the n_mom states of the FP64 Welford state
                            const double nb = blk_n, nn = static_cast<double>(n_mom) + nb;
                            const double inv_nb = 1.0 / nb, w_b = nb / nn, cross = static_cast<double>(n_mom) * w_b;
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                const double a = s1[p * BLK];
                                const double mb = static_cast<double>(ref[p * BLK]) + a * inv_nb;
                                const double m2b = fma(-a, a * inv_nb, static_cast<double>(s2[p * BLK]));
                                const double m = static_cast<double>(wf_mean[p * wf_stride + wf_idx]);
                                const double delta = mb - m;
                                wf_mean[p * wf_stride + wf_idx] = static_cast<W>(fma(delta, w_b, m));
                                wf_m2[p * wf_stride + wf_idx] += static_cast<W>(fma(delta * delta, cross, m2b));
                            }
                            n_mom += blk_n;
                            blk_n = 0;
                        }
                    }
                } else if (all_mode ? (t > ra.B) : on_grid) {
                    ++n_mom;
                    const W inv_n = inv_count<W>(n_mom);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const W x = static_cast<W>(th[p]);
                        W m = wf_mean[p * wf_stride + wf_idx];
                        const W d = x - m;
                        m = welford_fma(d, inv_n, m);
                        wf_mean[p * wf_stride + wf_idx] = m;
                        wf_m2[p * wf_stride + wf_idx] = welford_fma(d, x - m, wf_m2[p * wf_stride + wf_idx]);
                    }
                }
            }
            t_seg = seg_end;
            if (t_seg == to_adapt) {  // a window ends (the same t for every thread)
                const int a = n_acc - ad_acc0;
                ad_e += (a > ra.adapt_hi && ad_e < GAC_ADAPT_EMAX) - (a < ra.adapt_lo && ad_e > GAC_ADAPT_EMIN);
                ad_acc0 = n_acc;
                bm_k = adapt_bm_scale<R>(ad_e);
                to_adapt = (W_ad <= ra.B - t_seg) ? t_seg + W_ad : INT_MAX;
            }
        }
        if (t_end == ra.I) {
            if (ra.accept) ra.accept[c * ra.n_vox + v] = ra.I > 0 ? float(n_acc) / float(ra.I) : 0.0f;
            if (ra.nonfinite) ra.nonfinite[c * ra.n_vox + v] = n_bad;
            if (ra.step_scale) ra.step_scale[c * ra.n_vox + v] = exp2f(0.25f * static_cast<float>(ad_e));
        } else if constexpr (SLICED) {
#pragma unroll
            for (int p = 0; p < P; ++p) static_cast<R *>(ss.theta)[p * nchains + ch] = th[p];
            static_cast<R *>(ss.L)[ch] = L;
            ss.n_acc[ch] = n_acc;
            ss.n_bad[ch] = n_bad;
            ss.adapt[ch] = ad_e;
            ss.adapt[nchains + ch] = ad_acc0;
            if constexpr (kBlocked) {
                if (all_mode && blk_n > 0)
                    for (int k = 0; k < 3 * P; ++k) ss.blk[k * nchains + ch] = bs[k * BLK + tid];
            }
        }
    }

    // a9: pool the C chains of each voxel; the voxel's threads take its
    // parameters in turn
    if (t_end != ra.I) return;
    __syncthreads();
    if (active && (ra.mean || ra.std || ra.rhat)) {
        const int n_each = (ra.moments_mode == GAC_MOMENTS_ALL_POSTBURNIN) ? max(ra.I - ra.B, 0) : ra.S;
        for (int p = c; p < P; p += C)
            pool_chains(wf_mean + p * wf_stride + (wf_idx - c), wf_m2 + p * wf_stride + (wf_idx - c), C, n_each,
                        ra.mean ? ra.mean + p * ra.n_vox + v : nullptr, ra.std ? ra.std + p * ra.n_vox + v : nullptr,
                        ra.rhat ? ra.rhat + p * ra.n_vox + v : nullptr);
    }
}

// One job, one launch: every tile runs all I iterations.
template <int KIND, int PREC, bool TRACE>
__global__ void __launch_bounds__(mh_block<KIND, PREC>(), mh_launch_min_blocks<KIND, PREC>())
    mh_kernel(const ModelConst mc, const RunArgs ra) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SliceState none{};
    for (int64_t tile = blockIdx.x; tile < ra.n_tiles; tile += gridDim.x)
        run_tile<KIND, PREC, TRACE, false, mh_block<KIND, PREC>()>(mc, ra, none, tile, 0, ra.I, smem_raw);
}

}  // namespace gac
