// Lane-split one-launch Metropolis-Hastings kernel (mcmc.m hot path, Sec.
// 2.2.2) for problems with too few chains to fill the GPU.
//
// With one thread per chain, a few thousand chains leave most SMs with one
// working warp, and an iteration takes as long as its dependency chain
// (Philox rounds, Box-Muller, the forward model's recurrence, the likelihood
// sum, the decision).  Here each chain gets G consecutive lanes of a warp:
//  - lane g evaluates block g of the model's anchored recurrence (kAnchor
//    echoes; it reaches block g's anchors by the same g block steps the
//    one-thread kernel takes), the G block sums are exchanged with
//    __shfl_sync, and every lane adds them with the one-thread kernel's
//    Kahan sequence, so L', every decision and every output are
//    bit-identical to mh_kernel's (MIXED);
//  - random numbers rotate over the lanes: for the round of iterations
//    t0 .. t0+G-1, lane g draws the Philox words of iteration t0+g and the
//    parts of its Box-Muller pairs and acceptance log that do not depend on
//    the chain, one round ahead, and each iteration takes them from that
//    lane by shuffle;
//  - lane g keeps the FP64 Welford accumulators (and the MIXED block
//    partials) of parameters g, g+G, ... and stores those samples.
// Every lane of a warp runs the same iterations (lanes past the tile's last
// voxel compute on a valid row and write nothing), so the shuffles always
// see a converged warp.
//
// Scope (the host checks it and otherwise launches mh_kernel): MIXED
// precision, one launch per job, no trace, a mono-exponential or 3-pool
// model with evenly spaced acquisitions in 2..G blocks of kAnchor.
#pragma once
#include <type_traits>

#include "mh_kernel.cuh"

namespace gac {

constexpr unsigned kFullMask = 0xffffffffu;

// The random quantities of one iteration that do not depend on the chain's
// state: per Box-Muller pair log2 u1 and the angle's sine and cosine, the
// acceptance word and its FP32 log.
template <int P>
struct SplitDraw {
    static constexpr int kPairs = (P + 1) / 2;
    float lg[kPairs], sn[kPairs], cs[kPairs];
    float lu;
    uint32_t w_acc;
};

template <int P>
__device__ __forceinline__ SplitDraw<P> split_draw(uint32_t t, uint32_t vg, uint32_t c, uint32_t k0,
                                                   uint32_t k1) {
    constexpr int NW = n_words(P);
    uint32_t w[4 * n_calls(P)];
    draw_words(w, t, vg, c, k0, k1);
    SplitDraw<P> d;
#pragma unroll
    for (int j = 0; j < SplitDraw<P>::kPairs; ++j) bm_prefix(w[2 * j], w[2 * j + 1], d.lg[j], d.sn[j], d.cs[j]);
    d.w_acc = w[NW - 1];
    d.lu = __logf(u01_f(d.w_acc));
    return d;
}

// A draw's Philox calls in flight, so that their ten rounds can be spread
// over the iterations of a round (the same rounds, keys and words as
// draw_words).
template <int P>
struct PhiloxRun {
    uint32_t c[n_calls(P)][4];
};

template <int P>
__device__ __forceinline__ PhiloxRun<P> philox_start(uint32_t t, uint32_t vg, uint32_t c) {
    PhiloxRun<P> s;
#pragma unroll
    for (int k = 0; k < n_calls(P); ++k) {
        s.c[k][0] = t;
        s.c[k][1] = vg;
        s.c[k][2] = (c << 8) | static_cast<uint32_t>(k);
        s.c[k][3] = 0u;
    }
    return s;
}

// Rounds r0 .. r1-1 of every call.
template <int P>
__device__ __forceinline__ void philox_part(PhiloxRun<P> &s, int r0, int r1, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r < r0 || r >= r1) continue;  // constant after unrolling
#pragma unroll
        for (int k = 0; k < n_calls(P); ++k)
            philox_round(s.c[k][0], s.c[k][1], s.c[k][2], s.c[k][3], k0 + static_cast<uint32_t>(r) * kPhiloxW0,
                         k1 + static_cast<uint32_t>(r) * kPhiloxW1);
    }
}

// The draw from a finished run (as split_draw).
template <int P>
__device__ __forceinline__ SplitDraw<P> split_prefix(const PhiloxRun<P> &s) {
    constexpr int NW = n_words(P);
    uint32_t w[4 * n_calls(P)];
#pragma unroll
    for (int k = 0; k < n_calls(P); ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) w[4 * k + j] = s.c[k][j];
    SplitDraw<P> d;
#pragma unroll
    for (int j = 0; j < SplitDraw<P>::kPairs; ++j) bm_prefix(w[2 * j], w[2 * j + 1], d.lg[j], d.sn[j], d.cs[j]);
    d.w_acc = w[NW - 1];
    d.lu = __logf(u01_f(d.w_acc));
    return d;
}

// The draw of lane `src` of the warp.
template <int P>
__device__ __forceinline__ SplitDraw<P> split_take(const SplitDraw<P> &d, int src) {
    SplitDraw<P> o;
#pragma unroll
    for (int j = 0; j < SplitDraw<P>::kPairs; ++j) {
        o.lg[j] = __shfl_sync(kFullMask, d.lg[j], src);
        o.sn[j] = __shfl_sync(kFullMask, d.sn[j], src);
        o.cs[j] = __shfl_sync(kFullMask, d.cs[j], src);
    }
    o.lu = __shfl_sync(kFullMask, d.lu, src);
    o.w_acc = __shfl_sync(kFullMask, d.w_acc, src);
    return o;
}

// The measurements of lane g's block (echoes g kAnchor ..), kept in registers
// for the whole run: real values, or (re, im) pairs for complex data.
template <int KIND>
struct LaneRows {
    using T = typename std::conditional<model_complex(KIND), float2, float>::type;
    T y[kAnchor];
};

template <int KIND>
__device__ __forceinline__ LaneRows<KIND> lane_rows(const float *row, int g, int n) {
    LaneRows<KIND> r;
#pragma unroll
    for (int i = 0; i < kAnchor; ++i) {
        const int k = min(g * kAnchor + i, n - 1);  // lanes past the last echo read a valid one, unused
        if constexpr (model_complex(KIND)) r.y[i] = reinterpret_cast<const float2 *>(row)[k];
        else r.y[i] = row[k];
    }
    return r;
}

// ResidualVisitor on the block's registers: echo k is entry k - a.
template <int KIND>
struct LaneResidual {
    KahanSum &acc;
    const LaneRows<KIND> &rows;
    int a;
    __device__ __forceinline__ void operator()(int k, float sr, float si) const {
        acc.add2(__ffma2_rn(make_float2(sr, si), f2(-1.0f), rows.y[k - a]));
    }
    __device__ __forceinline__ void operator()(int k, float s) const { acc.add(__fsub_rn(rows.y[k - a], s)); }
};

// Log-likelihood of theta, lanes lane0 .. lane0+G-1 together: lane g sums the
// squared residuals of block g (plain FP32, as KahanSum within a block), the
// block sums are shared, and every lane adds them in block order with
// Kahan's compensation, closing with the empty block that KahanSum::value()
// adds when the last block is full.  The same value in every lane, equal to
// loglik_f<KIND, KahanSum>.  (The first step from s = c = 0 gives s = b_0
// and c = b_0 - b_0 exactly -- 0, or NaN when b_0 is not finite -- as a
// block sum is never -0.)
template <int KIND, int G>
__device__ __forceinline__ float split_loglik(const float *th, const LaneRows<KIND> &rows, float inv_s2,
                                              const ModelConst &mc, int g, int lane0) {
    const int n = mc.n_acq;
    const int nb = (n + kAnchor - 1) / kAnchor;
    const int a = g * kAnchor;
    const int cnt = min(max(n - a, 0), kAnchor);  // 0: the lane has no block
    // echoes past cnt are skipped by predicates, not branches: the same
    // visits as the one-thread kernel's full and partial blocks
    KahanSum acc;
    LaneResidual<KIND> vis{acc, rows, a};
    if constexpr (KIND == GAC_MODEL_MONOEXP) {
        const MonoRec mr = monoexp_setup_f(th, mc);
        float anchor = mr.anchor;
#pragma unroll
        for (int b = 0; b + 1 < G; ++b) anchor = b < g ? __fmul_rn(anchor, mr.rk) : anchor;
        monoexp_block_f<false>(anchor, mr.r1, a, cnt, vis);
    } else {
        static_assert(KIND == GAC_MODEL_MWI3, "lane split: mono-exponential and 3-pool models");
        const Mwi3Rec r = mwi3_setup_f(th, mc);
        float2 X = r.X, Y = r.Y, Z = r.Z;
#pragma unroll
        for (int b = 0; b + 1 < G; ++b) {
            float2 Xn = X, Yn = Y, Zn = Z;
            mwi3_next_anchor(r, Xn, Yn, Zn);
            if (b < g) {
                X = Xn;
                Y = Yn;
                Z = Zn;
            }
        }
        mwi3_block_f<false>(r, X, Y, Z, a, cnt, vis);
    }
    const float bsum = acc.p.x + acc.p.y;
    float s = __shfl_sync(kFullMask, bsum, lane0), c = s - s;
#pragma unroll
    for (int b = 1; b < G; ++b) {
        const float v = __shfl_sync(kFullMask, bsum, lane0 + b);
        const float yv = v - c;
        const float t = s + yv;
        const float cn = (t - s) - yv;
        s = b < nb ? t : s;
        c = b < nb ? cn : c;
    }
    const float closed = s + (0.0f - c);
    if (n == nb * kAnchor) s = closed;
    return -0.5f * s * inv_s2;
}


// Normals of one iteration from its draw: Box-Muller's finish with the chain's
// current step multiplier (bm_finish, as box_muller_f).
template <int P>
__device__ __forceinline__ void split_normals(const SplitDraw<P> &d, float bm_k, float (&z)[P]) {
#pragma unroll
    for (int j = 0; 2 * j < P; ++j) {
        float z0, z1;
        bm_finish(d.lg[j], d.sn[j], d.cs[j], bm_k, z0, z1);
        z[2 * j] = z0;
        if (2 * j + 1 < P) z[2 * j + 1] = z1;
    }
}

// Shared-memory bytes of a split block of `threads` threads (threads / G
// chain slots): FP64 Welford accumulators, the measurement tile and, for
// moments over every post-burn-in state, the FP32 block partials.
__host__ __device__ inline size_t split_smem_bytes(int P, int G, int threads, int VB, int row_stride,
                                                   bool blocked) {
    return tile_smem_bytes(P, sizeof(double), VB, row_stride, true, blocked, threads / G);
}

// One tile of voxels, all I iterations (the one-launch driver of run_tile,
// MIXED, with G lanes per chain; ALL: moments over every post-burn-in state).
// The loop is laid out for latency: an iteration's critical path is
// proposal -> model -> shuffled block sums -> decision, and the next
// iteration's draw and normals, which do not depend on the decision, are
// taken in between; thinning and adaptation share one rare branch.
template <int KIND, int G, bool ALL>
__device__ __forceinline__ void run_tile_split(const ModelConst &mc, const RunArgs &ra, int64_t tile,
                                               unsigned char *smem) {
    using W = double;
    constexpr int P = model_n_par(KIND);
    const int nthr = blockDim.x;
    const int CB = nthr / G;  // chain slots of the block
    const int tid = threadIdx.x;
    const int C = ra.C;
    const int VB = ra.vox_per_block;
    const int M = mc.n_meas;
    const int slot = tid / G, g = tid - slot * G;
    const int lane0 = (tid & 31) - g;  // first lane of this chain's group
    const int lv = slot / C, c = slot - lv * C;
    const int64_t v0 = tile * VB;
    const int64_t left = ra.n_vox - v0;
    const int nv = left < VB ? static_cast<int>(left) : VB;
    const bool active = slot < VB * C && lv < nv;
    W *wf_mean = reinterpret_cast<W *>(smem);
    W *wf_m2 = wf_mean + P * CB;
    float *ytile = reinterpret_cast<float *>(wf_m2 + P * CB);
    float *bs = ytile + VB * ra.row_stride;  // ALL: FP32 block partials s1 [P][CB], s2, reference

    // a1: stage measurements of voxels [v0, v0 + nv) (and the model's table)
    __syncthreads();
    model_smem_load<KIND>(mc);
    {
        const float *src = ra.data + v0 * M;
        const int total = nv * M;
        if (ra.data_vec4) {
            const float4 *src4 = reinterpret_cast<const float4 *>(src);
            for (int i = tid; i < total / 4; i += nthr) {
                const float4 q = __ldg(src4 + i);
                const int e = 4 * i, row = e / M, col = e - row * M;
                float *dst = ytile + row * ra.row_stride + col;
                dst[0] = q.x;
                dst[1] = q.y;
                dst[2] = q.z;
                dst[3] = q.w;
            }
        } else {
            for (int i = tid; i < total; i += nthr) {
                const int row = i / M, col = i - row * M;
                ytile[row * ra.row_stride + col] = __ldg(src + i);
            }
        }
    }
    __syncthreads();

    // lanes without a chain of their own follow voxel v0's chain 0 (writing
    // nothing), so that every shuffle sees a converged warp; warps without
    // any chain skip the iterations
    const int lvr = active ? lv : 0, cr = active ? c : 0;
    const int64_t v = v0 + lvr;
    const LaneRows<KIND> rows = lane_rows<KIND>(ytile + lvr * ra.row_stride, g, mc.n_acq);
    const float sig = ra.sigma ? __ldg(ra.sigma + v) : ra.sigma_scalar;
    const float inv_s2 = 1.0f / (sig * sig);
    const uint32_t vg = static_cast<uint32_t>(ra.voxel_base + static_cast<uint64_t>(v));
    const uint32_t cu = static_cast<uint32_t>(cr);
    const int64_t ch = v * C + cr;

    int n_acc = 0, n_bad = 0, ad_e = 0;
    if (__any_sync(kFullMask, active)) {
        // a2: initial state
        float th[P];
        if (ra.x0) {
            const float *x0 = ra.x0 + ch * P;
#pragma unroll
            for (int p = 0; p < P; ++p) th[p] = fminf(fmaxf(x0[p], mc.lb_f[p]), mc.ub_f[p]);
        } else {
            uint32_t w0[4 * ((P + 3) / 4)];
            draw_words(w0, kInitIteration, vg, cu, ra.k0, ra.k1);
#pragma unroll
            for (int p = 0; p < P; ++p) th[p] = fmaf(mc.ub_f[p] - mc.lb_f[p], u01_f(w0[p]), mc.lb_f[p]);
        }
        float L = split_loglik<KIND, G>(th, rows, inv_s2, mc, g, lane0);
        if (active) {
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (p % G == g) {
                    wf_mean[p * CB + slot] = 0.0;
                    wf_m2[p * CB + slot] = 0.0;
                }
        }
        int ad_acc0 = 0, n_mom = 0, blk_n = 0;
        // thinned moments: lane g's parameters p = g + kG in registers.  Each
        // Welford update (mh_kernel's, operation for operation) is split over
        // two thinning events: d = x - m and m += d / n at its own, M2 += d (x -
        // m) at the next, beside that one's first half -- two independent FP64
        // chains instead of one twice as long (each FP64 instruction holds the
        // sub-partition's FP64 pipe for ~76 cycles, and nothing else hides it)
        constexpr int PL = (P + G - 1) / G;
        double wm[PL], wm2[PL], wxd[PL], wd[PL];
#pragma unroll
        for (int k = 0; k < PL; ++k) wm[k] = wm2[k] = wxd[k] = wd[k] = 0.0;
        bool wpend = false;  // the previous update's second half is pending
        int to_thin = ra.B + ra.T;
        const int W_ad = ra.adapt_window;
        int to_adapt = (W_ad > 0 && W_ad <= ra.B) ? W_ad : INT_MAX;
        int t_event = min(to_thin, to_adapt);  // the next iteration that thins or ends a window
        float bm_k = adapt_bm_scale<float>(ad_e);

        // draws of this round and the next (lane g: iteration t0 + g), and
        // the first iteration's normals
        // cur, nxt: the draws of this round and the next (the next one's
        // Box-Muller prefixes are taken in this round's first iteration, from
        // the finished Philox run `wnx`); `pr`: the Philox calls of the round
        // after next, advanced a part in every iteration of this round
        SplitDraw<P> cur = split_draw<P>(static_cast<uint32_t>(1 + g), vg, cu, ra.k0, ra.k1);
        SplitDraw<P> nxt;
        PhiloxRun<P> wnx = philox_start<P>(static_cast<uint32_t>(1 + G + g), vg, cu);
        philox_part<P>(wnx, 0, 10, ra.k0, ra.k1);
        PhiloxRun<P> pr = philox_start<P>(static_cast<uint32_t>(1 + 2 * G + g), vg, cu);
        float z[P];
        float lu;
        uint32_t w_acc;
        {
            const SplitDraw<P> d = split_take<P>(cur, lane0);
            split_normals<P>(d, bm_k, z);
            lu = d.lu;
            w_acc = d.w_acc;
        }
        for (int t0 = 1; t0 <= ra.I; t0 += G) {
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const int t = t0 + i;
                if (t > ra.I) break;  // the same t for every lane
                if (i == 0) nxt = split_prefix<P>(wnx);
                philox_part<P>(pr, (10 * i) / G, (10 * (i + 1)) / G, ra.k0, ra.k1);
                // a4: proposal
                float prop[P];
#pragma unroll
                for (int p = 0; p < P; ++p)
                    prop[p] = fminf(fmaxf(fmaf(mc.step_f[p], z[p], th[p]), mc.lb_f[p]), mc.ub_f[p]);
                // the next iteration's draw and normals: independent of this decision
                const SplitDraw<P> dn = split_take<P>(i + 1 < G ? cur : nxt, lane0 + (i + 1 < G ? i + 1 : 0));
                float zn[P];
                split_normals<P>(dn, bm_k, zn);
                // a5 + a6: forward model and likelihood, lanes together
                const float Lp = split_loglik<KIND, G>(prop, rows, inv_s2, mc, g, lane0);
                // a7: accept_mixed, with its rare FP64 re-decision and the rare
                // thinning / adaptation events in one branch
                const float d32 = Lp - L;
                const float margin = fmaf(0x1p-22f, fabsf(d32), 1e-5f);
                const float gap = d32 - lu;
                bool acc = gap > 0.0f;
                const bool near = !(fabsf(gap) > margin);
                n_bad += !isfinite(Lp);
                // the FP32 decision takes effect at once; the rare branch below
                // corrects it where the FP64 re-decision differs.  Only the
                // lanes with a near decision enter it between events (it holds
                // no warp-wide operation); at a thinning or adaptation event
                // every lane does
                float th_old[P];
                const float L_old = L;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    th_old[p] = th[p];
                    th[p] = acc ? prop[p] : th[p];
                }
                L = acc ? Lp : L;
                n_acc += acc ? 1 : 0;
                if (__builtin_expect(near || t == t_event, 0)) {
                    if (near) {
                        const bool acc64 = log(u01_d(w_acc)) < static_cast<double>(Lp) - static_cast<double>(L_old);
                        if (acc64 != acc) {
#pragma unroll
                            for (int p = 0; p < P; ++p) th[p] = acc64 ? prop[p] : th_old[p];
                            L = acc64 ? Lp : L_old;
                            n_acc += acc64 ? 1 : -1;
                            acc = acc64;
                        }
                    }
                    if (t == t_event) {
                        if (t == to_thin) {
                            to_thin += ra.T;
                            const float *x = th;
                            if (ra.samples && active) {
                                const int sidx = (t - ra.B) / ra.T - 1;
                                float *dst = ra.samples + ((static_cast<int64_t>(sidx) * C + c) * P) * ra.n_vox + v;
#pragma unroll
                                for (int p = 0; p < P; ++p)
                                    if (p % G == g) dst[p * ra.n_vox] = x[p];
                            }
                            if constexpr (!ALL) {
                                ++n_mom;
                                const W inv_n = inv_count<W, true>(n_mom);
#pragma unroll
                                for (int p = 0; p < P; ++p)
                                    if (p % G == g) {
                                        const int k = p / G;
                                        if (wpend) wm2[k] = welford_fma(wd[k], wxd[k] - wm[k], wm2[k]);
                                        wxd[k] = static_cast<W>(x[p]);
                                        wd[k] = wxd[k] - wm[k];
                                        wm[k] = welford_fma(wd[k], inv_n, wm[k]);
                                    }
                                wpend = true;
                            }
                        }
                        if (t == to_adapt) {  // a window of the burn-in adaptation ends
                            const int a = n_acc - ad_acc0;
                            ad_e += (a > ra.adapt_hi && ad_e < GAC_ADAPT_EMAX) - (a < ra.adapt_lo && ad_e > GAC_ADAPT_EMIN);
                            ad_acc0 = n_acc;
                            bm_k = adapt_bm_scale<float>(ad_e);
                            to_adapt = (W_ad <= ra.B - t) ? t + W_ad : INT_MAX;
                            split_normals<P>(dn, bm_k, zn);  // the next iteration takes the new steps
                        }
                        t_event = min(to_thin, to_adapt);
                    }
                }
                if constexpr (ALL) {
                    if (t > ra.B) {
                        float *s1 = bs + slot, *s2 = bs + P * CB + slot, *ref = bs + 2 * P * CB + slot;
                        if (blk_n == 0) {
#pragma unroll
                            for (int p = 0; p < P; ++p)
                                if (p % G == g) {
                                    ref[p * CB] = th[p];
                                    s1[p * CB] = 0.0f;
                                    s2[p * CB] = 0.0f;
                                }
                        } else {
#pragma unroll
                            for (int p = 0; p < P; ++p)
                                if (p % G == g) {
                                    const float dd = th[p] - ref[p * CB];
                                    s1[p * CB] += dd;
                                    s2[p * CB] = fmaf(dd, dd, s2[p * CB]);
                                }
                        }
                        if (++blk_n == kMomBlock || t == ra.I) {
                            const double nb = blk_n, nn = static_cast<double>(n_mom) + nb;
                            const double inv_nb = 1.0 / nb, w_b = nb / nn, cross = static_cast<double>(n_mom) * w_b;
#pragma unroll
                            for (int p = 0; p < P; ++p)
                                if (p % G == g && active) {
                                    const double a = s1[p * CB];
                                    const double mb = static_cast<double>(ref[p * CB]) + a * inv_nb;
                                    const double m2b = fma(-a, a * inv_nb, static_cast<double>(s2[p * CB]));
                                    const double m = wf_mean[p * CB + slot];
                                    const double delta = mb - m;
                                    wf_mean[p * CB + slot] = fma(delta, w_b, m);
                                    wf_m2[p * CB + slot] += fma(delta * delta, cross, m2b);
                                }
                            n_mom += blk_n;
                            blk_n = 0;
                        }
                    }
                }
#pragma unroll
                for (int p = 0; p < P; ++p) z[p] = zn[p];
                lu = dn.lu;
                w_acc = dn.w_acc;
            }
            cur = nxt;
            wnx = pr;
            pr = philox_start<P>(static_cast<uint32_t>(t0 + 3 * G + g), vg, cu);
        }
        if constexpr (!ALL) {
            if (wpend) {
#pragma unroll
                for (int k = 0; k < PL; ++k) wm2[k] = welford_fma(wd[k], wxd[k] - wm[k], wm2[k]);
            }
            if (active) {
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (p % G == g) {
                        wf_mean[p * CB + slot] = wm[p / G];
                        wf_m2[p * CB + slot] = wm2[p / G];
                    }
            }
        }
    }
    if (active && g == 0) {
        if (ra.accept) ra.accept[c * ra.n_vox + v] = ra.I > 0 ? float(n_acc) / float(ra.I) : 0.0f;
        if (ra.nonfinite) ra.nonfinite[c * ra.n_vox + v] = n_bad;
        if (ra.step_scale) ra.step_scale[c * ra.n_vox + v] = exp2f(0.25f * static_cast<float>(ad_e));
    }

    // a9: pool the C chains of each voxel; the voxel's C * G threads take its
    // parameters in turn
    __syncthreads();
    if (active && (ra.mean || ra.std || ra.rhat)) {
        const int n_each = ALL ? max(ra.I - ra.B, 0) : ra.S;
        for (int p = c * G + g; p < P; p += C * G)
            pool_chains(wf_mean + p * CB + (slot - c), wf_m2 + p * CB + (slot - c), C, n_each,
                        ra.mean ? ra.mean + p * ra.n_vox + v : nullptr, ra.std ? ra.std + p * ra.n_vox + v : nullptr,
                        ra.rhat ? ra.rhat + p * ra.n_vox + v : nullptr);
    }
}

// Small problems only: no register cap beyond the block size (the 3-pool
// form would spill under the one-thread kernel's 2-blocks-per-SM cap).
template <int KIND, int G, bool ALL>
__global__ void __launch_bounds__(kBlock, 1)
    mh_split_kernel(const ModelConst mc, const RunArgs ra) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int64_t tile = blockIdx.x; tile < ra.n_tiles; tile += gridDim.x)
        run_tile_split<KIND, G, ALL>(mc, ra, tile, smem_raw);
}

}  // namespace gac
