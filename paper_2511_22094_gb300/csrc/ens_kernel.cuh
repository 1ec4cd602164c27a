// Affine-invariant ensemble sampler (the paper's second mcmc.m algorithm,
// Sec. 2.2.2: Nwalkers walkers, one stepSize).  Goodman & Weare's stretch
// move with the two-halves parallel update (Foreman-Mackey et al. 2013):
// walkers 0..H-1 (H = L/2) form half 0 and H..L-1 half 1; iteration t moves
// every walker of half 0 against the current half 1, then every walker of
// half 1 against the updated half 0.  Walker k uses one Philox call with
// counter (t, voxel, k << 8, 0): word 0 picks its partner j in the other half
// (floor(w0 H / 2^32)), word 1 the stretch z = ((a-1) u + 1)^2 / a, word 2 the
// acceptance uniform.  Proposal Y = X_j + z (X_k - X_j); outside the prior
// box it is rejected, otherwise accepted iff log u < (P-1) log z + L(Y) - L(X_k).
//
// Layout: a block holds VB = floor(256 / H) voxels x H threads; thread i of
// voxel lv owns walkers i and H + i.  The walkers' positions and
// log-likelihoods live in shared memory ([VB][L][P] and [VB][L]); the two
// half-steps of an iteration are separated by block barriers, so a half
// reads only positions the other half finished writing.  The measurement
// tile, the likelihood, the precision variants, thinning and the Welford
// moments are those of the MH kernel.
#pragma once
#include "mh_kernel.cuh"

namespace gac {

struct EnsArgs {
    float stretch;    // a > 1
    float inv_stretch;
    double stretch_d;
    int H;            // walkers per half
};

__host__ __device__ inline size_t ens_smem_bytes(int P, size_t r_bytes, size_t w_bytes, int VB, int L,
                                                 int row_stride, bool blocked_moments = false) {
    return 2 * static_cast<size_t>(P) * VB * L * w_bytes  // Welford per walker
           + static_cast<size_t>(VB) * L * P * r_bytes     // positions
           + static_cast<size_t>(VB) * L * r_bytes         // log-likelihoods
           + static_cast<size_t>(VB) * row_stride * sizeof(float)
           + (blocked_moments ? 3 * static_cast<size_t>(P) * VB * L * sizeof(float) : 0);  // block partials
}

// Blocks of 128 threads (5 voxels of 25 threads at 50 walkers), 4 per SM:
// finer blocks than the MH kernel's balance the SMs better at the same 16
// warps (measured 4.6% faster on the 3-pool benchmark than 2 blocks of 256).
constexpr int kEnsBlock = 128;

// BLOCKED (MIXED, moments over every post-burn-in state): the blocked FP32
// accumulation; a separate instantiation so that the other modes keep their
// code unchanged.
template <int KIND, int PREC, bool TRACE, bool BLOCKED = false>
__global__ void __launch_bounds__(kEnsBlock, 4) ens_kernel(const ModelConst mc, const RunArgs ra, const EnsArgs ea) {
    using R = typename PrecTraits<PREC>::R;
    using W = typename PrecTraits<PREC>::W;
    constexpr int P = model_n_par(KIND);
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int L = ra.C, H = ea.H, VB = ra.vox_per_block, M = mc.n_meas;
    const int nw = VB * L;  // walkers per block
    W *wf_mean = reinterpret_cast<W *>(smem_raw);   // [P][nw]
    W *wf_m2 = wf_mean + P * nw;                     // [P][nw]
    R *X = reinterpret_cast<R *>(wf_m2 + P * nw);    // [VB][L][P]
    R *LL = X + nw * P;                              // [VB][L]
    float *ytile = reinterpret_cast<float *>(LL + nw);
    // MIXED, moments over every post-burn-in state: FP32 block partials per
    // walker, s1 [P][nw], s2, reference (the MH kernel's blocked accumulation)
    float *const bs = ytile + VB * ra.row_stride;

    const int tid = threadIdx.x;
    const int lv = tid / H;
    const int i = tid - lv * H;
    const bool lane_used = tid < VB * H;

    for (int64_t tile = blockIdx.x; tile < ra.n_tiles; tile += gridDim.x) {
        const int64_t v0 = tile * VB;
        const int64_t left = ra.n_vox - v0;
        const int nv = left < VB ? static_cast<int>(left) : VB;
        __syncthreads();
        model_smem_load<KIND>(mc);
        {
            const float *src = ra.data + v0 * M;
            for (int e = tid; e < nv * M; e += blockDim.x) {
                const int row = e / M, col = e - row * M;
                ytile[row * ra.row_stride + col] = __ldg(src + e);
            }
        }
        __syncthreads();
        const bool active = lane_used && lv < nv;
        const int64_t v = v0 + lv;
        const uint32_t vg = static_cast<uint32_t>(ra.voxel_base + static_cast<uint64_t>(active ? v : 0));
        const float *y = ytile + lv * ra.row_stride;
        R inv_s2 = R(1);
        if (active) {
            const float sig = ra.sigma ? __ldg(ra.sigma + v) : ra.sigma_scalar;
            inv_s2 = R(1) / (R(sig) * R(sig));
        }
        int n_acc[2] = {0, 0}, n_bad[2] = {0, 0};

        // initial walkers (prior draw at counter iteration 0xFFFFFFFF, or x0)
        if (active) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = h * H + i;
                R *xk = X + (lv * L + k) * P;
                if (ra.x0) {
                    const float *x0 = ra.x0 + (v * L + k) * P;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if constexpr (PREC == GAC_PREC_FP64)
                            xk[p] = fmin(fmax(static_cast<double>(x0[p]), mc.lb_d[p]), mc.ub_d[p]);
                        else
                            xk[p] = fminf(fmaxf(x0[p], mc.lb_f[p]), mc.ub_f[p]);
                    }
                } else {
                    uint32_t w0[4 * ((P + 3) / 4)];
                    draw_words(w0, kInitIteration, vg, static_cast<uint32_t>(k), ra.k0, ra.k1);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if constexpr (PREC == GAC_PREC_FP64)  // uncontracted, as in the FP64 definition
                            xk[p] = __dadd_rn(mc.lb_d[p], __dmul_rn(mc.ub_d[p] - mc.lb_d[p], u01_d(w0[p])));
                        else
                            xk[p] = fmaf(mc.ub_f[p] - mc.lb_f[p], u01_f(w0[p]), mc.lb_f[p]);
                    }
                }
                R th[P];
#pragma unroll
                for (int p = 0; p < P; ++p) th[p] = xk[p];
                LL[lv * L + k] = loglik_any<KIND, PREC>(th, y, inv_s2, mc);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    wf_mean[p * nw + lv * L + k] = W(0);
                    wf_m2[p * nw + lv * L + k] = W(0);
                }
            }
        }
        const bool all_mode = ra.moments_mode == GAC_MOMENTS_ALL_POSTBURNIN;
        constexpr bool blocked = BLOCKED && PREC == GAC_PREC_MIXED;
        int n_mom = 0, blk_n = 0;
        int to_thin = ra.B + ra.T;
        for (int t = 1; t <= ra.I; ++t) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __syncthreads();  // the other half's positions are final
                if (active) {
                    const int k = h * H + i;
                    uint32_t w[4];
                    draw_words(w, static_cast<uint32_t>(t), vg, static_cast<uint32_t>(k), ra.k0, ra.k1);
                    const int j = (1 - h) * H + static_cast<int>((static_cast<uint64_t>(w[0]) * H) >> 32);
                    R z;
                    if constexpr (PREC == GAC_PREC_FP64) {
                        // FP64: every rounding of z and of the proposal is the
                        // plain left-to-right one (no fused multiply-add).  The
                        // stretch moves amplify a one-ulp difference in a
                        // walker by e^{E log z} per accepted move, so only
                        // identically rounded positions stay comparable with an
                        // FP64 reference over thousands of iterations.
                        const double s = __dadd_rn(__dmul_rn(ea.stretch_d - 1.0, u01_d(w[1])), 1.0);
                        z = __dmul_rn(s, s) / ea.stretch_d;
                    } else {
                        const float s = fmaf(ea.stretch - 1.0f, u01_f(w[1]), 1.0f);
                        z = s * s * ea.inv_stretch;
                    }
                    const R *xk = X + (lv * L + k) * P;
                    const R *xj = X + (lv * L + j) * P;
                    R th[P], prop[P];
                    bool inside = true;
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        th[p] = xk[p];
                        const R xjp = xj[p];
                        if constexpr (PREC == GAC_PREC_FP64) {
                            prop[p] = __dadd_rn(xjp, __dmul_rn(z, th[p] - xjp));
                            inside = inside && prop[p] >= mc.lb_d[p] && prop[p] <= mc.ub_d[p];
                        } else {
                            prop[p] = fmaf(z, th[p] - xjp, xjp);
                            inside = inside && prop[p] >= mc.lb_f[p] && prop[p] <= mc.ub_f[p];
                        }
                    }
                    const R Lk = LL[lv * L + k];
                    R Lp = R(0);
                    bool acc = false;
                    if (inside) {
                        Lp = loglik_any<KIND, PREC>(prop, y, inv_s2, mc);
                        n_bad[h] += !isfinite(Lp);
                        // log u < (P - 1) log z + L(Y) - L(X_k): the z factor
                        // enters as an offset of the likelihood difference
                        R logz_term;
                        if constexpr (PREC == GAC_PREC_FP64) logz_term = (P - 1) * log(z);
                        else logz_term = static_cast<float>(P - 1) * __logf(z);  // z in [1/a, a]
                        acc = accept_step<PREC>(Lp + logz_term, Lk, w[2]);
                    }
                    if constexpr (TRACE) {
                        if (v < ra.trace_n) {
                            gac_trace_rec *rec = ra.trace + (v * L + k) * static_cast<int64_t>(ra.I) + (t - 1);
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                rec->theta[p] = static_cast<double>(th[p]);
                                rec->prop[p] = static_cast<double>(prop[p]);
                            }
                            rec->L = static_cast<double>(Lk);
                            rec->Lp = inside ? static_cast<double>(Lp) : __longlong_as_double(0x7ff8000000000000ll);
                            rec->w_acc = w[2];
                            rec->accepted = acc ? 1 : 0;
                        }
                    }
                    if (acc) {
                        R *xw = X + (lv * L + k) * P;
#pragma unroll
                        for (int p = 0; p < P; ++p) xw[p] = prop[p];
                        LL[lv * L + k] = Lp;
                        ++n_acc[h];
                    }
                }
            }
            // thinning grid and moments (own walkers' positions are final)
            const bool on_grid = (t == to_thin);
            if (on_grid) to_thin += ra.T;
            const bool take = all_mode ? (t > ra.B) : on_grid;
            if (active && (on_grid || take)) {
                if (take && !blocked) ++n_mom;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = h * H + i;
                    const R *xk = X + (lv * L + k) * P;
                    if (on_grid && ra.samples) {
                        const int s = (t - ra.B) / ra.T - 1;
                        float *dst = ra.samples + ((static_cast<int64_t>(s) * L + k) * P) * ra.n_vox + v;
#pragma unroll
                        for (int p = 0; p < P; ++p) dst[p * ra.n_vox] = static_cast<float>(xk[p]);
                    }
                    if (take && blocked) {
                        float *s1 = bs + lv * L + k, *s2 = s1 + P * nw, *ref = s2 + P * nw;
                        if (blk_n == 0) {  // the block's first state is its reference
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                ref[p * nw] = static_cast<float>(xk[p]);
                                s1[p * nw] = 0.0f;
                                s2[p * nw] = 0.0f;
                            }
                        } else {
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                const float d = static_cast<float>(xk[p]) - ref[p * nw];
                                s1[p * nw] += d;
                                s2[p * nw] = fmaf(d, d, s2[p * nw]);
                            }
                        }
                    } else if (take) {
                        const W inv_n = W(1) / W(n_mom);
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            const W x = static_cast<W>(xk[p]);
                            const int q = p * nw + lv * L + k;
                            W m = wf_mean[q];
                            const W d = x - m;
                            m += d * inv_n;
                            wf_mean[q] = m;
                            wf_m2[q] += d * (x - m);
                        }
                    }
                }
            }
            // a full block (or the run's last states) merges into the FP64 Welford state
            if (blocked && t > ra.B && (++blk_n == kMomBlock || t == ra.I)) {
                if (active) {
                    const double nb = blk_n, nn = static_cast<double>(n_mom) + nb;
                    const double inv_nb = 1.0 / nb, w_b = nb / nn, cross = static_cast<double>(n_mom) * w_b;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = h * H + i;
                        const float *s1 = bs + lv * L + k, *s2 = s1 + P * nw, *ref = s2 + P * nw;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            const int q = p * nw + lv * L + k;
                            const double a = s1[p * nw];
                            const double mb = static_cast<double>(ref[p * nw]) + a * inv_nb;
                            const double m2b = fma(-a, a * inv_nb, static_cast<double>(s2[p * nw]));
                            const double m = static_cast<double>(wf_mean[q]);
                            const double delta = mb - m;
                            wf_mean[q] = static_cast<W>(fma(delta, w_b, m));
                            wf_m2[q] += static_cast<W>(fma(delta * delta, cross, m2b));
                        }
                    }
                }
                n_mom += blk_n;
                blk_n = 0;
            }
        }
        if (active) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = h * H + i;
                if (ra.accept) ra.accept[k * ra.n_vox + v] = ra.I > 0 ? float(n_acc[h]) / float(ra.I) : 0.0f;
                if (ra.nonfinite) ra.nonfinite[k * ra.n_vox + v] = n_bad[h];
            }
        }
        __syncthreads();
        // pool the walkers of each voxel; its threads take the parameters in turn
        if (active && (ra.mean || ra.std)) {
            const int n_each = all_mode ? max(ra.I - ra.B, 0) : ra.S;
            for (int p = i; p < P; p += H)
                pool_chains(wf_mean + p * nw + lv * L, wf_m2 + p * nw + lv * L, L, n_each,
                            ra.mean ? ra.mean + p * ra.n_vox + v : nullptr, ra.std ? ra.std + p * ra.n_vox + v : nullptr,
                            static_cast<double *>(nullptr));
        }
    }
}

}  // namespace gac
