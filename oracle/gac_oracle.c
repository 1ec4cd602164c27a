/*
 * gac_oracle.c -- plain FP64 CPU oracle for the voxel-wise Metropolis-Hastings
 * sampler of GACELLE's mcmc.m (Chan et al., arXiv 2511.22094, Sec. 2.2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The CUDA library never
 * links, includes or calls it, and it shares no source with the CUDA path:
 * its Philox generator, forward models, likelihood, sampler and moment code
 * are written here a second time, slowly and plainly, in double precision.
 *
 * What it computes, in the paper's order:
 *   - Gaussian log-likelihood of the measured signal given the forward model
 *     (Sec. 2.2.2: "the likelihood is Gaussian"; weighting by voxel SNR as in
 *     Eq. 1);
 *   - a normal random-walk proposal with a per-parameter step (the xStepSize
 *     option, Sec. 2.2.2), clamped to the uniform-prior bounds;
 *   - Metropolis acceptance, burn-in, thinning and the posterior mean/SD of the
 *     thinned samples (Sec. 2.2.2 options; Sec. 2.3.1 out.mean / out.std).
 *   Forward models: mono-exponential decay (Eq. 3), the 3-pool complex
 *   myelin-water GRE model and the spherical-mean Standard Model (Sec. 2.1,
 *   model list; closed forms stated below), and a linear test model whose
 *   posterior is known exactly.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), from its published
 * definition: counter (t, voxel, chain<<8 | call, 0), key (seed lo, seed hi).
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, library routines (erf/erfi, Gauss-Legendre
 * quadrature, cuRAND's host Philox), exact linear-Gaussian posteriors and
 * brute-force grid posteriors.  No function is "parity unpinned".
 */
#define _XOPEN_SOURCE 700 /* j0, j1 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MONOEXP 1
#define ORC_MWI3 2
#define ORC_SMT 3
#define ORC_AXCAL 4
#define ORC_LINEAR 100

#define ORC_INIT_ITER 0xFFFFFFFFu

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3" (SC'11): ten rounds of a multiply-hi/lo + xor bijection */
/* on four 32-bit words, with a Weyl-sequence key schedule.                  */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)mult0 * (uint64_t)x[0];
        uint64_t prod1 = (uint64_t)mult1 * (uint64_t)x[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ x[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ x[3] ^ k1;
        uint32_t n3 = lo0;
        x[0] = n0; x[1] = n1; x[2] = n2; x[3] = n3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

/* The n words of one (iteration t, voxel v, chain c) draw: call k of the
 * generator supplies words 4k..4k+3. */
void orc_words(uint64_t seed, uint32_t t, uint32_t v, uint32_t c, int n, uint32_t *w) {
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    for (int k = 0; 4 * k < n; ++k) {
        uint32_t ctr[4] = {t, v, (c << 8) | (uint32_t)k, 0u};
        uint32_t out[4];
        orc_philox4x32_10(ctr, key, out);
        for (int j = 0; j < 4 && 4 * k + j < n; ++j) w[4 * k + j] = out[j];
    }
}

/* A 32-bit word to a uniform on the open interval (0, 1): (w + 1/2) 2^-32. */
double orc_u01(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }

/* Words used per MH iteration for P parameters: two per Box-Muller pair for
 * the P normals, then one for the acceptance uniform (the last word). */
int orc_n_words(int n_par) { return 2 * ((n_par + 1) / 2) + 1; }

/* Box-Muller: pair j takes u1 = u01(w[2j]), u2 = u01(w[2j+1]);
 * z[2j] = sqrt(-2 ln u1) cos(2 pi u2), z[2j+1] = sqrt(-2 ln u1) sin(2 pi u2). */
void orc_normals_from_words(const uint32_t *w, int n_par, double *z) {
    for (int j = 0; 2 * j < n_par; ++j) {
        double u1 = orc_u01(w[2 * j]);
        double u2 = orc_u01(w[2 * j + 1]);
        double radius = sqrt(-2.0 * log(u1));
        double angle = 2.0 * ORC_PI * u2;
        z[2 * j] = radius * cos(angle);
        if (2 * j + 1 < n_par) z[2 * j + 1] = radius * sin(angle);
    }
}

/* ------------------------------------------------------------------------ */
/* Forward signal models                                                     */
/* ------------------------------------------------------------------------ */

int orc_n_par(int kind) {
    switch (kind) {
    case ORC_MONOEXP: return 2;
    case ORC_MWI3: return 9;
    case ORC_SMT: return 4;
    case ORC_AXCAL: return 4;
    case ORC_LINEAR: return 2;
    default: return -1;
    }
}

/* Real-valued measurements per voxel: complex models count re and im;
 * AxCaliberSMT takes (b, Delta, delta) triplets. */
int orc_n_meas(int kind, int n_acq) {
    if (kind == ORC_MWI3) return 2 * n_acq;
    if (kind == ORC_AXCAL) return (n_acq % 3 == 0) ? n_acq / 3 : -1;
    if (orc_n_par(kind) < 0) return -1;
    return n_acq;
}

/* g(x) = integral_0^1 exp(-x u^2) du, the orientation average of a stick
 * (spherical-mean technique).  For x > 1 it is sqrt(pi) erf(sqrt x)/(2 sqrt x);
 * for x <= 1 (including x < 0, the erfi branch) the power series
 * sum_n (-x)^n / (n! (2n+1)), whose terms are all positive when x < 0. */
double orc_g(double x) {
    if (x > 1.0) {
        double s = sqrt(x);
        return sqrt(ORC_PI) * erf(s) / (2.0 * s);
    }
    double term = 1.0; /* (-x)^n / n! */
    double sum = 1.0;
    for (int n = 1; n < 400; ++n) {
        term *= -x / (double)n;
        double add = term / (double)(2 * n + 1);
        sum += add;
        if (fabs(add) <= 1e-18 * fabs(sum)) break;
    }
    return sum;
}

/* m-th positive zero (m >= 1) of J1'(x) = J0(x) - J1(x)/x, by bisection on
 * [(m - 1/4) pi - 1, (m - 1/4) pi + 0.2], which holds exactly one zero
 * (McMahon: the zeros lie just below (m - 1/4) pi). */
double orc_j1p_zero(int m) {
    double lo = (m - 0.25) * ORC_PI - 1.0, hi = (m - 0.25) * ORC_PI + 0.2;
    if (lo < 0.5) lo = 0.5;
    double flo = j0(lo) - j1(lo) / lo;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double fm = j0(mid) - j1(mid) / mid;
        if ((fm < 0.0) == (flo < 0.0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

/* e^{-y} - 1 + y, without the cancellation of the plain form for small y. */
static double e_minus_one_plus(double y) { return expm1(-y) + y; }

/* -ln E_perp of a cylinder of radius R [um] with intrinsic diffusivity D
 * [um^2/ms] under a pulsed-gradient pair (b [ms/um^2], separation Delta,
 * duration delta [ms]) in the Gaussian phase approximation (Neuman 1974;
 * van Gelderen et al. 1994):
 *   kappa = 2 gamma^2 G^2 sum_m R^6 / (D^2 x_m^6 (x_m^2 - 1)) N_m,
 *   N_m = 2 delta q - 2 + 2 e^{-q delta} + 2 e^{-q Delta}
 *         - e^{-q (Delta - delta)} - e^{-q (Delta + delta)},  q = x_m^2 D / R^2,
 * x_m the zeros of J1', gamma^2 G^2 = b / (delta^2 (Delta - delta/3)).  N_m
 * is summed as 2E(q delta) + 2E(q Delta) - E(q (Delta - delta)) -
 * E(q (Delta + delta)) with E(y) = e^{-y} - 1 + y (the same sum; the linear
 * and constant terms cancel exactly).  ORC_AX_TERMS zeros. */
#define ORC_AX_TERMS 100
static double orc_zeros[ORC_AX_TERMS];
__attribute__((constructor)) static void orc_init_zeros(void) {
    for (int m = 0; m < ORC_AX_TERMS; ++m) orc_zeros[m] = orc_j1p_zero(m + 1);
}

double orc_cyl_kappa(double b, double Delta, double delta, double R, double D) {
    const double *zeros = orc_zeros;
    double g2 = b / (delta * delta * (Delta - delta / 3.0));
    double sum = 0.0;
    for (int m = 0; m < ORC_AX_TERMS; ++m) {
        double x = zeros[m], x2 = x * x;
        double q = x2 * D / (R * R);
        double N = 2.0 * e_minus_one_plus(q * delta) + 2.0 * e_minus_one_plus(q * Delta) -
                   e_minus_one_plus(q * (Delta - delta)) - e_minus_one_plus(q * (Delta + delta));
        double r2 = R * R;
        sum += (r2 * r2 * r2) / (D * D * x2 * x2 * x2 * (x2 - 1.0)) * N;
    }
    return 2.0 * g2 * sum;
}

/* AxCaliberSMT's fixed diffusivities [um^2/ms] (Sec. 2.5): intra-axonal and
 * extra-axonal parallel 1.7, free water 3. */
#define ORC_AX_DA 1.7
#define ORC_AX_DEPAR 1.7
#define ORC_AX_DCSF 3.0

/* Evaluates the forward model at theta; writes n_meas(kind, n_acq) reals.
 *  MONOEXP (Eq. 3):  s_k = S0 exp(-R2* TE_k), theta = (S0, R2* [1/s]),
 *                    acq = TE [ms].
 *  MWI3:  S(t) = exp(i phi0) sum_{j in MW,IW,EW} A_j exp(-t/T2*_j) exp(-i 2 pi df_j t),
 *         theta = (A_MW, A_IW, A_EW, T2*_MW, T2*_IW, T2*_EW [ms], df_MW, df_IW [Hz],
 *         phi0 [rad]), df_EW = 0, acq = TE [ms]; output (re, im) per echo.
 *  SMT:   s(b) = f g(b Da) + (1 - f) exp(-b De_perp) g(b (De_par - De_perp)), S0 = 1,
 *         theta = (f, Da, De_par, De_perp) [um^2/ms], acq = b [ms/um^2].
 *  AXCAL: AxCaliberSMT (Sec. 2.5, after Fan et al. 2020), S0 = 1:
 *         s = (1 - f_csf) [f_n e^{-k} g(b Da - k) + (1 - f_n) e^{-b De_R} g(b (De_par - De_R))]
 *             + f_csf e^{-b D_csf},  k = orc_cyl_kappa(b, Delta, delta, a/2, Da),
 *         the restricted cylinder's spherical mean being the orientation
 *         average of e^{-b Da u^2 - k (1 - u^2)};
 *         theta = (a [um, axon diameter], f_n, f_csf, De_R [um^2/ms]),
 *         acq = (b [ms/um^2], Delta [ms], delta [ms]) per measurement.
 *  LINEAR: s_k = a + c t_k, theta = (a, c), acq = t. */
int orc_forward(int kind, const double *acq, int n_acq, const double *theta, double *s) {
    switch (kind) {
    case ORC_MONOEXP:
        for (int k = 0; k < n_acq; ++k) s[k] = theta[0] * exp(-theta[1] * acq[k] * 1e-3);
        return 0;
    case ORC_MWI3:
        for (int k = 0; k < n_acq; ++k) {
            double t = acq[k], re = 0.0, im = 0.0;
            for (int j = 0; j < 3; ++j) {
                double amp = theta[j] * exp(-t / theta[3 + j]);
                double df = (j < 2) ? theta[6 + j] : 0.0;
                double ang = theta[8] - 2.0 * ORC_PI * df * t * 1e-3;
                re += amp * cos(ang);
                im += amp * sin(ang);
            }
            s[2 * k] = re;
            s[2 * k + 1] = im;
        }
        return 0;
    case ORC_SMT:
        for (int k = 0; k < n_acq; ++k) {
            double b = acq[k];
            double f = theta[0], da = theta[1], dpar = theta[2], dperp = theta[3];
            double intra = orc_g(b * da);
            double extra = exp(-b * dperp) * orc_g(b * (dpar - dperp));
            s[k] = f * intra + (1.0 - f) * extra;
        }
        return 0;
    case ORC_AXCAL: {
        if (n_acq % 3 != 0) return -1;
        double R = 0.5 * theta[0], fn = theta[1], fcsf = theta[2], der = theta[3];
        for (int k = 0; k < n_acq / 3; ++k) {
            double b = acq[3 * k], Delta = acq[3 * k + 1], delta = acq[3 * k + 2];
            double kap = orc_cyl_kappa(b, Delta, delta, R, ORC_AX_DA);
            double restricted = exp(-kap) * orc_g(b * ORC_AX_DA - kap);
            double hindered = exp(-b * der) * orc_g(b * (ORC_AX_DEPAR - der));
            s[k] = (1.0 - fcsf) * (fn * restricted + (1.0 - fn) * hindered) + fcsf * exp(-b * ORC_AX_DCSF);
        }
        return 0;
    }
    case ORC_LINEAR:
        for (int k = 0; k < n_acq; ++k) s[k] = theta[0] + theta[1] * acq[k];
        return 0;
    default:
        return -1;
    }
}

/* Gaussian log-likelihood, constant dropped: L = -1/2 sum_m ((y_m - s_m)/sigma)^2. */
double orc_loglik(int kind, const double *acq, int n_acq, const double *theta,
                  const float *y, double sigma) {
    int m = orc_n_meas(kind, n_acq);
    double s[512];
    if (m < 0 || m > 512) return NAN;
    orc_forward(kind, acq, n_acq, theta, s);
    double sum = 0.0;
    for (int i = 0; i < m; ++i) {
        double r = ((double)y[i] - s[i]) / sigma;
        sum += r * r;
    }
    return -0.5 * sum;
}

/* ------------------------------------------------------------------------ */
/* Metropolis-Hastings sampler                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int kind;
    int n_acq;
    const double *acq;
    int n_par;
    const double *lb, *ub, *step;
} orc_model;

typedef struct {
    int iterations; /* I */
    int burnin;     /* B, a count of iterations */
    int thin;       /* T */
    int n_chains;   /* C */
    uint64_t seed;
    uint64_t voxel_base;  /* global index of voxel 0, used in the counter */
    int moments_mode;     /* 0: thinned samples, 1: every post-burn-in state */
    int n_threads;        /* 0: all available */
    int adapt_window;     /* 0: fixed steps; > 0: burn-in adaptation window (below) */
    double adapt_target;  /* target acceptance rate of the adaptation, in (0, 1) */
} orc_opts;

/* Step adaptation during burn-in (an extension: the paper's steps are fixed).
 * Each chain carries an integer exponent e, starting at 0, and proposes with
 * the steps xStepSize * 2^(e/4).  After iteration t with t % W == 0 and
 * t <= B (W = adapt_window), let a be the number of proposals the chain
 * accepted in iterations t-W+1 .. t: e rises by one if a > target * W and
 * falls by one if a < target * W, within [ORC_ADAPT_EMIN, ORC_ADAPT_EMAX].
 * After burn-in the steps stay fixed, so the states that enter the moments
 * come from a Metropolis-Hastings chain with a fixed proposal. */
#define ORC_ADAPT_EMIN (-48)
#define ORC_ADAPT_EMAX 16

/* Number of thinned samples per chain: t in {B+T, B+2T, ...} <= I. */
int orc_n_samples(int iterations, int burnin, int thin) {
    if (thin <= 0 || iterations <= burnin) return 0;
    return (iterations - burnin) / thin;
}

static double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

/* One chain of one voxel.  path (optional) receives the state after each
 * iteration t = 0..I as [I+1][P]; pooled (optional) receives the states that
 * enter the moments, `per_chain` values per parameter, as [P][per_chain]. */
static void run_chain(const orc_model *m, const float *y, double sigma, const float *x0,
                      const orc_opts *o, uint32_t vg, uint32_t c, int64_t v, int64_t n_vox,
                      double *samples, double *pooled, int per_chain, double *accept_rate,
                      int32_t *nonfinite, double *step_scale, double *path) {
    int P = m->n_par, I = o->iterations, B = o->burnin, T = o->thin;
    int S = orc_n_samples(I, B, T);
    int nw = orc_n_words(P);
    double theta[64], prop[64], z[64];
    uint32_t w[160];

    if (x0) {
        for (int p = 0; p < P; ++p) theta[p] = clampd((double)x0[p], m->lb[p], m->ub[p]);
    } else {
        orc_words(o->seed, ORC_INIT_ITER, vg, c, P, w);
        for (int p = 0; p < P; ++p) theta[p] = m->lb[p] + (m->ub[p] - m->lb[p]) * orc_u01(w[p]);
    }
    double L = orc_loglik(m->kind, m->acq, m->n_acq, theta, y, sigma);
    if (path) memcpy(path, theta, sizeof(double) * P);

    long n_acc = 0, n_bad = 0, n_acc_window_start = 0;
    int n_pooled = 0;
    int e = 0;            /* adaptation exponent */
    double lambda = 1.0;  /* step multiplier 2^(e/4) */
    for (int t = 1; t <= I; ++t) {
        orc_words(o->seed, (uint32_t)t, vg, c, nw, w);
        orc_normals_from_words(w, P, z);
        for (int p = 0; p < P; ++p)
            prop[p] = clampd(theta[p] + m->step[p] * (lambda * z[p]), m->lb[p], m->ub[p]);
        double Lp = orc_loglik(m->kind, m->acq, m->n_acq, prop, y, sigma);
        if (!isfinite(Lp)) ++n_bad;
        double log_u = log(orc_u01(w[nw - 1]));
        if (log_u < Lp - L) { /* strict; NaN compares false and rejects */
            memcpy(theta, prop, sizeof(double) * P);
            L = Lp;
            ++n_acc;
        }
        if (o->adapt_window > 0 && t <= B && t % o->adapt_window == 0) {
            double a = (double)(n_acc - n_acc_window_start);
            double target = o->adapt_target * (double)o->adapt_window;
            if (a > target && e < ORC_ADAPT_EMAX) ++e;
            if (a < target && e > ORC_ADAPT_EMIN) --e;
            lambda = exp2(0.25 * (double)e);
            n_acc_window_start = n_acc;
        }
        if (path) memcpy(path + (size_t)t * P, theta, sizeof(double) * P);
        int on_grid = (t > B) && T > 0 && ((t - B) % T == 0);
        if (on_grid) {
            int s = (t - B) / T - 1;
            if (samples && s < S)
                for (int p = 0; p < P; ++p)
                    samples[(((size_t)s * o->n_chains + c) * P + p) * n_vox + v] = theta[p];
        }
        if (pooled) {
            int take = (o->moments_mode == 1) ? (t > B) : on_grid;
            if (take && n_pooled < per_chain) {
                for (int p = 0; p < P; ++p) pooled[(size_t)p * per_chain + n_pooled] = theta[p];
                ++n_pooled;
            }
        }
    }
    if (accept_rate) accept_rate[(size_t)c * n_vox + v] = I > 0 ? (double)n_acc / (double)I : 0.0;
    if (nonfinite) nonfinite[(size_t)c * n_vox + v] = (int32_t)n_bad;
    if (step_scale) step_scale[(size_t)c * n_vox + v] = lambda;
}

/* Potential scale reduction factor of C chains of n values each (x[c * stride
 * + i], i < n), Gelman & Rubin (1992) without chain splitting:
 *   W = mean over chains of the within-chain variances (n-1 divisor),
 *   B/n = variance of the chain means (C-1 divisor),
 *   R-hat = sqrt(((n-1)/n W + B/n) / W).
 * NaN for C < 2 or n < 2 (and for W = B = 0); +inf for W = 0 < B. */
double orc_rhat(const double *x, int C, int n, size_t stride) {
    if (C < 2 || n < 2) return NAN;
    double mean_of_means = 0.0;
    for (int c = 0; c < C; ++c) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += x[(size_t)c * stride + i];
        mean_of_means += sum / n;
    }
    mean_of_means /= C;
    double W = 0.0, B_over_n = 0.0;
    for (int c = 0; c < C; ++c) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += x[(size_t)c * stride + i];
        double chain_mean = sum / n;
        double ss = 0.0;
        for (int i = 0; i < n; ++i) {
            double d = x[(size_t)c * stride + i] - chain_mean;
            ss += d * d;
        }
        W += ss / (n - 1);
        B_over_n += (chain_mean - mean_of_means) * (chain_mean - mean_of_means);
    }
    W /= C;
    B_over_n /= (C - 1);
    double var_plus = (double)(n - 1) / n * W + B_over_n;
    return sqrt(var_plus / W);
}

/* Mean and SD (n-1 divisor) of the pooled values of C chains, stored chain
 * after chain as [P][per_chain] blocks; n = 0 gives NaN, n = 1 an SD of 0;
 * R-hat of the chains per parameter. */
static void pooled_moments(const double *pooled, int C, int per_chain, int P, int64_t v,
                           int64_t n_vox, double *mean, double *std, double *rhat) {
    size_t n_all = (size_t)C * per_chain;
    for (int p = 0; p < P; ++p) {
        double sum = 0.0;
        for (int c = 0; c < C; ++c)
            for (int i = 0; i < per_chain; ++i)
                sum += pooled[(size_t)c * per_chain * P + (size_t)p * per_chain + i];
        double mu = n_all > 0 ? sum / (double)n_all : NAN;
        double ss = 0.0;
        for (int c = 0; c < C; ++c)
            for (int i = 0; i < per_chain; ++i) {
                double d = pooled[(size_t)c * per_chain * P + (size_t)p * per_chain + i] - mu;
                ss += d * d;
            }
        double sd = n_all > 1 ? sqrt(ss / (double)(n_all - 1)) : (n_all == 1 ? 0.0 : NAN);
        if (mean) mean[(size_t)p * n_vox + v] = mu;
        if (std) std[(size_t)p * n_vox + v] = sd;
        if (rhat)
            rhat[(size_t)p * n_vox + v] =
                orc_rhat(pooled + (size_t)p * per_chain, C, per_chain, (size_t)per_chain * P);
    }
}

/* Runs C chains for each of n_vox voxels.  data: [n_vox][n_meas] float (complex
 * data interleaved re, im); sigma: [n_vox] or NULL (then sigma_scalar);
 * x0: [n_vox][C][P] or NULL.  Outputs (each may be NULL):
 *   mean, std   [P][n_vox]      pooled over chains (two-pass, n-1 divisor);
 *   samples     [S][C][P][n_vox];
 *   accept_rate [C][n_vox]      accepted / I;
 *   nonfinite   [C][n_vox]      iterations with a non-finite proposal likelihood;
 *   rhat        [P][n_vox]      R-hat over the chains of the moment values;
 *   step_scale  [C][n_vox]      final step multiplier 2^(e/4) (1 without adaptation).
 * Moments of n = 0 values are NaN; the SD of one value is 0.
 * Returns 0, or -1 on invalid arguments; *threads_used = OpenMP threads. */
int orc_mcmc_run(const orc_model *m, const float *data, int64_t n_vox, const float *sigma,
                 float sigma_scalar, const float *x0, const orc_opts *o, double *mean,
                 double *std, double *samples, double *accept_rate, int32_t *nonfinite,
                 double *rhat, double *step_scale, int *threads_used) {
    int P = m->n_par;
    if (P != orc_n_par(m->kind) || P > 64 || o->n_chains < 1 || o->iterations < 0 ||
        o->burnin < 0 || o->thin < 1 || n_vox < 0 || o->adapt_window < 0 ||
        (o->adapt_window > 0 && !(o->adapt_target > 0.0 && o->adapt_target < 1.0)))
        return -1;
    int M = orc_n_meas(m->kind, m->n_acq);
    int C = o->n_chains, I = o->iterations, B = o->burnin;
    int S = orc_n_samples(I, B, o->thin);
    int per_chain = (o->moments_mode == 1) ? (I > B ? I - B : 0) : S;
    int nt = 1;
#ifdef _OPENMP
    nt = o->n_threads > 0 ? o->n_threads : omp_get_max_threads();
#endif
    if (threads_used) *threads_used = nt;

#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t v = 0; v < n_vox; ++v) {
        const float *y = data + (size_t)v * M;
        double sig = sigma ? (double)sigma[v] : (double)sigma_scalar;
        uint32_t vg = (uint32_t)(o->voxel_base + (uint64_t)v);
        size_t n_all = (size_t)C * per_chain;
        double *pooled = (double *)malloc(sizeof(double) * (n_all * P + 1));
        for (int c = 0; c < C; ++c) {
            const float *x0v = x0 ? x0 + ((size_t)v * C + c) * P : NULL;
            run_chain(m, y, sig, x0v, o, vg, (uint32_t)c, v, n_vox, samples,
                      pooled + (size_t)c * per_chain * P, per_chain, accept_rate, nonfinite,
                      step_scale, NULL);
        }
        pooled_moments(pooled, C, per_chain, P, v, n_vox, mean, std, rhat);
        free(pooled);
    }
    return 0;
}

/* The whole path of one chain (state after each iteration, [I+1][P]), for
 * tests of the thinning grid and of the sampler's stationary distribution. */
int orc_chain_path(const orc_model *m, const float *y, double sigma, const float *x0,
                   const orc_opts *o, uint64_t voxel, int chain, double *path,
                   double *accept_rate, double *step_scale) {
    if (m->n_par != orc_n_par(m->kind) || m->n_par > 64 || o->iterations < 0 ||
        o->adapt_window < 0 || (o->adapt_window > 0 && !(o->adapt_target > 0.0 && o->adapt_target < 1.0)))
        return -1;
    orc_opts one = *o;
    one.n_chains = chain + 1;
    double acc = 0.0;
    int32_t bad = 0;
    /* accept_rate/nonfinite are indexed [c][v] with n_vox = 1, v = 0 */
    double acc_buf[256], scale_buf[256];
    int32_t bad_buf[256];
    if (chain >= 256) return -1;
    run_chain(m, y, sigma, x0, &one, (uint32_t)(o->voxel_base + voxel), (uint32_t)chain, 0, 1,
              NULL, NULL, 0, acc_buf, bad_buf, scale_buf, path);
    acc = acc_buf[chain];
    if (step_scale) *step_scale = scale_buf[chain];
    bad = bad_buf[chain];
    (void)bad;
    if (accept_rate) *accept_rate = acc;
    return 0;
}

/* Lock-step acceptance check: for each recorded step n, recompute in FP64 the
 * likelihoods of the current state theta[n] and the proposal prop[n] (each
 * [n][P]) and the decision log u01(w_acc[n]) < L' - L. */
int orc_lockstep(const orc_model *m, const float *y, double sigma, int64_t n,
                 const double *theta, const double *prop, const uint32_t *w_acc, double *L,
                 double *Lp, int32_t *accept) {
    int P = m->n_par;
    for (int64_t i = 0; i < n; ++i) {
        double l0 = orc_loglik(m->kind, m->acq, m->n_acq, theta + (size_t)i * P, y, sigma);
        double l1 = orc_loglik(m->kind, m->acq, m->n_acq, prop + (size_t)i * P, y, sigma);
        if (L) L[i] = l0;
        if (Lp) Lp[i] = l1;
        if (accept) accept[i] = log(orc_u01(w_acc[i])) < l1 - l0;
    }
    return 0;
}

/* Forward model over many parameter vectors: theta [n][P] -> s [n][M]. */
int orc_forward_many(int kind, const double *acq, int n_acq, int64_t n, const double *theta,
                     double *s) {
    int P = orc_n_par(kind), M = orc_n_meas(kind, n_acq);
    if (P < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_forward(kind, acq, n_acq, theta + (size_t)i * P, s + (size_t)i * M);
    return 0;
}

/* Log-likelihood over many (theta, voxel) pairs: theta [n][P], y [n][M], sigma [n]. */
int orc_loglik_many(int kind, const double *acq, int n_acq, int64_t n, const double *theta,
                    const float *y, const float *sigma, double *L) {
    int P = orc_n_par(kind), M = orc_n_meas(kind, n_acq);
    if (P < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        L[i] = orc_loglik(kind, acq, n_acq, theta + (size_t)i * P, y + (size_t)i * M, (double)sigma[i]);
    return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Words of many draws: out [n][nw] for (t[i], v[i], c[i]). */
int orc_words_many(uint64_t seed, const uint32_t *t, const uint32_t *v, const uint32_t *c,
                   int64_t n, int nw, uint32_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_words(seed, t[i], v[i], c[i], nw, out + (size_t)i * nw);
    return 0;
}

/* Proposal normals of many draws: words [n][nw] -> z [n][P]. */
int orc_normals_many(const uint32_t *words, int64_t n, int nw, int n_par, double *z) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) orc_normals_from_words(words + (size_t)i * nw, n_par, z + (size_t)i * n_par);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Affine-invariant ensemble sampler (the paper's second mcmc.m algorithm,   */
/* Sec. 2.2.2: Nwalkers walkers, one stepSize for all parameters).           */
/* Goodman & Weare's stretch move (CAMCoS 5, 2010) with the two-halves       */
/* parallel update of Foreman-Mackey et al. (PASP 125, 2013):                */
/*   walkers 0..L/2-1 form half 0, L/2..L-1 half 1; iteration t moves every  */
/*   walker of half 0 against the current half 1, then every walker of       */
/*   half 1 against the updated half 0.                                      */
/* Walker k draws one Philox call, counter (t, voxel, k<<8, 0):              */
/*   word 0 picks its partner j in the other half, j = floor(w0 (L/2) 2^-32);*/
/*   word 1 gives the stretch z = ((a-1) u + 1)^2 / a, u = u01(w1), whose    */
/*   density is proportional to 1/sqrt(z) on [1/a, a] (a = stepSize);        */
/*   word 2 is the acceptance uniform.                                       */
/* Proposal Y = X_j + z (X_k - X_j).  Y outside the prior box has prior 0    */
/* and is rejected; otherwise accept iff log u < (P-1) log z + L(Y) - L(X_k).*/
/* Thinning, moments and outputs are those of the MH sampler, with walkers   */
/* in place of chains.                                                       */
/* ------------------------------------------------------------------------ */

/* Stretch factor from a word: inverse CDF of g(z) ~ 1/sqrt(z) on [1/a, a]. */
double orc_stretch_z(uint32_t w, double a) {
    double s = (a - 1.0) * orc_u01(w) + 1.0;
    return s * s / a;
}

static void ensemble_voxel(const orc_model *m, const float *y, double sigma, const float *x0v,
                           const orc_opts *o, double a, uint32_t vg, int64_t v, int64_t n_vox,
                           double *samples, double *pooled, int per_chain, double *accept_rate,
                           int32_t *nonfinite, double *path) {
    int P = m->n_par, L = o->n_chains, H = L / 2, I = o->iterations, B = o->burnin, T = o->thin;
    int S = orc_n_samples(I, B, T);
    double *X = (double *)malloc(sizeof(double) * (size_t)L * P);
    double *LL = (double *)malloc(sizeof(double) * L);
    long *acc = (long *)calloc((size_t)L, sizeof(long));
    long *bad = (long *)calloc((size_t)L, sizeof(long));
    int *npool = (int *)calloc((size_t)L, sizeof(int));
    uint32_t w[64];
    double Yp[64];

    for (int k = 0; k < L; ++k) {
        double *xk = X + (size_t)k * P;
        if (x0v) {
            for (int p = 0; p < P; ++p) xk[p] = clampd((double)x0v[(size_t)k * P + p], m->lb[p], m->ub[p]);
        } else {
            orc_words(o->seed, ORC_INIT_ITER, vg, (uint32_t)k, P, w);
            for (int p = 0; p < P; ++p) xk[p] = m->lb[p] + (m->ub[p] - m->lb[p]) * orc_u01(w[p]);
        }
        LL[k] = orc_loglik(m->kind, m->acq, m->n_acq, xk, y, sigma);
    }
    if (path) memcpy(path, X, sizeof(double) * (size_t)L * P);
    for (int t = 1; t <= I; ++t) {
        for (int h = 0; h < 2; ++h) {
            int other = (1 - h) * H;
            for (int i = 0; i < H; ++i) {
                int k = h * H + i;
                orc_words(o->seed, (uint32_t)t, vg, (uint32_t)k, 3, w);
                int j = other + (int)(((uint64_t)w[0] * (uint64_t)H) >> 32);
                double z = orc_stretch_z(w[1], a);
                const double *xk = X + (size_t)k * P, *xj = X + (size_t)j * P;
                int inside = 1;
                for (int p = 0; p < P; ++p) {
                    Yp[p] = xj[p] + z * (xk[p] - xj[p]);
                    if (!(Yp[p] >= m->lb[p] && Yp[p] <= m->ub[p])) inside = 0;
                }
                if (!inside) continue;
                double Ly = orc_loglik(m->kind, m->acq, m->n_acq, Yp, y, sigma);
                if (!isfinite(Ly)) ++bad[k];
                double log_u = log(orc_u01(w[2]));
                if (log_u < (double)(P - 1) * log(z) + Ly - LL[k]) {
                    memcpy(X + (size_t)k * P, Yp, sizeof(double) * P);
                    LL[k] = Ly;
                    ++acc[k];
                }
            }
        }
        if (path) memcpy(path + (size_t)t * L * P, X, sizeof(double) * (size_t)L * P);
        int on_grid = (t > B) && ((t - B) % T == 0);
        int take = (o->moments_mode == 1) ? (t > B) : on_grid;
        for (int k = 0; k < L; ++k) {
            const double *xk = X + (size_t)k * P;
            if (on_grid && samples) {
                int idx = (t - B) / T - 1;
                if (idx < S)
                    for (int p = 0; p < P; ++p) samples[(((size_t)idx * L + k) * P + p) * n_vox + v] = xk[p];
            }
            if (take && pooled && npool[k] < per_chain) {
                double *blk = pooled + (size_t)k * per_chain * P;
                for (int p = 0; p < P; ++p) blk[(size_t)p * per_chain + npool[k]] = xk[p];
                ++npool[k];
            }
        }
    }
    for (int k = 0; k < L; ++k) {
        if (accept_rate) accept_rate[(size_t)k * n_vox + v] = I > 0 ? (double)acc[k] / (double)I : 0.0;
        if (nonfinite) nonfinite[(size_t)k * n_vox + v] = (int32_t)bad[k];
    }
    free(X); free(LL); free(acc); free(bad); free(npool);
}

/* Ensemble run over n_vox voxels; o->n_chains = walkers L (even, >= 4),
 * a = stepSize > 1.  Same inputs and outputs as orc_mcmc_run. */
int orc_ensemble_run(const orc_model *m, const float *data, int64_t n_vox, const float *sigma,
                     float sigma_scalar, const float *x0, const orc_opts *o, double a, double *mean,
                     double *std, double *samples, double *accept_rate, int32_t *nonfinite,
                     int *threads_used) {
    int P = m->n_par;
    if (P != orc_n_par(m->kind) || P > 64 || o->n_chains < 4 || (o->n_chains & 1) ||
        o->n_chains > 256 || o->iterations < 0 || o->burnin < 0 || o->thin < 1 || n_vox < 0 || !(a > 1.0))
        return -1;
    int M = orc_n_meas(m->kind, m->n_acq);
    int L = o->n_chains, I = o->iterations, B = o->burnin;
    int S = orc_n_samples(I, B, o->thin);
    int per_chain = (o->moments_mode == 1) ? (I > B ? I - B : 0) : S;
    int nt = 1;
#ifdef _OPENMP
    nt = o->n_threads > 0 ? o->n_threads : omp_get_max_threads();
#endif
    if (threads_used) *threads_used = nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t v = 0; v < n_vox; ++v) {
        size_t n_all = (size_t)L * per_chain;
        double *pooled = (double *)malloc(sizeof(double) * (n_all * P + 1));
        ensemble_voxel(m, data + (size_t)v * M, sigma ? (double)sigma[v] : (double)sigma_scalar,
                       x0 ? x0 + (size_t)v * L * P : NULL, o, a,
                       (uint32_t)(o->voxel_base + (uint64_t)v), v, n_vox, samples, pooled, per_chain,
                       accept_rate, nonfinite, NULL);
        pooled_moments(pooled, L, per_chain, P, v, n_vox, mean, std, NULL);
        free(pooled);
    }
    return 0;
}

/* Every walker's state after each iteration t = 0..I of one voxel: path
 * [I+1][L][P]. */
int orc_ensemble_path(const orc_model *m, const float *y, double sigma, const float *x0v,
                      const orc_opts *o, double a, uint64_t voxel, double *path, double *accept_rate) {
    if (m->n_par != orc_n_par(m->kind) || o->n_chains < 4 || (o->n_chains & 1) || !(a > 1.0)) return -1;
    ensemble_voxel(m, y, sigma, x0v, o, a, (uint32_t)(o->voxel_base + voxel), 0, 1, NULL, NULL, 0,
                   accept_rate, NULL, path);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole-volume gradient fit (askadam.m, Sec. 2.2.1, Eq. 2, 4, 5)            */
/* ------------------------------------------------------------------------ */

/* dg/dx of g(x) = int_0^1 exp(-x u^2) du: -int_0^1 u^2 exp(-x u^2) du, which
 * integration by parts turns into (exp(-x) - g(x)) / (2x); for |x| <= 1 the
 * term-wise derivative of the power series, sum_n n (-x)^(n-1) (-1) / (n! (2n+1)). */
double orc_dg(double x) {
    if (fabs(x) > 1.0) return (exp(-x) - orc_g(x)) / (2.0 * x);
    double term = 1.0; /* (-x)^(n-1) / (n-1)! */
    double sum = 0.0;
    for (int n = 1; n < 400; ++n) {
        if (n > 1) term *= -x / (double)(n - 1);
        double add = -term / (double)(2 * n + 1);
        sum += add;
        if (fabs(add) <= 1e-18 * fabs(sum)) break;
    }
    return sum;
}

/* Forward model s [M] and its Jacobian J [M][P] (J[m][p] = ds_m / dtheta_p),
 * differentiated by hand from the forms of orc_forward (MONOEXP, MWI3, SMT,
 * LINEAR).  Returns 0, or -1 for a kind without a Jacobian. */
int orc_jacobian(int kind, const double *acq, int n_acq, const double *theta, double *s, double *J) {
    int P = orc_n_par(kind);
    if (orc_forward(kind, acq, n_acq, theta, s) != 0) return -1;
    switch (kind) {
    case ORC_MONOEXP:
        for (int k = 0; k < n_acq; ++k) {
            double decay = exp(-1e-3 * acq[k] * theta[1]);
            J[k * P + 0] = decay;
            J[k * P + 1] = -1e-3 * acq[k] * theta[0] * decay;
        }
        return 0;
    case ORC_MWI3:
        for (int k = 0; k < n_acq; ++k) {
            double tk = acq[k];
            double *Jr = J + (size_t)(2 * k) * P, *Ji = J + (size_t)(2 * k + 1) * P;
            for (int p = 0; p < P; ++p) Jr[p] = Ji[p] = 0.0;
            for (int j = 0; j < 3; ++j) {
                double decay = exp(-tk / theta[3 + j]);
                double dfj = j < 2 ? theta[6 + j] : 0.0;
                double phase = theta[8] - 2.0 * ORC_PI * 1e-3 * dfj * tk;
                double c = cos(phase), sn = sin(phase);
                double amp = theta[j] * decay;
                Jr[j] = decay * c; /* d/dA_j */
                Ji[j] = decay * sn;
                double dT = amp * tk / (theta[3 + j] * theta[3 + j]); /* d/dT2*_j */
                Jr[3 + j] = dT * c;
                Ji[3 + j] = dT * sn;
                if (j < 2) { /* d phase / d df = -2 pi t 1e-3 */
                    double w = 2.0 * ORC_PI * 1e-3 * tk;
                    Jr[6 + j] = amp * w * sn;
                    Ji[6 + j] = -amp * w * c;
                }
            }
            Jr[8] = -s[2 * k + 1]; /* d/dphi0 of S: i S */
            Ji[8] = s[2 * k];
        }
        return 0;
    case ORC_SMT:
        for (int k = 0; k < n_acq; ++k) {
            double bk = acq[k];
            double f = theta[0], da = theta[1], dpar = theta[2], dperp = theta[3];
            double g_in = orc_g(bk * da), ex = exp(-bk * dperp), g_ex = orc_g(bk * (dpar - dperp));
            double dg_ex = orc_dg(bk * (dpar - dperp));
            J[k * P + 0] = g_in - ex * g_ex;
            J[k * P + 1] = f * bk * orc_dg(bk * da);
            J[k * P + 2] = (1.0 - f) * ex * bk * dg_ex;
            J[k * P + 3] = -(1.0 - f) * bk * ex * (g_ex + dg_ex);
        }
        return 0;
    case ORC_LINEAR:
        for (int k = 0; k < n_acq; ++k) {
            J[k * P + 0] = 1.0;
            J[k * P + 1] = acq[k];
        }
        return 0;
    default:
        return -1;
    }
}

/* Least-squares slope of y[0..n-1] against 0..n-1. */
double orc_window_slope(const double *y, int n) {
    double xm = 0.5 * (n - 1), ym = 0.0, sxy = 0.0, sxx = 0.0;
    for (int i = 0; i < n; ++i) ym += y[i];
    ym /= n;
    for (int i = 0; i < n; ++i) {
        sxy += (i - xm) * (y[i] - ym);
        sxx += (i - xm) * (i - xm);
    }
    return sxx > 0.0 ? sxy / sxx : 0.0;
}

typedef struct {
    int nx, ny, nz;         /* voxel grid, N = nx ny nz, voxel v = x + nx (y + ny z) */
    int loss;               /* 1: L1, 2: L2 */
    int iterations;         /* maximum number of updates */
    double lr, beta1, beta2, eps;   /* Adam (Kingma & Ba) */
    double tol;             /* stop once the loss is below tol (0: off) */
    double conv_value;      /* stop once |slope| of the last conv_window losses < conv_value (0: off) */
    int conv_window;
    double lambda;          /* total-variation weight (Eq. 4) */
    uint32_t tv_params;     /* bit p: total variation on parameter p */
    int tv_dims;            /* 2 or 3 (x, y[, z]) */
} orc_fit_opts;

static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

/* Adam on the whole volume.  The optimiser works on normalised parameters
 * u = (theta - lb) / (ub - lb), clamped to [0, 1] after every update.  The
 * loss at iteration t, evaluated at the current parameters, is
 *   D = (1 / (n_mask M)) sum_{v in mask} sum_m rho(w_v (y_vm - s_vm)),
 *       rho = |r| (L1) or r^2 (L2)                                   (Eq. 2)
 *   + (lambda / n_mask) sum_{p in tv} sum_{v, v + e_d in mask} |u_p(v + e_d) - u_p(v)|
 *                                                                   (Eq. 4, 5)
 * with subgradient sign(0) = 0; then the Adam step (bias-corrected moments)
 * updates every masked voxel.  After the update the loop stops if the loss is
 * below tol, or if t >= conv_window and the least-squares slope of the last
 * conv_window losses is below conv_value in magnitude.  theta [N][P] holds the
 * initial parameters on entry and the fitted ones on return; loss_hist[t-1]
 * receives the loss of iteration t; *iters_done the number of updates. */
int orc_fit_run(const orc_model *m, const float *data, const uint8_t *mask, const float *weight,
                const orc_fit_opts *o, double *theta, double *loss_hist, int *iters_done) {
    int P = m->n_par, M = orc_n_meas(m->kind, m->n_acq);
    int64_t N = (int64_t)o->nx * o->ny * o->nz;
    if (P != orc_n_par(m->kind) || M < 1 || N < 1 || (o->loss != 1 && o->loss != 2) || o->iterations < 0 ||
        (o->tv_dims != 2 && o->tv_dims != 3) || M > 512)
        return -1;
    double *u = (double *)malloc(sizeof(double) * N * P);
    double *mom1 = (double *)calloc((size_t)N * P, sizeof(double));
    double *mom2 = (double *)calloc((size_t)N * P, sizeof(double));
    double *grad = (double *)malloc(sizeof(double) * N * P);
    double *hist = (double *)malloc(sizeof(double) * (o->iterations + 1));
    if (!u || !mom1 || !mom2 || !grad || !hist) return -1;
    int64_t n_mask = 0;
    for (int64_t v = 0; v < N; ++v) n_mask += mask ? (mask[v] != 0) : 1;
    for (int64_t v = 0; v < N; ++v)
        for (int p = 0; p < P; ++p) {
            double range = m->ub[p] - m->lb[p];
            u[v * P + p] = range > 0.0 ? (theta[v * P + p] - m->lb[p]) / range : 0.0;
        }
    int done = 0;
    for (int t = 1; t <= o->iterations; ++t) {
        double data_loss = 0.0, tv_loss = 0.0;
        /* data term and its gradient, voxel by voxel */
        for (int64_t v = 0; v < N; ++v) {
            for (int p = 0; p < P; ++p) grad[v * P + p] = 0.0;
            if (mask && !mask[v]) continue;
            double th[64], s[512], J[512 * 12];
            for (int p = 0; p < P; ++p) th[p] = m->lb[p] + u[v * P + p] * (m->ub[p] - m->lb[p]);
            orc_jacobian(m->kind, m->acq, m->n_acq, th, s, J);
            double w = weight ? (double)weight[v] : 1.0;
            for (int k = 0; k < M; ++k) {
                double r = w * ((double)data[v * M + k] - s[k]);
                double drho_ds = (o->loss == 1) ? -w * sgn(r) : -2.0 * w * r;
                data_loss += (o->loss == 1) ? fabs(r) : r * r;
                for (int p = 0; p < P; ++p) grad[v * P + p] += drho_ds * J[k * P + p];
            }
        }
        double scale = 1.0 / ((double)n_mask * M);
        for (int64_t v = 0; v < N; ++v)
            for (int p = 0; p < P; ++p) grad[v * P + p] *= scale * (m->ub[p] - m->lb[p]); /* d/du */
        data_loss *= scale;
        /* total variation over pairs of neighbouring masked voxels */
        for (int p = 0; p < P && o->lambda != 0.0; ++p) {
            if (!((o->tv_params >> p) & 1u)) continue;
            for (int64_t v = 0; v < N; ++v) {
                if (mask && !mask[v]) continue;
                int x = (int)(v % o->nx), y = (int)((v / o->nx) % o->ny), z = (int)(v / ((int64_t)o->nx * o->ny));
                int nb[3] = {x + 1 < o->nx, y + 1 < o->ny, z + 1 < o->nz};
                int64_t step[3] = {1, o->nx, (int64_t)o->nx * o->ny};
                for (int d = 0; d < o->tv_dims; ++d) {
                    if (!nb[d]) continue;
                    int64_t w2 = v + step[d];
                    if (mask && !mask[w2]) continue;
                    double diff = u[w2 * P + p] - u[v * P + p];
                    tv_loss += fabs(diff);
                    grad[w2 * P + p] += o->lambda / (double)n_mask * sgn(diff);
                    grad[v * P + p] -= o->lambda / (double)n_mask * sgn(diff);
                }
            }
        }
        double loss = data_loss + o->lambda / (double)n_mask * tv_loss;
        /* Adam */
        double c1 = 1.0 - pow(o->beta1, t), c2 = 1.0 - pow(o->beta2, t);
        for (int64_t v = 0; v < N; ++v) {
            if (mask && !mask[v]) continue;
            for (int p = 0; p < P; ++p) {
                size_t i = (size_t)v * P + p;
                mom1[i] = o->beta1 * mom1[i] + (1.0 - o->beta1) * grad[i];
                mom2[i] = o->beta2 * mom2[i] + (1.0 - o->beta2) * grad[i] * grad[i];
                double step_u = o->lr * (mom1[i] / c1) / (sqrt(mom2[i] / c2) + o->eps);
                u[i] = fmin(fmax(u[i] - step_u, 0.0), 1.0);
            }
        }
        hist[t - 1] = loss;
        if (loss_hist) loss_hist[t - 1] = loss;
        done = t;
        if (o->tol > 0.0 && loss < o->tol) break;
        if (o->conv_value > 0.0 && o->conv_window > 1 && t >= o->conv_window &&
            fabs(orc_window_slope(hist + t - o->conv_window, o->conv_window)) < o->conv_value)
            break;
    }
    for (int64_t v = 0; v < N; ++v) /* voxels outside the mask keep their initial parameters */
        if (!mask || mask[v])
            for (int p = 0; p < P; ++p) theta[v * P + p] = m->lb[p] + u[v * P + p] * (m->ub[p] - m->lb[p]);
    if (iters_done) *iters_done = done;
    free(hist);
    free(u);
    free(mom1);
    free(mom2);
    free(grad);
    return 0;
}
