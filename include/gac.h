/*
 * gac.h -- C ABI of libgac.so: GB300-native voxel-wise Metropolis-Hastings
 * sampling of qMRI forward models (the hot path of GACELLE's mcmc.m, Chan et
 * al., arXiv 2511.22094, Sec. 2.2.2).
 *
 * Conventions for every entry point
 *   - Every function returns a gac_status; nothing aborts or exits.  On a
 *     status other than GAC_OK, gac_last_error() returns a message for the
 *     calling thread, and output buffers may have been partially written only
 *     where the description says so.
 *   - Array pointers may be host or device memory; the library asks CUDA
 *     which (cudaPointerGetAttributes).  Host buffers are staged through
 *     device memory the library allocates and frees within the call.  Device
 *     buffers are used in place and must stay valid until the call returns.
 *   - Inputs are owned by the caller and only read during the call;
 *     gac_model_register and gac_server_submit copy what they keep.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are synchronous with respect to the host: when one returns GAC_OK its
 *     results are in the caller's buffers.
 *   - All layouts are C order (last index fastest).
 */
#ifndef GAC_H
#define GAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GAC_OK = 0,
    GAC_ERR_INVALID_ARG = 1,   /* a pointer, size, bound or option is invalid */
    GAC_ERR_UNKNOWN_MODEL = 2, /* model_id / kind not registered or not known */
    GAC_ERR_BUDGET = 3,        /* serving: a job larger than the whole HBM budget */
    GAC_ERR_OOM = 4,           /* device allocation failed */
    GAC_ERR_CUDA = 5,          /* a CUDA call failed (message names it) */
    GAC_ERR_TIMEOUT = 6,       /* a bounded wait expired */
    GAC_ERR_NOT_READY = 7,     /* reserved */
    GAC_ERR_CANCELLED = 8,     /* serving: the job was cancelled */
    GAC_ERR_UNKNOWN_JOB = 9    /* serving: no such job id */
} gac_status;

/* Forward signal models (Sec. 2.1 model list; Eq. 3).  Parameter order and
 * units:
 *  MONOEXP (Eq. 3)  s_k = S0 exp(-R2* TE_k).  theta = (S0, R2* [1/s]),
 *                   acq = TE [ms].  2 parameters, n_acq real measurements.
 *  MWI3   3-pool complex multi-echo GRE myelin-water model
 *         S(t) = exp(i phi0) sum_{j=MW,IW,EW} A_j exp(-t/T2*_j) exp(-i 2 pi df_j t),
 *         df_EW = 0.  theta = (A_MW, A_IW, A_EW, T2*_MW, T2*_IW, T2*_EW [ms],
 *         df_MW, df_IW [Hz], phi0 [rad]); acq = TE [ms].  9 parameters,
 *         2*n_acq real measurements (re, im interleaved per echo).
 *  SMT    spherical-mean Standard Model, S(b=0) = 1:
 *         s(b) = f g(b Da) + (1-f) exp(-b De_perp) g(b (De_par - De_perp)),
 *         g(x) = integral_0^1 exp(-x u^2) du.  theta = (f, Da, De_par, De_perp)
 *         [um^2/ms]; acq = b [ms/um^2].  4 parameters, n_acq measurements.
 *         Registration requires b >= 0 and b*(ub[De_perp] - lb[De_par]) <= 12.
 *  LINEAR_TEST  s_k = a + c t_k, theta = (a, c), acq = t (a test model whose
 *         posterior is known exactly). */
typedef enum {
    GAC_MODEL_MONOEXP = 1,
    GAC_MODEL_MWI3 = 2,
    GAC_MODEL_SMT = 3,
    GAC_MODEL_AXCAL_SMT = 4,
    GAC_MODEL_LINEAR_TEST = 100
} gac_model_kind;

#define GAC_MAX_PAR 12
#define GAC_MAX_ACQ 64
#define GAC_MAX_MODELS 4096

typedef struct {
    int kind;           /* gac_model_kind */
    int n_acq;          /* echoes or b-values, 1..GAC_MAX_ACQ */
    const double *acq;  /* host [n_acq]: TE [ms], b [ms/um^2] or t */
    int n_par;          /* must equal the kind's parameter count */
    const double *lb;   /* host [n_par]: uniform-prior lower bounds */
    const double *ub;   /* host [n_par]: upper bounds, ub >= lb */
    const double *step; /* host [n_par]: proposal SD per parameter (xStepSize), >= 0 */
} gac_model_desc;

/* Registers a forward model with its acquisition parameters, prior bounds and
 * proposal steps (Sec. 2.3.1: users supply the forward model, bounds and
 * options; Sec. 2.2.2: xStepSize).  Copies every array.  Single-precision
 * paths round acq/lb/ub/step to float.  Returns a model id >= 1 in *model_id;
 * registering a description equal to an earlier one returns the earlier id.
 * Errors: INVALID_ARG (NULL, sizes, lb > ub, negative step, non-finite
 * values, SMT range), UNKNOWN_MODEL (kind), and INVALID_ARG when
 * GAC_MAX_MODELS distinct models are registered already.  Thread-safe. */
gac_status gac_model_register(const gac_model_desc *desc, int *model_id);

/* Parameter count and real measurements per voxel of a registered model. */
gac_status gac_model_info(int model_id, int *n_par, int *n_meas);

/* Arithmetic of the sampler.  MIXED (default): forward model and residuals in
 * FP32, the likelihood summed in FP32 within blocks of six acquisitions and
 * the block sums added with Kahan's compensation, the acceptance decision
 * taken with FP64 semantics, FP64 moment accumulators.  FP32: everything in
 * FP32, plain sums.  FP64: everything in FP64. */
enum { GAC_PREC_MIXED = 0, GAC_PREC_FP32 = 1, GAC_PREC_FP64 = 2 };
/* What the posterior moments average: the thinned samples (default, as the
 * paper's output) or every post-burn-in state.  On the MIXED path the latter
 * sums the states of each block of 64 consecutive post-burn-in iterations in
 * FP32, as deviations from the block's first state, and merges each block
 * into the FP64 accumulators (pairwise update of count, mean and M2); the
 * result agrees with a per-state FP64 update to the FP32 rounding of the
 * block sums (~1e-7 of the posterior SD). */
enum { GAC_MOMENTS_THINNED = 0, GAC_MOMENTS_ALL_POSTBURNIN = 1 };

typedef struct {
    int iterations;      /* I >= 0 (the `iteration` option, Sec. 2.2.2) */
    int burnin;          /* B >= 0, a count (the paper's ratio r is floor(r*I)) */
    int thin;            /* T >= 1 (`thinning`) */
    int n_chains;        /* C, 1..64 (Table 1: "4 independent proposals") */
    uint64_t seed;       /* Philox key */
    uint64_t voxel_base; /* global index of voxel 0 in the RNG counter; lets a
                            volume split into pieces reproduce the whole run */
    int precision;       /* GAC_PREC_* */
    int moments_mode;    /* GAC_MOMENTS_* */
    int trace_n_vox;     /* >0: record every step of the chains of voxels
                            [0, trace_n_vox) into gac_result.trace */
    int adapt_window;    /* 0 (default): fixed steps, as in the paper.  W > 0:
                            adapt each chain's steps during burn-in (below) */
    double adapt_target; /* target acceptance rate of the adaptation, in (0, 1) */
    int lanes_per_chain; /* gac_mcmc_run only (other entry points ignore it).
                            0 (default): the library chooses; 1: one thread per
                            chain; 2 or 4: that many lanes of a warp per chain,
                            each evaluating one block of six echoes, the block
                            sums combined by warp shuffles (MIXED precision,
                            mono-exponential or 3-pool model with evenly spaced
                            echoes in at most that many blocks, trace_n_vox 0;
                            GAC_ERR_INVALID_ARG otherwise).  Results do not
                            depend on it, bit for bit; the library uses lanes
                            when the chains are too few to give every SM
                            sub-partition a warp. */
} gac_mcmc_opts;

/* Step adaptation during burn-in (an extension; the paper has no
 * counterpart: its xStepSize steps are fixed).  Each chain proposes with
 * xStepSize * 2^(e/4) for an integer e starting at 0.  After each iteration t
 * with t % W == 0 and t <= B, with a = the proposals the chain accepted in
 * iterations t-W+1 .. t: e += 1 if a > adapt_target * W, e -= 1 if
 * a < adapt_target * W, kept within [GAC_ADAPT_EMIN, GAC_ADAPT_EMAX].  The
 * steps are fixed after burn-in, so the post-burn-in states are those of a
 * Metropolis-Hastings chain with a fixed proposal.  MH only. */
#define GAC_ADAPT_EMIN (-48)
#define GAC_ADAPT_EMAX 16

/* One recorded MH step (lock-step parity checks): state before the step,
 * the clamped proposal, both log-likelihoods, the acceptance word and the
 * decision.  Values are the kernel's own, widened to double. */
typedef struct {
    double theta[GAC_MAX_PAR];
    double prop[GAC_MAX_PAR];
    double L, Lp;
    uint32_t w_acc;
    int32_t accepted;
} gac_trace_rec;

/* Caller-allocated outputs; any pointer may be NULL to skip that output.
 * S = floor((I - B)/T) when I > B, else 0.  Moments of n = 0 values are NaN,
 * the SD of one value is 0. */
typedef struct {
    double *mean;         /* [P][N] posterior mean (out.mean.<p>, Sec. 2.3.1) */
    double *std;          /* [P][N] posterior SD, n-1 divisor (out.std.<p>) */
    float *samples;       /* [S][C][P][N] thinned states, t = B+T, B+2T, ... */
    float *accept_rate;   /* [C][N] accepted proposals / I */
    int32_t *nonfinite;   /* [C][N] steps whose proposal likelihood was not finite */
    gac_trace_rec *trace; /* [trace_n_vox][C][I] */
    double *rhat;         /* [P][N] R-hat of the C chains over the values that
                             enter the moments (Gelman & Rubin 1992, no
                             splitting): sqrt(((n-1)/n W + B/n) / W), W the
                             mean within-chain variance, B/n the variance of
                             the chain means.  NaN if C < 2 or n < 2 (and if
                             W = B = 0), +inf if W = 0 < B.  MH only. */
    float *step_scale;    /* [C][N] final step multiplier 2^(e/4) (1 without
                             adaptation).  MH only. */
} gac_result;

/* Bytes of each gac_result buffer in the order mean, std, samples,
 * accept_rate, nonfinite, trace, rhat, step_scale (bytes[8]). */
gac_status gac_result_sizes(int model_id, int64_t n_vox, const gac_mcmc_opts *opts,
                            size_t bytes[8]);

/* Runs C Metropolis-Hastings chains for each of n_vox voxels (Sec. 2.2.2):
 * per iteration a Gaussian random-walk proposal clamped to [lb, ub], the
 * forward model at all acquisitions, the Gaussian log-likelihood
 * L = -1/2 sum_m ((y_m - s_m)/sigma)^2, acceptance iff log u < L' - L, and on
 * the thinning grid a stored sample and a Welford moment update.
 *   data   [n_vox][n_meas] float32 (complex data as re, im pairs)
 *   sigma  [n_vox] float32 noise SD per real measurement, or NULL to use
 *          sigma_scalar for every voxel (must then be > 0)
 *   x0     [n_vox][C][P] float32 initial states (clamped into the bounds), or
 *          NULL for a uniform-prior draw from the RNG
 * Random numbers: Philox4x32-10 with counter (t, voxel_base + v,
 * c << 8 | call, 0) and key (seed lo, seed hi); t = 0xFFFFFFFF for the initial
 * draw.  Results depend only on (inputs, opts), not on the GPU's occupancy or
 * on how a volume is split (use voxel_base).  n_vox = 0 returns GAC_OK.
 * Errors: INVALID_ARG, UNKNOWN_MODEL, OOM, CUDA. */
gac_status gac_mcmc_run(int model_id, const void *data, int64_t n_vox, const float *sigma,
                        float sigma_scalar, const float *x0, const gac_mcmc_opts *opts,
                        gac_result *out, void *stream);

/* Forward model at n parameter vectors theta [n][P] (double) into s [n][M]
 * (double), using the same device arithmetic as the sampler for `precision`
 * (theta is rounded to float first on the FP32/MIXED paths).  Used to build
 * synthetic data and to test the forward model (Eq. 3 and the forms above). */
gac_status gac_forward(int model_id, const double *theta, int64_t n, int precision, double *s,
                       void *stream);

/* Log-likelihood L = -1/2 sum_m ((y_m - s_m(theta_i))/sigma_i)^2 of n
 * (theta_i, voxel i) pairs: theta [n][P] double, data [n][M] float32,
 * sigma [n] float32; L [n] double.  Same arithmetic as the sampler. */
gac_status gac_loglik(int model_id, const double *theta, int64_t n, const float *data,
                      const float *sigma, int precision, double *L, void *stream);

/* Test entry points of the random-number layer.
 * gac_philox_words: for i in [0, n): the n_words words of (t_i, v_i, c_i) for
 *   key `seed` -> out [n][n_words] (uint32); t, v, c are [n] uint32.
 * gac_normals: the P proposal normals of (t_i, v_i, c_i) as the sampler draws
 *   them (Box-Muller on words 2j, 2j+1) -> z [n][P] double, and the
 *   acceptance word -> w_acc [n]. */
gac_status gac_philox_words(uint64_t seed, const uint32_t *t, const uint32_t *v,
                            const uint32_t *c, int64_t n, int n_words, uint32_t *out,
                            void *stream);
gac_status gac_normals(uint64_t seed, const uint32_t *t, const uint32_t *v, const uint32_t *c,
                       int64_t n, int n_par, int precision, double *z, uint32_t *w_acc,
                       void *stream);

/* Pipe-rate probe (not part of the method: the denominators of the
 * sampler's arithmetic roofline, measured on the device).  Runs one kernel of
 * 4 blocks of 256 threads per SM, each thread 8 independent chains of 4096
 * dependent steps of operation `op`, after one warm-up launch, and writes the
 * median over SMs of results per SM clock (clock64 around each block's loop;
 * an SM's span runs from its first block's start to its last block's end).
 * FFMA2 counts two results per step.  Synchronises `stream`.  Errors:
 * GAC_ERR_INVALID_ARG for an unknown op or a NULL output, GAC_ERR_CUDA. */
typedef enum {
    GAC_PIPE_FFMA = 0,    /* fma.rn.f32 */
    GAC_PIPE_FFMA2 = 1,   /* paired FP32 fma (two results) */
    GAC_PIPE_EX2 = 2,     /* ex2.approx.ftz.f32 */
    GAC_PIPE_SIN = 3,     /* sin.approx.ftz.f32 (cos runs on the same unit) */
    GAC_PIPE_LG2 = 4,     /* lg2.approx.ftz.f32 */
    GAC_PIPE_RSQRT = 5,   /* rsqrt.approx.ftz.f32 */
    GAC_PIPE_RCP = 6,     /* rcp.approx.ftz.f32 */
    GAC_PIPE_SQRT = 7,    /* sqrt.approx.ftz.f32 */
    GAC_PIPE_DFMA = 8,    /* fma.rn.f64 */
    GAC_PIPE_IMAD_HI = 9, /* mad.hi.u32 (Philox's high products) */
    GAC_PIPE_LOP3 = 10    /* lop3.b32 (three-input xor) */
} gac_pipe_op;
gac_status gac_pipe_rate(int op, double *per_clk_sm, void *stream);

/* Affine-invariant ensemble sampler (the paper's second mcmc.m algorithm,
 * Sec. 2.2.2: Nwalkers walkers and one stepSize for all parameters; Table 1:
 * 50 walkers x 2000 iterations).  Goodman & Weare's stretch move with the
 * two-halves parallel update: walkers 0..L/2-1 move against the other half,
 * then walkers L/2..L-1 against the updated first half.  Walker k uses the
 * Philox call (t, voxel, k << 8, 0): word 0 picks its partner j in the other
 * half, word 1 the stretch z = ((a-1) u + 1)^2 / a (density ~ 1/sqrt(z) on
 * [1/a, a], a = `stretch`), word 2 the acceptance uniform.  The proposal
 * X_j + z (X_k - X_j) is rejected outside the prior box, otherwise accepted
 * iff log u < (P-1) log z + L(Y) - L(X_k).
 * Arguments, outputs and precision variants as gac_mcmc_run, with
 * opts->n_chains = L walkers (even, 4..128) in place of chains; x0 is
 * [n_vox][L][P]; step sizes of the registration are not used; trace records
 * hold L' = NaN for proposals outside the box.  INVALID_ARG for
 * opts->adapt_window != 0 or non-NULL out->rhat / out->step_scale (MH only). */
gac_status gac_ensemble_run(int model_id, const void *data, int64_t n_vox, const float *sigma,
                            float sigma_scalar, const float *x0, const gac_mcmc_opts *opts,
                            double stretch, gac_result *out, void *stream);

/* Whole-volume gradient fit (askadam.m, Sec. 2.2.1; Eq. 2, 4, 5): Adam over
 * all voxels of an nx x ny x nz grid (voxel v = x + nx (y + ny z)) at once.
 * The optimiser works on normalised parameters u = (theta - lb) / (ub - lb),
 * clamped to [0, 1] after every update.  Iteration t evaluates, at the
 * current parameters, the loss
 *   (1 / (n_mask M)) sum_{v in mask} sum_m rho(w_v (y_vm - s_vm)),
 *       rho(r) = |r| (L1) or r^2 (L2),
 *   + (tv_lambda / n_mask) sum_{p in tv_params} sum_{d < tv_dims}
 *       sum_{v, v + e_d in mask} |u_p(v + e_d) - u_p(v)|
 * and its (sub)gradient (sign(0) = 0), takes one Adam step (bias-corrected
 * moments, learning_rate, beta1, beta2, epsilon), records the loss, and
 * stops if the loss < tol (tol > 0) or if t >= convergence_window and the
 * least-squares slope of the last convergence_window losses is below
 * convergence_value in magnitude (convergence_value > 0).  Models: mono-
 * exponential, 3-pool, Standard Model and the linear test model (analytic
 * Jacobians); AxCaliberSMT is rejected. */
enum { GAC_FIT_L1 = 1, GAC_FIT_L2 = 2 };
typedef struct {
    int nx, ny, nz;
    int loss;                 /* GAC_FIT_L1 | GAC_FIT_L2 */
    int iterations;           /* maximum number of updates */
    double learning_rate, beta1, beta2, epsilon;
    double tol;
    double convergence_value;
    int convergence_window;   /* 2..4096 when convergence_value > 0 */
    double tv_lambda;
    uint32_t tv_params;       /* bit p: total variation on parameter p */
    int tv_dims;              /* 2 (x, y) or 3 (x, y, z) */
    int precision;            /* GAC_PREC_FP32 or GAC_PREC_FP64 */
} gac_fit_opts;

/*   data     [N][n_meas] float32 (host or device)
 *   mask     [N] uint8 (nonzero = fitted) or NULL for every voxel
 *   weight   [N] float32 w_v or NULL for 1
 *   theta    [N][P] double: initial parameters in, fitted parameters out
 *            (voxels outside the mask keep theirs)
 *   loss_history [iterations] double or NULL: the loss of each iteration
 *   *iterations_done: the number of updates taken
 * Synchronous.  Errors: INVALID_ARG (also for grids of 2^31 / P voxels or more:
 * the kernels index [P][N] arrays with 32 bits), UNKNOWN_MODEL, OOM, CUDA. */
gac_status gac_fit_run(int model_id, const void *data, const uint8_t *mask, const float *weight,
                       const gac_fit_opts *opts, double *theta, double *loss_history, int *iterations_done,
                       void *stream);

/* Allocation-free variant of gac_mcmc_run.  The paper has no counterpart to
 * this entry point; it exists for callers that cannot allocate device
 * memory: an application that has handed the GPU's memory to its own pool
 * (a deep-learning framework's caching allocator, an on-scanner
 * reconstruction pipeline with a fixed memory plan), or a latency-critical
 * loop that must not pay the device-wide synchronisation that cudaMalloc and
 * cudaFree imply.  It allocates nothing: it runs the same sampler in slices
 * of slice_iterations iterations (one kernel launch each) and keeps the
 * chains' state between slices in one fixed array of
 * GAC_NOALLOC_STATE_BYTES that the library holds in device memory on every
 * GPU where it is loaded, until the process exits.
 *   - Every array (data, sigma, x0 and the result buffers) must be device
 *     memory; host pointers are rejected with GAC_ERR_INVALID_ARG.
 *   - The chain state needs about (20 P + 20) bytes per chain (P parameters),
 *     32 P + 20 with moments over every post-burn-in state (the FP32 block
 *     partials of that mode are carried between slices): n_vox * n_chains
 *     must stay within GAC_NOALLOC_STATE_BYTES of it (e.g. ~335,000 chains
 *     of the 9-parameter model); larger runs are rejected with
 *     GAC_ERR_INVALID_ARG and a message giving the limit.
 *   - precision must be GAC_PREC_MIXED and trace_n_vox 0; results equal
 *     gac_mcmc_run's for the same inputs.
 *   - Each call looks up the array's device address in the current context
 *     (a host-side query), so calls after a device reset use the new
 *     context's array.
 *   - All calls share the one array, and it keeps the last call's contents
 *     (each call initialises the state it uses, so nothing needs clearing).
 *     Calls whose kernels overlap on the GPU -- on different streams or from
 *     different threads -- race on it and must not be issued.
 *   - Synchronous like gac_mcmc_run: it returns after synchronising
 *     `stream`, once the last slice has finished.  lanes_per_chain is
 *     ignored.  Errors: INVALID_ARG, UNKNOWN_MODEL, CUDA. */
#define GAC_NOALLOC_STATE_BYTES (64u << 20)
gac_status gac_mcmc_run_noalloc(int model_id, const void *data, int64_t n_vox, const float *sigma,
                                float sigma_scalar, const float *x0, const gac_mcmc_opts *opts,
                                int slice_iterations, gac_result *out, void *stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of fit jobs on one GPU.
 *
 * A server owns a scheduler thread.  Submitted jobs wait in arrival order
 * until their device memory fits under the HBM budget (and a resident slot is
 * free); admitted jobs are uploaded on a copy stream while others compute.
 * The scheduler then runs rounds: each round is one launch per model kind of
 * a persistent kernel whose blocks claim work items -- (job, tile of voxels,
 * slice of iterations) -- from every resident job, so small and large jobs
 * share the GPU.  Chain state (theta, L, counters, Welford accumulators)
 * stays in HBM between slices.  Two rounds are in flight: the next one is
 * planned and queued behind the running one.  A job's results are copied
 * back behind its last round, and its memory returns to the budget once
 * that copy is done.
 * Results equal those of gac_mcmc_run with the same inputs: the random
 * numbers depend only on (seed, t, voxel, chain) and slices resume exactly.
 * Serving runs the MIXED precision path; trace_n_vox must be 0.
 * Threads: submit, poll, wait, cancel and get_stats may be called from any
 * host threads at once; destroy must not overlap any other call on the same
 * server.
 * ---------------------------------------------------------------------- */
typedef struct gac_server gac_server;

/* hbm_budget_bytes: device memory the server may hold for jobs (inputs,
 * chain state, outputs); max_resident_jobs: jobs on the device at once
 * (1..1024).  Does not touch the GPU until the first job is admitted. */
gac_status gac_server_create(size_t hbm_budget_bytes, int max_resident_jobs, gac_server **out);

/* Bytes of device memory a job would hold while resident. */
gac_status gac_server_job_bytes(int model_id, int64_t n_vox, const gac_mcmc_opts *opts,
                                int keep_samples, int has_sigma, size_t *bytes);

/* Queues a job: copies data [n_vox][n_meas] and sigma [n_vox] (or uses
 * sigma_scalar) from host or device memory and returns at once with *job_id.
 * keep_samples: also return the thinned samples.  Errors: INVALID_ARG
 * (including precision != MIXED or trace_n_vox != 0), UNKNOWN_MODEL, BUDGET
 * (the job alone exceeds the whole budget), OOM (host staging). */
gac_status gac_server_submit(gac_server *srv, int model_id, const void *data, int64_t n_vox,
                             const float *sigma, float sigma_scalar, const gac_mcmc_opts *opts,
                             int keep_samples, uint64_t *job_id);

/* Non-blocking.  *done = 0 while the job is queued or running.  When done,
 * copies the results into `out` (any pointer may be NULL; host or device),
 * sets *latency_s to the time from submit to completion, forgets the job and
 * returns GAC_OK -- or the job's error status (CANCELLED, CUDA, OOM).
 * Errors: UNKNOWN_JOB. */
gac_status gac_server_poll(gac_server *srv, uint64_t job_id, int *done, gac_result *out,
                           double *latency_s);

/* Blocks until the job is done or timeout_s passes (GAC_ERR_TIMEOUT); then
 * behaves as gac_server_poll.  timeout_s >= 0 (INFINITY waits without end);
 * otherwise INVALID_ARG.  If another thread collects the job first (poll or
 * wait), this call returns UNKNOWN_JOB. */
gac_status gac_server_wait(gac_server *srv, uint64_t job_id, double timeout_s, gac_result *out,
                           double *latency_s);

/* Cancels a queued or running job; its memory is released behind the rounds
 * already in flight.  Polling it afterwards returns GAC_ERR_CANCELLED (a job
 * whose last round was already queued completes normally). */
gac_status gac_server_cancel(gac_server *srv, uint64_t job_id);

/* Counters: jobs queued, resident, finished; bytes in use; rounds run; and
 * where the scheduler thread's time went: waiting for the rounds' kernels
 * after its own work for the round was done (gpu_s), preparing rounds
 * (round_host_s), admitting and retiring jobs (allocations, uploads queued;
 * admit_s, mostly overlapped with running rounds). */
typedef struct {
    int64_t queued, resident, finished, rounds;
    size_t bytes_in_use, budget;
    double gpu_s, round_host_s, admit_s;
} gac_server_stats;
gac_status gac_server_get_stats(gac_server *srv, gac_server_stats *st);

/* Stops the scheduler (after the current round), frees every job (results
 * not yet collected are lost).  No other call on `srv` may run meanwhile or
 * follow it. */
gac_status gac_server_destroy(gac_server *srv);

/* Message for the last non-OK status on the calling thread ("" if none). */
const char *gac_last_error(void);

/* Library version string. */
const char *gac_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GAC_H */
