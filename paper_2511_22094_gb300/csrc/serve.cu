// Serving runtime: continuous batching of MH fit jobs on one GPU
// (gac_server_* in include/gac.h).
//
// Jobs arrive from any host thread.  A scheduler thread admits them in
// arrival order while their device memory fits under the HBM budget, uploads
// them on a copy stream, and runs rounds.  A round is one launch of
// serve_kernel, a persistent kernel whose blocks claim work items (job, tile
// of voxels, iteration slice) from every resident job through an atomic
// counter; the block copies its job's descriptor into shared memory and runs
// the same tile routine as gac_mcmc_run, with chain state in HBM between
// slices.  Two rounds are in flight: while round r runs, round r+1 is planned
// from the iterations the earlier rounds will have reached, launched behind
// it on the same streams, and only then does the host wait for round r-1, so
// the GPU does not idle between rounds.  A job's last round enqueues its
// result download on the copy stream behind that round's kernels; its memory
// returns to the budget when the download is done.  No device code waits on
// the host: every wait is a host-side stream/event synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gac.h"
#include "gac_internal.h"
#include "mh_kernel.cuh"

namespace gac {

struct ServeJob {
    ModelConst mc;
    RunArgs ra;
    SliceState ss;
};

// A round's share of one job: iterations t_begin+1 .. t_end of every tile.
// The tiles of a kind's jobs are numbered consecutively from 0 (first_item
// of each entry), and blocks claim tile numbers through an atomic counter.
struct RoundJob {
    int32_t job;  // index into the round's job table
    int32_t t_begin;
    int32_t t_end;
    int32_t pad;
    int64_t first_item;
};

// The tile a block has claimed.
struct WorkItem {
    int32_t job;
    int32_t t_begin;
    int32_t t_end;
    int32_t pad;
    int64_t tile;
};

// Copies n bytes (a multiple of 4) cooperatively.
__device__ __forceinline__ void block_copy(void *dst, const void *src, int n) {
    int *d = static_cast<int *>(dst);
    const int *s = static_cast<const int *>(src);
    for (int i = threadIdx.x; i < n / 4; i += blockDim.x) d[i] = s[i];
}

// One kernel per model kind, so that each runs at its own register
// footprint; a round launches the kinds present concurrently on their own
// streams, and their blocks share the SMs.
template <int KIND>
__global__ void __launch_bounds__(kBlock, mh_min_blocks<KIND, GAC_PREC_MIXED>()) serve_kernel(const ServeJob *jobs, const RoundJob *rj, int n_rj,
                                                          int n_items, int *next_item) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) ServeJob s_job;
    __shared__ WorkItem s_item;
    __shared__ int s_idx;
    int cur_job = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_idx = atomicAdd(next_item, 1);
            if (s_idx < n_items) {  // the last entry whose first tile is <= s_idx
                int lo = 0, hi = n_rj - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (rj[mid].first_item <= s_idx) lo = mid;
                    else hi = mid - 1;
                }
                const RoundJob r = rj[lo];
                s_item.job = r.job;
                s_item.t_begin = r.t_begin;
                s_item.t_end = r.t_end;
                s_item.tile = s_idx - r.first_item;
            }
        }
        __syncthreads();
        if (s_idx >= n_items) break;
        const WorkItem wi = s_item;
        if (wi.job != cur_job) {
            __syncthreads();
            block_copy(&s_job, &jobs[wi.job], sizeof(ServeJob));
            cur_job = wi.job;
            __syncthreads();
        }
        run_tile<KIND, GAC_PREC_MIXED, false, true>(s_job.mc, s_job.ra, s_job.ss, wi.tile, wi.t_begin,
                                                    wi.t_end, smem_raw);
    }
}

constexpr int kKinds = 5;
static const int kKindOf[kKinds] = {GAC_MODEL_MONOEXP, GAC_MODEL_MWI3, GAC_MODEL_SMT, GAC_MODEL_AXCAL_SMT,
                                    GAC_MODEL_LINEAR_TEST};
static int kind_slot(int kind) {
    for (int i = 0; i < kKinds; ++i)
        if (kKindOf[i] == kind) return i;
    return -1;
}
static const void *serve_fn(int slot) {
    switch (slot) {
    case 0: return reinterpret_cast<const void *>(&serve_kernel<GAC_MODEL_MONOEXP>);
    case 1: return reinterpret_cast<const void *>(&serve_kernel<GAC_MODEL_MWI3>);
    case 2: return reinterpret_cast<const void *>(&serve_kernel<GAC_MODEL_SMT>);
    case 3: return reinterpret_cast<const void *>(&serve_kernel<GAC_MODEL_AXCAL_SMT>);
    default: return reinterpret_cast<const void *>(&serve_kernel<GAC_MODEL_LINEAR_TEST>);
    }
}
static void launch_serve(int slot, int grid, size_t smem, cudaStream_t s, const ServeJob *jobs,
                         const RoundJob *rj, int n_rj, int n, int *counter) {
    switch (slot) {
    case 0: serve_kernel<GAC_MODEL_MONOEXP><<<grid, kBlock, smem, s>>>(jobs, rj, n_rj, n, counter); break;
    case 1: serve_kernel<GAC_MODEL_MWI3><<<grid, kBlock, smem, s>>>(jobs, rj, n_rj, n, counter); break;
    case 2: serve_kernel<GAC_MODEL_SMT><<<grid, kBlock, smem, s>>>(jobs, rj, n_rj, n, counter); break;
    case 3: serve_kernel<GAC_MODEL_AXCAL_SMT><<<grid, kBlock, smem, s>>>(jobs, rj, n_rj, n, counter); break;
    default: serve_kernel<GAC_MODEL_LINEAR_TEST><<<grid, kBlock, smem, s>>>(jobs, rj, n_rj, n, counter); break;
    }
}

// ------------------------------------------------------------------ host --
static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Page-locked host buffers are slow to allocate and free (every page is
// pinned), so the server keeps the ones its jobs release and hands them out
// again: sizes are rounded up to powers of two from 64 KiB, and the cache is
// emptied when the server is destroyed.
class PinnedCache {
  public:
    static size_t size_class(size_t bytes) {
        size_t c = 64 << 10;
        while (c < bytes) c <<= 1;
        return c;
    }
    cudaError_t get(void **p, size_t bytes) {
        const size_t c = size_class(bytes);
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto &v = free_[c];
            if (!v.empty()) {
                *p = v.back();
                v.pop_back();
                return cudaSuccess;
            }
        }
        return cudaMallocHost(p, c);
    }
    void put(void *p, size_t bytes) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        free_[size_class(bytes)].push_back(p);
    }
    ~PinnedCache() {
        for (auto &kv : free_)
            for (void *p : kv.second) cudaFreeHost(p);
    }

  private:
    std::mutex mu_;
    std::map<size_t, std::vector<void *>> free_;
};

enum class JobState { Queued, Uploading, Running, Finishing, Done, Failed, Cancelled };

struct Job {
    uint64_t id = 0;
    ModelConst mc;
    gac_mcmc_opts opts;
    int64_t n_vox = 0;
    int keep_samples = 0;
    int S = 0;
    size_t bytes = 0;
    JobState state = JobState::Queued;
    gac_status err = GAC_OK;
    bool cancel = false;
    int t_done = 0;
    double t_submit = 0, t_finish = 0;
    // host copies of inputs (pinned) and results (pinned)
    float *h_data = nullptr, *h_sigma = nullptr;
    float sigma_scalar = 0.0f;
    double *h_mean = nullptr, *h_std = nullptr, *h_rhat = nullptr;
    float *h_samples = nullptr, *h_acc = nullptr, *h_scale = nullptr;
    int32_t *h_bad = nullptr;
    // device block holding inputs, state and outputs
    void *d_block = nullptr;
    ServeJob desc;
    cudaEvent_t ev = nullptr;  // upload or download completion
};

// Layout of one job's device block.
struct JobLayout {
    size_t data, sigma, theta, L, n_acc, n_bad, adapt, wf_mean, wf_m2, blk, mean, std, acc, bad, rhat, scale,
        samples, total;
};

static size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static JobLayout job_layout(const ModelConst &mc, int64_t n_vox, const gac_mcmc_opts &o, int keep_samples,
                            bool has_sigma) {
    const size_t N = static_cast<size_t>(n_vox), P = mc.n_par, C = o.n_chains, M = mc.n_meas;
    const size_t S = keep_samples ? n_samples(o.iterations, o.burnin, o.thin) : 0;
    JobLayout l;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
    l.data = take(N * M * 4);
    l.sigma = take(has_sigma ? N * 4 : 0);
    l.theta = take(P * N * C * 4);
    l.L = take(N * C * 4);
    l.n_acc = take(N * C * 4);
    l.n_bad = take(N * C * 4);
    l.adapt = take(2 * N * C * 4);
    l.wf_mean = take(P * N * C * 8);
    l.wf_m2 = take(P * N * C * 8);
    l.blk = take(o.moments_mode == GAC_MOMENTS_ALL_POSTBURNIN ? 3 * P * N * C * 4 : 0);
    l.mean = take(P * N * 8);
    l.std = take(P * N * 8);
    l.acc = take(C * N * 4);
    l.bad = take(C * N * 4);
    l.rhat = take(P * N * 8);
    l.scale = take(C * N * 4);
    l.samples = take(S * C * P * N * 4);
    l.total = off;
    return l;
}

}  // namespace gac

using namespace gac;

struct gac_server {
    size_t budget = 0;
    int max_resident = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::vector<std::shared_ptr<Job>> resident;  // Uploading / Running / Finishing
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_id = 1;
    size_t in_use = 0;
    int64_t finished = 0, rounds = 0;
    bool stop = false;
    std::thread thr;
    bool started = false;
    int device = 0;
    // GPU resources, created by the scheduler thread
    // s_copy: allocations and uploads; s_down: result downloads and frees,
    // which wait for rounds in flight (kept off s_copy so uploads never queue
    // behind those waits)
    cudaStream_t s_compute = nullptr, s_copy = nullptr, s_down = nullptr;
    cudaStream_t s_kind[kKinds] = {};
    // per round buffer set b = round & 1 (two rounds in flight)
    cudaEvent_t ev_setup[2] = {}, ev_kind[2][kKinds] = {};
    PinnedCache pinned;  // destroyed after every job's buffers are back
    ServeJob *d_jobs[2] = {}, *h_jobs[2] = {};
    RoundJob *d_items[2] = {}, *h_items[2] = {};
    int *d_counter = nullptr;  // [2][kKinds]
    size_t cap_jobs[2] = {}, cap_items[2] = {};
    struct Inflight {
        int b;
        bool kind_ran[kKinds];
        int64_t work;
    };
    std::deque<Inflight> inflight;
    int64_t round_seq = 0;
    double t_last_done = 0;
    size_t smem = 0;
    int sms = 1;
    double ci_per_s = 2e10;   // throughput estimate, refined each round
    double round_target_s = 0.025;
    double t_gpu = 0, t_round_host = 0, t_admit = 0;  // scheduler time split

    void loop();
    gac_status init_gpu();
    gac_status admit_locked(int max_jobs = 1 << 30);
    gac_status run_round(bool *launched);
    gac_status wait_oldest_round();
    void retire_locked();
    void free_job(Job &j);
    void free_results(Job &j);
};

static gac_status round_alloc(void **d, void **h, size_t bytes) {
    cudaError_t e = cudaMalloc(d, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "server table");
    e = cudaMallocHost(h, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "server table (host)");
    return GAC_OK;
}

gac_status gac_server::init_gpu() {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if ((e = cudaStreamCreateWithFlags(&s_compute, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    if ((e = cudaStreamCreateWithFlags(&s_copy, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    if ((e = cudaStreamCreateWithFlags(&s_down, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    if ((e = cudaMalloc(&d_counter, 2 * kKinds * sizeof(int))) != cudaSuccess) return cuda_fail(e, "counter");
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaEventCreateWithFlags(&ev_setup[b], cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
        for (int i = 0; i < kKinds; ++i)
            if ((e = cudaEventCreateWithFlags(&ev_kind[b][i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "event");
    }
    for (int i = 0; i < kKinds; ++i)
        if ((e = cudaStreamCreateWithFlags(&s_kind[i], cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
    // the largest measurement tile any job can need (C = 1, 256 voxels, 64
    // complex echoes); each round launches with its own jobs' largest tile
    smem = static_cast<size_t>(kBlock) * row_stride_for(GAC_MODEL_MWI3, 2 * GAC_MAX_ACQ) * sizeof(float) +
           3 * static_cast<size_t>(GAC_MAX_PAR) * kBlock * sizeof(float);  // + all-post-burn-in block partials
    for (int i = 0; i < kKinds; ++i) {
        e = cudaFuncSetAttribute(serve_fn(i), cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return cuda_fail(e, "serve kernel smem");
        e = cudaFuncSetAttribute(serve_fn(i), cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return cuda_fail(e, "serve kernel carveout");
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms < 1) sms = 1;
    keep_staging_pool();  // job blocks come from the stream-ordered pool
    return GAC_OK;
}

void gac_server::free_job(Job &j) {
    // stream-ordered: after the job's upload (a job is freed only once its
    // event has completed), its download and every round launched so far (a
    // cancelled job may be in one)
    if (j.d_block && s_down)
        for (int b = 0; b < 2; ++b)
            for (int i = 0; i < kKinds; ++i) cudaStreamWaitEvent(s_down, ev_kind[b][i], 0);
    if (j.d_block) cudaFreeAsync(j.d_block, s_down ? s_down : cudaStream_t{});
    j.d_block = nullptr;
    if (j.ev) cudaEventDestroy(j.ev);
    j.ev = nullptr;
    const size_t N = j.n_vox;
    pinned.put(j.h_data, N * j.mc.n_meas * 4);
    pinned.put(j.h_sigma, N * 4);
    j.h_data = j.h_sigma = nullptr;
}

void gac_server::free_results(Job &j) {
    const size_t N = j.n_vox, P = j.mc.n_par, C = j.opts.n_chains;
    pinned.put(j.h_mean, P * N * 8);
    pinned.put(j.h_std, P * N * 8);
    pinned.put(j.h_rhat, P * N * 8);
    pinned.put(j.h_acc, C * N * 4);
    pinned.put(j.h_bad, C * N * 4);
    pinned.put(j.h_scale, C * N * 4);
    pinned.put(j.h_samples, static_cast<size_t>(j.S) * C * P * N * 4);
    j.h_mean = j.h_std = j.h_rhat = nullptr;
    j.h_samples = j.h_acc = j.h_scale = nullptr;
    j.h_bad = nullptr;
}

// Admits queued jobs in arrival order while they fit, at most max_jobs of
// them (caller holds mu).
gac_status gac_server::admit_locked(int max_jobs) {
    int admitted = 0;
    while (!queue.empty() && admitted < max_jobs) {
        auto jp = queue.front();
        Job &j = *jp;
        if (j.cancel) {
            queue.pop_front();
            j.state = JobState::Cancelled;
            free_job(j);
            cv_done.notify_all();
            continue;
        }
        if (static_cast<int>(resident.size()) >= max_resident || in_use + j.bytes > budget) break;
        queue.pop_front();
        const bool has_sigma = j.h_sigma != nullptr;
        JobLayout l = job_layout(j.mc, j.n_vox, j.opts, j.keep_samples, has_sigma);
        cudaError_t e = cudaMallocAsync(&j.d_block, l.total, s_copy);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming);
        const size_t N = j.n_vox, P = j.mc.n_par, C = j.opts.n_chains;
        if (e == cudaSuccess) e = cudaMemcpyAsync(static_cast<char *>(j.d_block) + l.data, j.h_data,
                                                  N * j.mc.n_meas * 4, cudaMemcpyHostToDevice, s_copy);
        if (e == cudaSuccess && has_sigma)
            e = cudaMemcpyAsync(static_cast<char *>(j.d_block) + l.sigma, j.h_sigma, N * 4, cudaMemcpyHostToDevice,
                                s_copy);
        // results on the host (pinned)
        auto pin = [&](auto **p, size_t bytes) { return pinned.get(reinterpret_cast<void **>(p), bytes); };
        if (e == cudaSuccess) e = pin(&j.h_mean, P * N * 8);
        if (e == cudaSuccess) e = pin(&j.h_std, P * N * 8);
        if (e == cudaSuccess) e = pin(&j.h_acc, C * N * 4);
        if (e == cudaSuccess) e = pin(&j.h_bad, C * N * 4);
        if (e == cudaSuccess) e = pin(&j.h_rhat, P * N * 8);
        if (e == cudaSuccess) e = pin(&j.h_scale, C * N * 4);
        if (e == cudaSuccess && j.keep_samples && j.S > 0) e = pin(&j.h_samples, static_cast<size_t>(j.S) * C * P * N * 4);
        if (e == cudaSuccess) e = cudaEventRecord(j.ev, s_copy);
        if (e != cudaSuccess) {
            cudaGetLastError();
            j.err = e == cudaErrorMemoryAllocation ? GAC_ERR_OOM : GAC_ERR_CUDA;
            j.state = JobState::Failed;
            cudaStreamSynchronize(s_copy);  // an upload may be in flight into the block
            free_job(j);
            free_results(j);
            cv_done.notify_all();
            continue;
        }
        char *b = static_cast<char *>(j.d_block);
        RunArgs &ra = j.desc.ra;
        std::memset(&ra, 0, sizeof ra);
        ra.data = reinterpret_cast<const float *>(b + l.data);
        ra.sigma = has_sigma ? reinterpret_cast<const float *>(b + l.sigma) : nullptr;
        ra.sigma_scalar = j.sigma_scalar;
        ra.mean = reinterpret_cast<double *>(b + l.mean);
        ra.std = reinterpret_cast<double *>(b + l.std);
        ra.samples = (j.keep_samples && j.S > 0) ? reinterpret_cast<float *>(b + l.samples) : nullptr;
        ra.accept = reinterpret_cast<float *>(b + l.acc);
        ra.nonfinite = reinterpret_cast<int32_t *>(b + l.bad);
        ra.n_vox = j.n_vox;
        ra.C = j.opts.n_chains;
        ra.I = j.opts.iterations;
        ra.B = j.opts.burnin;
        ra.T = j.opts.thin;
        ra.S = n_samples(j.opts.iterations, j.opts.burnin, j.opts.thin);
        ra.k0 = static_cast<uint32_t>(j.opts.seed);
        ra.k1 = static_cast<uint32_t>(j.opts.seed >> 32);
        ra.voxel_base = j.opts.voxel_base;
        ra.moments_mode = j.opts.moments_mode;
        ra.vox_per_block = kBlock / ra.C;
        ra.row_stride = row_stride_for(j.mc.kind, j.mc.n_meas);
        ra.data_vec4 = (j.mc.n_meas % 4) == 0;
        ra.n_tiles = (j.n_vox + ra.vox_per_block - 1) / ra.vox_per_block;
        set_adaptation(ra, &j.opts);
        ra.rhat = reinterpret_cast<double *>(b + l.rhat);
        ra.step_scale = reinterpret_cast<float *>(b + l.scale);
        SliceState &ss = j.desc.ss;
        ss.theta = b + l.theta;
        ss.L = b + l.L;
        ss.n_acc = reinterpret_cast<int32_t *>(b + l.n_acc);
        ss.n_bad = reinterpret_cast<int32_t *>(b + l.n_bad);
        ss.adapt = reinterpret_cast<int32_t *>(b + l.adapt);
        ss.wf_mean = b + l.wf_mean;
        ss.wf_m2 = b + l.wf_m2;
        ss.blk = j.opts.moments_mode == GAC_MOMENTS_ALL_POSTBURNIN ? reinterpret_cast<float *>(b + l.blk) : nullptr;
        j.desc.mc = j.mc;
        in_use += j.bytes;
        j.state = JobState::Uploading;
        resident.push_back(jp);
        ++admitted;
    }
    return GAC_OK;
}

// Moves finished downloads to Done and releases cancelled jobs (mu held).
void gac_server::retire_locked() {
    for (auto it = resident.begin(); it != resident.end();) {
        Job &j = **it;
        bool drop = false;
        if (j.state == JobState::Finishing && cudaEventQuery(j.ev) == cudaSuccess) {
            j.state = JobState::Done;
            j.t_finish = now_s();
            ++finished;
            drop = true;
        } else if (j.cancel && (j.state == JobState::Running || j.state == JobState::Uploading)) {
            cudaEventSynchronize(j.ev);
            j.state = JobState::Cancelled;
            free_results(j);
            drop = true;
        }
        if (drop) {
            in_use -= j.bytes;
            free_job(j);
            it = resident.erase(it);
            cv_done.notify_all();
        } else {
            ++it;
        }
    }
}

// Plans round r from the iterations the launched rounds will have reached,
// launches it behind them, queues the downloads of the jobs it completes,
// then admits and retires jobs while the GPU works.  *launched = false when
// no job can run.
gac_status gac_server::run_round(bool *launched) {
    *launched = false;
    // choose the jobs and the slice length under the lock
    std::vector<std::shared_ptr<Job>> run;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &jp : resident) {
            Job &j = *jp;
            if (j.cancel) continue;
            if (j.state == JobState::Uploading && cudaEventQuery(j.ev) == cudaSuccess) j.state = JobState::Running;
            // a Running job has rounds left to plan (the round that reaches its last
            // iteration turns it into Finishing); a zero-iteration job takes one
            // empty round, which initialises its chains and writes its outputs
            if (j.state == JobState::Running) run.push_back(jp);
        }
    }
    if (run.empty()) return GAC_OK;
    const double t_prep = now_s();
    // Slice lengths.  A round is about round_target_s of work at the current
    // throughput estimate.  Jobs are taken in order of remaining work: one
    // whose remainder fits in half of what is left of the first half of the
    // round's budget runs to completion in this round (small jobs leave
    // quickly instead of advancing in lock-step with large ones).  The others
    // get the rest of the budget -- at least half of it, so that a stream of
    // small arrivals cannot starve a large job -- in order of their slowdown
    // so far (time since submission over the job's time alone at the current
    // throughput), each as many iterations as the remaining budget allows and
    // at least 16: the job that has waited longest relative to its size goes
    // first instead of every large job advancing at a shared rate.
    std::vector<size_t> order(run.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    auto remaining = [&](size_t i) {
        const Job &j = *run[i];
        return static_cast<double>(j.opts.iterations - j.t_done) * j.n_vox * j.opts.n_chains;
    };
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return remaining(a) < remaining(b); });
    double budget_ci = round_target_s * ci_per_s;
    double small_ci = 0.5 * budget_ci;
    std::vector<int> t_end(run.size(), -1);
    std::vector<size_t> big;
    for (size_t i : order) {
        const double rem = remaining(i);
        if (rem <= 0.5 * small_ci) {
            t_end[i] = run[i]->opts.iterations;
            small_ci -= rem;
            budget_ci -= rem;
        } else {
            big.push_back(i);
        }
    }
    const double now = now_s();
    auto slowdown = [&](size_t i) {
        const Job &j = *run[i];
        const double alone = static_cast<double>(j.opts.iterations) * j.n_vox * j.opts.n_chains / ci_per_s;
        return (now - j.t_submit) / std::max(alone, 1e-9);
    };
    std::stable_sort(big.begin(), big.end(), [&](size_t a, size_t c) { return slowdown(a) > slowdown(c); });
    double left = std::max(budget_ci, 0.0);
    for (size_t i : big) {
        const Job &j = *run[i];
        const int64_t chains = j.n_vox * j.opts.n_chains;
        const int64_t k = std::max<int64_t>(16, static_cast<int64_t>(left / static_cast<double>(chains)));
        t_end[i] = static_cast<int>(std::min<int64_t>(j.opts.iterations, j.t_done + k));
        left = std::max(0.0, left - static_cast<double>(t_end[i] - j.t_done) * chains);
    }
    // this round's buffer set: its previous user, round r-2, has completed
    const int b = static_cast<int>(round_seq & 1);
    const size_t n_items = run.size();  // one round entry per job
    if (run.size() > cap_jobs[b]) {
        if (d_jobs[b]) cudaFree(d_jobs[b]);
        if (h_jobs[b]) cudaFreeHost(h_jobs[b]);
        d_jobs[b] = h_jobs[b] = nullptr;
        cap_jobs[b] = std::max<size_t>(run.size(), 2 * cap_jobs[b]);
        gac_status st = round_alloc(reinterpret_cast<void **>(&d_jobs[b]), reinterpret_cast<void **>(&h_jobs[b]),
                                    cap_jobs[b] * sizeof(ServeJob));
        if (st != GAC_OK) return st;
    }
    if (n_items > cap_items[b]) {
        if (d_items[b]) cudaFree(d_items[b]);
        if (h_items[b]) cudaFreeHost(h_items[b]);
        d_items[b] = h_items[b] = nullptr;
        cap_items[b] = std::max(n_items, 2 * cap_items[b]);
        gac_status st = round_alloc(reinterpret_cast<void **>(&d_items[b]), reinterpret_cast<void **>(&h_items[b]),
                                    cap_items[b] * sizeof(RoundJob));
        if (st != GAC_OK) return st;
    }
    // items grouped by model kind (one contiguous range per kind's kernel),
    // within a kind the longest slices first: blocks claim items in list
    // order, so the jobs that run to completion start at the beginning
    std::vector<size_t> by_len(run.size());
    for (size_t i = 0; i < by_len.size(); ++i) by_len[i] = i;
    std::stable_sort(by_len.begin(), by_len.end(), [&](size_t a, size_t c) {
        return t_end[a] - run[a]->t_done > t_end[c] - run[c]->t_done;
    });
    size_t k = 0;
    int64_t work = 0;
    size_t first_rj[kKinds] = {}, n_rj[kKinds] = {}, count_item[kKinds] = {}, smem_kind[kKinds] = {};
    for (size_t ji = 0; ji < run.size(); ++ji) h_jobs[b][ji] = run[ji]->desc;
    for (int slot = 0; slot < kKinds; ++slot) {
        first_rj[slot] = k;
        int64_t tiles = 0;
        for (size_t ji : by_len) {
            Job &j = *run[ji];
            if (kind_slot(j.mc.kind) != slot) continue;
            const RunArgs &ra = j.desc.ra;
            smem_kind[slot] = std::max(smem_kind[slot],
                                       tile_smem_bytes(j.mc.n_par, 8, ra.vox_per_block, ra.row_stride, false,
                                                       ra.moments_mode == GAC_MOMENTS_ALL_POSTBURNIN));
            work += static_cast<int64_t>(t_end[ji] - j.t_done) * j.n_vox * j.opts.n_chains;
            RoundJob &r = h_items[b][k++];
            r.job = static_cast<int32_t>(ji);
            r.t_begin = j.t_done;
            r.t_end = t_end[ji];
            r.pad = 0;
            r.first_item = tiles;
            tiles += ra.n_tiles;
        }
        n_rj[slot] = k - first_rj[slot];
        count_item[slot] = static_cast<size_t>(tiles);
    }
    int *counter = d_counter + b * kKinds;
    cudaError_t e = cudaMemcpyAsync(d_jobs[b], h_jobs[b], run.size() * sizeof(ServeJob), cudaMemcpyHostToDevice, s_compute);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_items[b], h_items[b], n_items * sizeof(RoundJob), cudaMemcpyHostToDevice, s_compute);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, kKinds * sizeof(int), s_compute);
    if (e == cudaSuccess) e = cudaEventRecord(ev_setup[b], s_compute);
    if (e != cudaSuccess) return cuda_fail(e, "round setup");
    Inflight rec{};
    rec.b = b;
    rec.work = work;
    for (int slot = 0; slot < kKinds; ++slot) {
        if (count_item[slot] == 0) continue;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_fn(slot), kBlock, smem_kind[slot]);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy");
        const size_t grid = std::min<size_t>(static_cast<size_t>(std::max(1, per_sm)) * sms, count_item[slot]);
        if ((e = cudaStreamWaitEvent(s_kind[slot], ev_setup[b], 0)) != cudaSuccess) return cuda_fail(e, "wait");
        launch_serve(slot, static_cast<int>(grid), smem_kind[slot], s_kind[slot], d_jobs[b], d_items[b] + first_rj[slot],
                     static_cast<int>(n_rj[slot]), static_cast<int>(count_item[slot]), counter + slot);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "serve kernel launch");
        if ((e = cudaEventRecord(ev_kind[b][slot], s_kind[slot])) != cudaSuccess) return cuda_fail(e, "event");
        rec.kind_ran[slot] = true;
    }
    inflight.push_back(rec);
    ++round_seq;
    *launched = true;
    const double t_launched = now_s();
    {
        // advance to the iterations this round reaches; a job it completes
        // downloads its results on the copy stream behind the round's kernel
        std::lock_guard<std::mutex> lk(mu);
        t_round_host += t_launched - t_prep;  // the counters are read under the lock
        const double t0 = now_s();
        for (size_t ji = 0; ji < run.size(); ++ji) {
            Job &j = *run[ji];
            j.t_done = t_end[ji];
            if (j.t_done < j.opts.iterations) continue;
            const size_t N = j.n_vox, P = j.mc.n_par, C = j.opts.n_chains;
            const RunArgs &ra = j.desc.ra;
            e = cudaStreamWaitEvent(s_down, ev_kind[b][kind_slot(j.mc.kind)], 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(j.h_mean, ra.mean, P * N * 8, cudaMemcpyDeviceToHost, s_down);
            if (e == cudaSuccess) e = cudaMemcpyAsync(j.h_std, ra.std, P * N * 8, cudaMemcpyDeviceToHost, s_down);
            if (e == cudaSuccess) e = cudaMemcpyAsync(j.h_acc, ra.accept, C * N * 4, cudaMemcpyDeviceToHost, s_down);
            if (e == cudaSuccess) e = cudaMemcpyAsync(j.h_bad, ra.nonfinite, C * N * 4, cudaMemcpyDeviceToHost, s_down);
            if (e == cudaSuccess) e = cudaMemcpyAsync(j.h_rhat, ra.rhat, P * N * 8, cudaMemcpyDeviceToHost, s_down);
            if (e == cudaSuccess) e = cudaMemcpyAsync(j.h_scale, ra.step_scale, C * N * 4, cudaMemcpyDeviceToHost, s_down);
            if (e == cudaSuccess && ra.samples)
                e = cudaMemcpyAsync(j.h_samples, ra.samples, static_cast<size_t>(j.S) * C * P * N * 4,
                                    cudaMemcpyDeviceToHost, s_down);
            if (e == cudaSuccess) e = cudaEventRecord(j.ev, s_down);
            if (e != cudaSuccess) return cuda_fail(e, "result download");
            j.state = JobState::Finishing;
        }
        // while the rounds run: retire finished downloads and admit queued
        // jobs (allocations and uploads), so that the host work overlaps the
        // kernels
        retire_locked();
        gac_status st = admit_locked();
        t_admit += now_s() - t0;
        if (st != GAC_OK) return st;
    }
    // keep one round queued behind the running one
    while (inflight.size() > 1) {
        gac_status st = wait_oldest_round();
        if (st != GAC_OK) return st;
    }
    return GAC_OK;
}

// Waits for the oldest round in flight; refines the throughput estimate from
// the interval between round completions (back-to-back rounds).
gac_status gac_server::wait_oldest_round() {
    if (inflight.empty()) return GAC_OK;
    const Inflight r = inflight.front();
    inflight.pop_front();
    const double t_wait = now_s();
    for (int slot = 0; slot < kKinds; ++slot) {
        if (!r.kind_ran[slot]) continue;
        cudaError_t e = cudaEventSynchronize(ev_kind[r.b][slot]);
        if (e != cudaSuccess) return cuda_fail(e, "serve kernel");
    }
    const double t = now_s();
    // a round that had ended before the host looked gives no timing, nor
    // does one that did not start right at its predecessor's end
    const bool waited = t - t_wait > 1e-4;
    if (waited && t_last_done > 0 && r.work > 0) {
        const double dt = t - t_last_done;
        if (dt > 1e-4) ci_per_s = 0.5 * ci_per_s + 0.5 * (r.work / dt);
    }
    t_last_done = (waited && !inflight.empty()) ? t : 0.0;
    std::lock_guard<std::mutex> lk(mu);
    t_gpu += t - t_wait;
    ++rounds;
    return GAC_OK;
}

void gac_server::loop() {
    gac_status st = init_gpu();
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (st == GAC_OK) {
                // with nothing on the GPU, admit one job to start a round at
                // once; otherwise admission waits for the next round's launch
                // (run_round admits while its kernels run), so that the GPU
                // does not idle between rounds while jobs are admitted
                bool busy = !inflight.empty();
                for (auto &jp : resident)
                    busy = busy || jp->state == JobState::Running || jp->state == JobState::Uploading;
                const double t0 = now_s();
                retire_locked();
                if (!busy) admit_locked(1);
                t_admit += now_s() - t0;
            }
            if (st != GAC_OK) {
                // the GPU side failed: fail every job so no caller waits forever
                for (auto &jp : queue) { jp->state = JobState::Failed; jp->err = st; }
                for (auto &jp : resident) { jp->state = JobState::Failed; jp->err = st; }
                queue.clear();
                resident.clear();
                inflight.clear();
                cv_done.notify_all();
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
                if (stop) break;
                continue;
            }
            if (stop) break;
            bool runnable = false, waiting = false;
            for (auto &jp : resident) {
                if (jp->state == JobState::Running ||
                    jp->state == JobState::Uploading)
                    runnable = true;
                if (jp->state == JobState::Finishing) waiting = true;
            }
            if (!runnable) {
                if (!inflight.empty() || waiting) {
                    // the last rounds and downloads: wait for them, then retire
                    lk.unlock();
                    while (st == GAC_OK && !inflight.empty()) st = wait_oldest_round();
                    if (st == GAC_OK) cudaStreamSynchronize(s_down);
                    continue;
                }
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
                if (stop) break;
                continue;
            }
        }
        bool launched = false;
        st = run_round(&launched);  // admits the queued jobs while the rounds run
        if (st == GAC_OK && !launched) {
            // only uploads in flight (or every runnable job already has its
            // rounds queued): finish the rounds, wait for the uploads
            while (st == GAC_OK && !inflight.empty()) st = wait_oldest_round();
            if (st == GAC_OK) cudaStreamSynchronize(s_copy);
        }
    }
    // shutdown: wait for the GPU, release everything
    for (int i = 0; i < kKinds; ++i)
        if (s_kind[i]) cudaStreamSynchronize(s_kind[i]);
    if (s_compute) cudaStreamSynchronize(s_compute);
    if (s_copy) cudaStreamSynchronize(s_copy);
    if (s_down) cudaStreamSynchronize(s_down);
    std::lock_guard<std::mutex> lk(mu);
    for (auto &kv : jobs) {
        free_job(*kv.second);
        free_results(*kv.second);
    }
    if (s_down) cudaStreamSynchronize(s_down);  // the stream-ordered frees
    for (int b = 0; b < 2; ++b) {
        if (d_jobs[b]) cudaFree(d_jobs[b]);
        if (h_jobs[b]) cudaFreeHost(h_jobs[b]);
        if (d_items[b]) cudaFree(d_items[b]);
        if (h_items[b]) cudaFreeHost(h_items[b]);
    }
    if (d_counter) cudaFree(d_counter);
    for (int i = 0; i < kKinds; ++i) {
        if (s_kind[i]) cudaStreamSynchronize(s_kind[i]);
        if (s_kind[i]) cudaStreamDestroy(s_kind[i]);
    }
    for (int b = 0; b < 2; ++b) {
        for (int i = 0; i < kKinds; ++i)
            if (ev_kind[b][i]) cudaEventDestroy(ev_kind[b][i]);
        if (ev_setup[b]) cudaEventDestroy(ev_setup[b]);
    }
    if (s_compute) cudaStreamDestroy(s_compute);
    if (s_copy) cudaStreamDestroy(s_copy);
    if (s_down) cudaStreamDestroy(s_down);
}

static gac_status job_bytes(const ModelConst &mc, int64_t n_vox, const gac_mcmc_opts &o, int keep, bool has_sigma,
                            size_t *bytes) {
    *bytes = job_layout(mc, n_vox, o, keep, has_sigma).total;
    return GAC_OK;
}

extern "C" {

gac_status gac_server_create(size_t hbm_budget_bytes, int max_resident_jobs, gac_server **out) {
    clear_error();
    if (!out) return fail(GAC_ERR_INVALID_ARG, "out must not be NULL");
    if (hbm_budget_bytes == 0) return fail(GAC_ERR_INVALID_ARG, "budget must be > 0");
    if (max_resident_jobs < 1 || max_resident_jobs > 1024)
        return fail(GAC_ERR_INVALID_ARG, "max_resident_jobs must be in [1, 1024]");
    gac_server *s = new (std::nothrow) gac_server();
    if (!s) return fail(GAC_ERR_OOM, "server");
    s->budget = hbm_budget_bytes;
    s->max_resident = max_resident_jobs;
    *out = s;
    return GAC_OK;
}

gac_status gac_server_job_bytes(int model_id, int64_t n_vox, const gac_mcmc_opts *opts, int keep_samples,
                                int has_sigma, size_t *bytes) {
    clear_error();
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (!bytes || n_vox < 0) return fail(GAC_ERR_INVALID_ARG, "bad arguments");
    if ((st = validate_opts(opts, n_vox)) != GAC_OK) return st;
    return job_bytes(mc, n_vox, *opts, keep_samples, has_sigma != 0, bytes);
}

gac_status gac_server_submit(gac_server *srv, int model_id, const void *data, int64_t n_vox, const float *sigma,
                             float sigma_scalar, const gac_mcmc_opts *opts, int keep_samples, uint64_t *job_id) {
    clear_error();
    if (!srv || !job_id) return fail(GAC_ERR_INVALID_ARG, "srv and job_id must not be NULL");
    ModelConst mc;
    gac_status st = model_get(model_id, &mc);
    if (st != GAC_OK) return st;
    if (n_vox < 1) return fail(GAC_ERR_INVALID_ARG, "n_vox must be >= 1");
    if ((st = validate_opts(opts, n_vox)) != GAC_OK) return st;
    if (opts->precision != GAC_PREC_MIXED) return fail(GAC_ERR_INVALID_ARG, "serving runs the MIXED precision path");
    if (opts->trace_n_vox != 0) return fail(GAC_ERR_INVALID_ARG, "serving does not trace");
    if (!data) return fail(GAC_ERR_INVALID_ARG, "data must not be NULL");
    if (!sigma && !(sigma_scalar > 0.0f)) return fail(GAC_ERR_INVALID_ARG, "sigma is NULL and sigma_scalar <= 0");
    size_t bytes = 0;
    job_bytes(mc, n_vox, *opts, keep_samples, sigma != nullptr, &bytes);
    if (bytes > srv->budget)
        return fail(GAC_ERR_BUDGET, "job needs %zu bytes, more than the whole budget of %zu", bytes, srv->budget);

    auto jp = std::make_shared<Job>();
    Job &j = *jp;
    j.mc = mc;
    j.opts = *opts;
    j.n_vox = n_vox;
    j.keep_samples = keep_samples ? 1 : 0;
    j.S = n_samples(opts->iterations, opts->burnin, opts->thin);
    j.bytes = bytes;
    j.sigma_scalar = sigma_scalar;
    const size_t dbytes = static_cast<size_t>(n_vox) * mc.n_meas * 4;
    cudaError_t e = srv->pinned.get(reinterpret_cast<void **>(&j.h_data), dbytes);
    if (e == cudaSuccess) e = cudaMemcpy(j.h_data, data, dbytes, cudaMemcpyDefault);
    if (e == cudaSuccess && sigma) {
        e = srv->pinned.get(reinterpret_cast<void **>(&j.h_sigma), static_cast<size_t>(n_vox) * 4);
        if (e == cudaSuccess) e = cudaMemcpy(j.h_sigma, sigma, static_cast<size_t>(n_vox) * 4, cudaMemcpyDefault);
    }
    if (e != cudaSuccess) {
        srv->pinned.put(j.h_data, dbytes);
        srv->pinned.put(j.h_sigma, static_cast<size_t>(n_vox) * 4);
        return cuda_fail(e, "staging job inputs");
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (!srv->started) {
        cudaGetDevice(&srv->device);
        srv->thr = std::thread([srv] { srv->loop(); });
        srv->started = true;
    }
    j.id = srv->next_id++;
    j.t_submit = now_s();
    srv->jobs[j.id] = jp;
    srv->queue.push_back(jp);
    *job_id = j.id;
    srv->cv_work.notify_all();
    return GAC_OK;
}

static gac_status deliver(gac_server *srv, std::map<uint64_t, std::shared_ptr<Job>>::iterator it, gac_result *out,
                          double *latency_s) {
    Job &j = *it->second;
    gac_status st = GAC_OK;
    if (j.state == JobState::Cancelled) {
        st = fail(GAC_ERR_CANCELLED, "job %llu was cancelled", static_cast<unsigned long long>(j.id));
    } else if (j.state == JobState::Failed) {
        st = fail(j.err, "job %llu failed", static_cast<unsigned long long>(j.id));
    } else {
        const size_t N = j.n_vox, P = j.mc.n_par, C = j.opts.n_chains;
        cudaError_t e = cudaSuccess;
        if (out) {
            if (out->mean && e == cudaSuccess) e = cudaMemcpy(out->mean, j.h_mean, P * N * 8, cudaMemcpyDefault);
            if (out->std && e == cudaSuccess) e = cudaMemcpy(out->std, j.h_std, P * N * 8, cudaMemcpyDefault);
            if (out->accept_rate && e == cudaSuccess) e = cudaMemcpy(out->accept_rate, j.h_acc, C * N * 4, cudaMemcpyDefault);
            if (out->nonfinite && e == cudaSuccess) e = cudaMemcpy(out->nonfinite, j.h_bad, C * N * 4, cudaMemcpyDefault);
            if (out->rhat && e == cudaSuccess) e = cudaMemcpy(out->rhat, j.h_rhat, P * N * 8, cudaMemcpyDefault);
            if (out->step_scale && e == cudaSuccess)
                e = cudaMemcpy(out->step_scale, j.h_scale, C * N * 4, cudaMemcpyDefault);
            if (out->samples && j.h_samples && e == cudaSuccess)
                e = cudaMemcpy(out->samples, j.h_samples, static_cast<size_t>(j.S) * C * P * N * 4, cudaMemcpyDefault);
        }
        if (e != cudaSuccess) st = cuda_fail(e, "copy results");
        if (latency_s) *latency_s = j.t_finish - j.t_submit;
    }
    srv->free_results(j);
    srv->jobs.erase(it);
    return st;
}

gac_status gac_server_poll(gac_server *srv, uint64_t job_id, int *done, gac_result *out, double *latency_s) {
    clear_error();
    if (!srv || !done) return fail(GAC_ERR_INVALID_ARG, "srv and done must not be NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return fail(GAC_ERR_UNKNOWN_JOB, "no job %llu", static_cast<unsigned long long>(job_id));
    const JobState s = it->second->state;
    if (s != JobState::Done && s != JobState::Failed && s != JobState::Cancelled) {
        *done = 0;
        return GAC_OK;
    }
    *done = 1;
    return deliver(srv, it, out, latency_s);
}

gac_status gac_server_wait(gac_server *srv, uint64_t job_id, double timeout_s, gac_result *out, double *latency_s) {
    clear_error();
    if (!srv) return fail(GAC_ERR_INVALID_ARG, "srv must not be NULL");
    if (!(timeout_s >= 0.0)) return fail(GAC_ERR_INVALID_ARG, "timeout_s must be >= 0");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return fail(GAC_ERR_UNKNOWN_JOB, "no job %llu", static_cast<unsigned long long>(job_id));
    auto jp = it->second;
    // timeouts beyond a year wait a year at a time (the clock's duration type
    // would overflow); the job's state is re-checked after every wake-up
    const double kMaxWait = 3.15e7;
    auto done = [&] {
        return jp->state == JobState::Done || jp->state == JobState::Failed || jp->state == JobState::Cancelled;
    };
    bool ok = false;
    for (double left = timeout_s; !ok;) {
        const double chunk = std::min(left, kMaxWait);
        ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(chunk), done);
        left -= chunk;
        if (left <= 0.0) break;
    }
    if (!ok) return fail(GAC_ERR_TIMEOUT, "job %llu not done after %.3f s", static_cast<unsigned long long>(job_id), timeout_s);
    // another thread may have collected the job (poll or wait) meanwhile
    it = srv->jobs.find(job_id);
    if (it == srv->jobs.end() || it->second != jp)
        return fail(GAC_ERR_UNKNOWN_JOB, "job %llu was collected by another call", static_cast<unsigned long long>(job_id));
    return deliver(srv, it, out, latency_s);
}

gac_status gac_server_cancel(gac_server *srv, uint64_t job_id) {
    clear_error();
    if (!srv) return fail(GAC_ERR_INVALID_ARG, "srv must not be NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return fail(GAC_ERR_UNKNOWN_JOB, "no job %llu", static_cast<unsigned long long>(job_id));
    Job &j = *it->second;
    if (j.state == JobState::Queued || j.state == JobState::Uploading || j.state == JobState::Running)
        j.cancel = true;
    srv->cv_work.notify_all();
    return GAC_OK;
}

gac_status gac_server_get_stats(gac_server *srv, gac_server_stats *st) {
    clear_error();
    if (!srv || !st) return fail(GAC_ERR_INVALID_ARG, "srv and st must not be NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    st->queued = static_cast<int64_t>(srv->queue.size());
    st->resident = static_cast<int64_t>(srv->resident.size());
    st->finished = srv->finished;
    st->rounds = srv->rounds;
    st->bytes_in_use = srv->in_use;
    st->budget = srv->budget;
    st->gpu_s = srv->t_gpu;
    st->round_host_s = srv->t_round_host;
    st->admit_s = srv->t_admit;
    return GAC_OK;
}

gac_status gac_server_destroy(gac_server *srv) {
    clear_error();
    if (!srv) return fail(GAC_ERR_INVALID_ARG, "srv must not be NULL");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->thr.joinable()) srv->thr.join();
    if (!srv->started) {
        for (auto &kv : srv->jobs) {
            srv->free_job(*kv.second);
            srv->free_results(*kv.second);
        }
    }
    delete srv;
    return GAC_OK;
}

}  // extern "C"
