"""Benchmark of the voxel-wise MH sampler (GACELLE mcmc.m hot path) on GB300.

One step = one gac_mcmc_run over the whole workload (every step of the path:
load, initialise, propose, forward model, likelihood, accept, thin/store,
moments).  Default workload: the 3-pool complex myelin-water model at
1,000,000 voxels x 4 chains x 5,000 iterations (burn-in 500, thinning 100,
samples stored), synthetic seeded data, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mwi3_1m|smt_1p5m|monoexp_4k] [--no-extras]

Prints one JSON line (rank 0).  At one GPU on the default workload the line
also carries `workloads` (the mono-exponential 4k and the Standard Model 1.5M
workloads, each timed like the headline) and `serving` (the 200-job serving
trace, continuous batching against one launch per job, Poisson arrivals and
all at t = 0), each with the clocks sampled while it ran.  Under torchrun each rank samples its own
volume of the same size (voxel_base = rank * N: weak scaling, no collective on
the data path; the barrier and max-over-ranks timing use the process group).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_22094_gb300 import workloads as W  # noqa: E402

METRIC = "voxel-MCMC chain-iterations/s"
UNIT = "chain-iter/s"

# Algorithmic operation counts per chain-iteration of the direct form of each
# model (every echo evaluated with its own exp / sin / cos), counted from the
# oracle's expression tree.  MUFU operations by the special-function op that
# serves them: ex2 (exp; erf counted as one exp-class op), sin (sin and cos),
# lg2 (log), sqrt, rcp.  FP32 = add/mul/fma/min/max; INT = Philox (10 rounds x
# (2 wide multiplies, 2 three-input xors, 2 key adds) per call).
#   3-pool: 24 echoes x 3 pools x (exp, sin, cos) + 3 rcp (1/T2*) + Box-Muller
#     5 pairs x (log, sqrt, sin, cos) + the acceptance log = 240
#   SMT: 6 b-values x (exp + 2 g, g = sqrt, erf, rcp) + 2 pairs + log = 51
#   mono-exp: 12 exp + 1 pair + log = 17
#   AxCaliberSMT: 2 timings x 18 cylinder-series terms x 3 exp + 16
#     measurements x (2 exp + 2 g) + 2 pairs + log = 245
OPS = {
    "mwi3_1m": dict(mufu=dict(ex2=72, sin=154, lg2=6, sqrt=5, rcp=3), fp32=520, int=180),
    "smt_1p5m": dict(mufu=dict(ex2=18, sin=4, lg2=3, sqrt=14, rcp=12), fp32=103, int=120),
    "monoexp_4k": dict(mufu=dict(ex2=12, sin=2, lg2=2, sqrt=1), fp32=65, int=60),
    "axcal_250k": dict(mufu=dict(ex2=172, sin=4, lg2=3, sqrt=34, rcp=32), fp32=888, int=120),
}
# Ensemble walker-move counts: the same model evaluation, one Philox call, no
# Box-Muller; the acceptance log and the stretch z's log, a few FP32 ops.
OPS_ENSEMBLE = {
    "mwi3_1m": dict(mufu=dict(ex2=72, sin=144, lg2=2, rcp=3), fp32=490, int=60),
    "smt_1p5m": dict(mufu=dict(ex2=18, lg2=2, sqrt=12, rcp=12), fp32=92, int=60),
    "monoexp_4k": dict(mufu=dict(ex2=12, lg2=2), fp32=64, int=60),
    "axcal_250k": dict(mufu=dict(ex2=172, lg2=2, sqrt=32, rcp=32), fp32=874, int=60),
}
# Data-sheet rates per SM clock, used only when the pipe-rate probe cannot run.
MUFU_PER_CLK_SM = 16
FP32_PER_CLK_SM = 128
ISSUE_PER_CLK_SM = 4  # warp-instructions


def _pipe_rates(gac, stream):
    """Results per SM clock of each arithmetic pipe operation, measured by the
    library's probe kernels (None if the probe fails)."""
    try:
        return {op: gac.gac_pipe_rate(op, stream) for op in gac.PIPE_OPS}
    except Exception:  # noqa: BLE001 - the roofline then falls back to the data sheet
        return None


def _alu_peaks(mix: dict, rates):
    """(MUFU results per SM clock for this operation mix, FP32 per SM clock,
    basis): the mix's time is sum_op n_op / rate_op."""
    if not rates:
        return MUFU_PER_CLK_SM, FP32_PER_CLK_SM, "data sheet"
    n = sum(mix.values())
    mufu = n / sum(k / rates[op] for op, k in mix.items())
    return mufu, rates["ffma"], "measured by the pipe-rate probe"

# From the ncu captures summarised under profiles/: DRAM bytes of one full
# launch of the sampler kernel (read + write) and executed warp instructions
# per 32 chain-iterations.  Reported only while the kernel's sources (their
# code: comments and layout aside) hash to the value they were measured with
# (otherwise null).
KERNEL_SOURCES = ("include/gac.h", "paper_2511_22094_gb300/csrc/mh_kernel.cuh",
                  "paper_2511_22094_gb300/csrc/models.cuh", "paper_2511_22094_gb300/csrc/philox.cuh")
# the measured kernel's own file; the lane-split kernel (the 4,096-voxel
# workload's) also depends on mh_split.cuh, the one-thread kernel does not
KIND_SOURCE = {"mwi3_1m": ("mh_mwi3.cu",), "smt_1p5m": ("mh_smt.cu",),
               "monoexp_4k": ("mh_monoexp.cu", "mh_split.cuh"), "axcal_250k": ("mh_axcal.cu",)}
MEASURED = {
    # traffic: DRAM bytes of a quarter-size launch (262,144 / 393,216 / 65,536
    # voxels, all iterations, so every term scales with the voxels) x 3.81;
    # the lines still in L2 when the small launch ends are not counted
    # (~1-3% of its writes).  warp_instr: from the small-case --set full captures.
    "mwi3_1m": dict(sources="a8792946f2bdfa8f", traffic_bytes=(78.07e6 + 1696.83e6) * 1e6 / 262144, warp_instr=918.8),
    "smt_1p5m": dict(sources="559b4e0b19e2b689", traffic_bytes=(32.19e6 + 1120.72e6) * 1.5e6 / 393216, warp_instr=495.2),
    "axcal_250k": dict(sources="493f595b548eebc5", traffic_bytes=(37.59e6 + 910.33e6) * 250000 / 65536, warp_instr=1215.1),
    # the lane-split kernel (2 lanes a chain): the 4,096-voxel workload's data
    # and samples stay in L2, so no DRAM figure
    "monoexp_4k": dict(sources="cd550974b7613703", traffic_bytes=None, warp_instr=368.8),
}


_C_TOKENS = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'', re.S)


def _code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace runs collapsed:
    edits to comments and layout leave the hash (and the kernel) unchanged."""
    text = _C_TOKENS.sub(lambda m: " " if m.group(0)[0] == "/" else m.group(0), text)
    return " ".join(text.split())


def _sources_hash(workload: str) -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES + tuple("paper_2511_22094_gb300/csrc/" + f for f in KIND_SOURCE[workload]):
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _measured(workload: str, sampler: str) -> dict:
    m = MEASURED.get(workload) if sampler == "mh" else None
    if not m or m["sources"] != _sources_hash(workload):
        return {}
    return m


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class RankGroup:
    """The benchmark's ranks: one process per GPU under torchrun (RANK,
    LOCAL_RANK, WORLD_SIZE and MASTER_* from the environment).  The process
    group carries only the barrier around the timed region and the
    max-over-ranks time; no collective touches the sampler's data."""

    def __init__(self, backend: str = "nccl"):
        self.world, self.rank, self.local = _dist()
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self, cuda: bool = True):
        if self.pg is not None:
            self.pg.barrier()
        if cuda:
            import torch
            torch.cuda.synchronize()

    def max_time(self, t: float, device) -> float:
        """The largest of the ranks' times (every rank gets it)."""
        if self.pg is None:
            return t
        import torch
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        self.pg.all_reduce(tt, op=self.pg.ReduceOp.MAX)
        return float(tt.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()
            self.pg = None


def weak_value(world: int, units_per_rank_step: int, steps: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank_step * steps / t_max


def _host_inputs_for_oracle(w, n):
    import oracle
    th = W.truths(w, 0, n)
    sig = W.sigma(w, th)
    y = W.noisy_data(oracle.forward(w.kind, w.acq, th), W.noise(w, 0, n), sig)
    return y, sig


def cpu_oracle_rate(w, target_s=15.0, sampler="mh", stretch=2.0):
    """Oracle (as it stands) on a bounded voxel sample of the workload, all
    host cores; returns (chain-iterations/s, threads, sample description)."""
    import oracle
    oracle.build()
    kw = dict(iterations=w.iterations, burnin=w.burnin, thin=w.thin, seed=w.mcmc_seed)

    def run(y, sig):
        if sampler == "ensemble":
            return oracle.ensemble_run(w.kind, w.acq, w.lb, w.ub, y, sig, n_walkers=w.n_chains,
                                       stretch=stretch, **kw)
        return oracle.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, n_chains=w.n_chains, **kw)

    pilot = 8
    y, sig = _host_inputs_for_oracle(w, pilot)
    t0 = time.perf_counter()
    run(y, sig)
    per_vox = (time.perf_counter() - t0) / pilot
    threads = oracle.max_threads()
    n = int(max(threads, min(w.n_vox, target_s / max(per_vox, 1e-9))))
    n = max(threads, (n // threads) * threads)
    y, sig = _host_inputs_for_oracle(w, n)
    t0 = time.perf_counter()
    r = run(y, sig)
    dt = time.perf_counter() - t0
    ci = n * w.n_chains * w.iterations
    return ci / dt, r["threads"], f"first {n} of {w.n_vox} voxels, all {w.n_chains} chains x {w.iterations} iterations ({dt:.1f} s)"


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_oracle_study(args):
    """The oracle's timing protocol: for every workload, chain-iterations/s of
    the FP64 oracle on all host cores and on one core (the paper's CPU
    baseline is one core), each the median of `repeats` runs on a bounded
    voxel sample (about `target` seconds a run), with the host described."""
    import platform

    import oracle
    oracle.build()
    repeats, target = 5, 2.0
    host = {"nproc": os.cpu_count(), "omp_threads": oracle.max_threads(), "cpu": _cpu_model(),
            "machine": platform.machine()}
    res = {}
    for name in ("monoexp_4k", "mwi3_1m", "smt_1p5m", "axcal_250k"):
        w = W.WORKLOADS[name]
        for label, nt in (("all_cores", 0), ("one_core", 1)):
            def run(n):
                y, sig = _host_inputs_for_oracle(w, n)
                t0 = time.perf_counter()
                r = oracle.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, n_chains=w.n_chains,
                                    iterations=w.iterations, burnin=w.burnin, thin=w.thin, seed=w.mcmc_seed,
                                    n_threads=nt)
                return time.perf_counter() - t0, r["threads"]
            dt, threads = run(threads_pilot := max(1, oracle.max_threads() if nt == 0 else 1))
            per_vox = dt / threads_pilot
            n = int(min(w.n_vox, max(threads, target / max(per_vox, 1e-9))))
            n = max(threads, (n // threads) * threads)
            rates = []
            for _ in range(repeats):
                dt, _ = run(n)
                rates.append(n * w.n_chains * w.iterations / dt)
            res.setdefault(name, {})[label] = {"value": float(np.median(rates)), "unit": UNIT, "threads": threads,
                                               "sample": f"first {n} voxels, all {w.n_chains} chains x "
                                                         f"{w.iterations} iterations; median of {repeats}",
                                               "min": float(min(rates)), "max": float(max(rates))}
    print(json.dumps({"metric": "oracle " + METRIC, "unit": UNIT, "host": host, "workloads": res}), flush=True)


FIT_METRIC = "whole-volume fit voxel-iterations/s"
FIT_UNIT = "voxel-iter/s"
# Algorithmic bytes of one voxel-update of the 3-pool fit: data row 48 x 4,
# parameters in and out 2 x 9 x 4, Adam moments in and out 4 x 9 x 4, mask 1,
# weight 4
FIT_BYTES = 48 * 4 + 2 * 9 * 4 + 4 * 9 * 4 + 1 + 4
# Direct-form counts per voxel-iteration of the 3-pool fit (24 echoes x 3
# pools: exp, sin, cos and 18 Jacobian entries per echo; Adam on 9 parameters)
FIT_OPS = dict(mufu=24 * 3 * 3, fp32=24 * (3 * 14 + 2 * 9 * 2) + 9 * 12)


def _fit_problem(w, shape):
    """The workload's volume as a grid, its truths' data, a start at the
    centre of the prior box, and a mask without the outer layer of voxels."""
    N = int(np.prod(shape))
    th = W.truths(w, 0, N)
    y = None  # built on the device by the caller
    theta0 = np.tile(0.5 * (np.array(w.lb) + np.array(w.ub)), (N, 1))
    x, yy, z = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    inner = ((x > 0) & (x < shape[0] - 1) & (yy > 0) & (yy < shape[1] - 1) & (z > 0) & (z < shape[2] - 1))
    mask = inner.transpose(2, 1, 0).reshape(-1).astype(np.uint8)  # voxel v = x + nx (y + ny z)
    return th, y, theta0, mask


def run_fit(args):
    """Whole-volume Adam fit (askadam.m, Sec. 2.2.1) of the 3-pool model on a
    100^3 grid (the 1M-voxel volume): L1 loss, Adam (lr 0.01), 3D total
    variation on the myelin-water amplitude (lambda 1e-3), `--fit-iterations`
    updates per step from the same start."""
    import torch
    from paper_2511_22094_gb300 import build
    build.build()
    from paper_2511_22094_gb300 import gac

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream()
    w = W.MWI3_1M
    shape = (100, 100, 100)
    N, P, M = int(np.prod(shape)), w.n_par, w.n_meas
    it = args.fit_iterations
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th_true, _, theta0, mask = _fit_problem(w, shape)
    th = torch.from_numpy(th_true).to(dev)
    sig = torch.from_numpy(W.sigma(w, th_true)).to(dev)
    s = torch.empty((N, M), dtype=torch.float64, device=dev)
    gac.gac_forward(mid, th, N, gac.PREC_FP64, s, stream)
    z = torch.from_numpy(W.noise(w, 0, N)).to(dev)
    y = (s + sig.double()[:, None] * z).float().contiguous()
    del s, z, th
    mk = torch.from_numpy(mask).to(dev)
    wt = (1.0 / sig).float().contiguous()  # volumetric weights ~ SNR (Eq. 1)
    th0 = torch.from_numpy(theta0).to(dev)
    theta = torch.empty_like(th0)
    hist = torch.empty(it, dtype=torch.float64, device=dev)
    opts = gac.make_fit_opts(shape, loss=gac.FIT_L1, iterations=it, learning_rate=0.01, tv_lambda=1e-3,
                             tv_params=0b1, tv_dims=3, precision=gac.PREC_FP32)

    def step():
        theta.copy_(th0)
        return gac.gac_fit_run(mid, y, mk, wt, opts, theta, hist, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for e0, e1 in ev:
            e0.record(stream)
            done = step()
            e1.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    t_total = sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3
    vi = N * it
    value = vi * args.steps / t_total
    # end to end: host (pinned) buffers in and out through the same call
    hy, hmk, hwt = y.cpu().pin_memory(), mk.cpu().pin_memory(), wt.cpu().pin_memory()
    hth = torch.empty((N, P), dtype=torch.float64).pin_memory()
    hh = torch.empty(it, dtype=torch.float64).pin_memory()
    h0 = torch.from_numpy(theta0)
    reps = max(1, min(args.steps, 3))
    hth.copy_(h0)
    gac.gac_fit_run(mid, hy, hmk, hwt, opts, hth, hh, stream)  # warm-up
    t0 = time.perf_counter()
    for _ in range(reps):
        hth.copy_(h0)
        gac.gac_fit_run(mid, hy, hmk, hwt, opts, hth, hh, stream)
    e2e_s = (time.perf_counter() - t0) / reps
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = (_peaks().get("sm_max_mhz") or 2070.0) * 1e6
    vi_s = vi / (t_total / args.steps)
    rates = _pipe_rates(gac, stream)
    fp32_clk = rates["ffma"] if rates else FP32_PER_CLK_SM
    peak = sms * fp32_clk * f_max / 1e9
    achieved = FIT_OPS["fp32"] * vi_s / 1e9
    hbm = _peaks().get("hbm_gbs")
    hbm_peak, hbm_basis = (hbm, "measured copy bandwidth") if hbm else (6800.0, "fallback")
    ach_gbs = FIT_BYTES * vi_s / 1e9
    line = {"metric": FIT_METRIC, "value": value, "unit": FIT_UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "mwi3_1m as a 100^3 grid", "loss": "L1", "optimiser": "Adam lr 0.01",
                       "tv": "3D, A_MW, lambda 1e-3", "mask": "inner 98^3", "iterations_per_step": it,
                       "updates_done": done},
            "roofline": {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ach_gbs / hbm_peak, "traffic": None, "peak_basis": hbm_basis,
                         "bytes_per_unit": FIT_BYTES,
                         "direct_form_equivalent": {
                             "pipe": "fp32", "count": "direct-form", "achieved": achieved, "peak": peak,
                             "unit": "Gop/s", "ratio": achieved / peak,
                             "peak_basis": f"{sms} SMs x {fp32_clk:.2f}/clk ("
                                           f"{'measured by the pipe-rate probe' if rates else 'data sheet'}) x "
                                           f"{f_max / 1e6:.0f} MHz (max SM clock)"}},
            "pipe_rates_per_sm_clk": rates,
            "e2e": {"value": vi / e2e_s, "unit": FIT_UNIT, "h2d_bytes_per_step": y.numel() * 4 + N * (1 + 4 + 8 * P),
                    "d2h_bytes_per_step": N * 8 * P + it * 8},
            "clocks": clocks, "gpu_launches": args.steps * (2 * it + 2), "wall_s": t_wall}
    if not args.no_cpu_baseline:
        import oracle
        sub = (20, 20, 20)
        ns = int(np.prod(sub))
        th_s, _, theta0_s, mask_s = _fit_problem(w, sub)
        ys = W.noisy_data(oracle.forward(w.kind, w.acq, th_s), W.noise(w, 0, ns), W.sigma(w, th_s))
        its = 1000
        t0 = time.perf_counter()
        oracle.fit_run(w.kind, w.acq, w.lb, w.ub, ys, theta0_s, shape=sub, mask=mask_s,
                       weight=1.0 / W.sigma(w, th_s), loss=1, iterations=its, lr=0.01, lam=1e-3, tv_params=1,
                       tv_dims=3)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ns * its / dt, "unit": FIT_UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"20^3 voxels x {its} updates ({dt:.1f} s)"}
    print(json.dumps(line), flush=True)


def run_reference(args, w):
    """Reference arm: the FP64 CPU oracle, timed on the host cores."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    rates = []
    for i in range(args.warmup + args.steps):
        rate, threads, sample = cpu_oracle_rate(w, target_s=max(5.0, 60.0 / max(args.steps + args.warmup, 1)),
                                                sampler=args.sampler, stretch=args.stretch)
        if i >= args.warmup:
            rates.append(rate)
    value = float(np.median(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": w.chain_iterations / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_vox": w.n_vox, "n_chains": w.n_chains,
                       "iterations": w.iterations, "burnin": w.burnin, "thin": w.thin},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _roofline(base_name, sampler, ci_s, rates, sms, clocks, meas):
    """The ALU roofline of a sampler workload at ci_s chain-iterations (or
    walker moves) per second.

    Headline (when an ncu count exists for the current kernel sources): the
    executed-instruction issue roofline, the warp instructions the kernel
    executes per chain-iteration (all pipes) against 4 warp-instructions per
    SM clock at the maximum SM clock -- the limit these issue- and
    FMA-pipe-bound kernels meet.  `direct_form_equivalent`: the model's
    direct-form MUFU and FP32+INT counts (every echo with its own exp, sin,
    cos) against the measured pipe rates; the kernels evaluate evenly spaced
    echoes by a recurrence and execute fewer special-function operations, so
    this ratio can exceed 1 and is not a fraction of a peak.  Without a count
    the headline falls back to it."""
    f_max = (_peaks().get("sm_max_mhz") or 2070.0) * 1e6
    ops = (OPS_ENSEMBLE if sampler == "ensemble" else OPS)[base_name]
    n_mufu = sum(ops["mufu"].values())
    mufu_clk, fp32_clk, rate_basis = _alu_peaks(ops["mufu"], rates)
    t_mufu = n_mufu / (sms * mufu_clk * f_max)
    t_alu = (ops["fp32"] + ops["int"]) / (sms * fp32_clk * f_max)
    if t_mufu >= t_alu:
        pipe, achieved, peak = "mufu", n_mufu * ci_s / 1e9, sms * mufu_clk * f_max / 1e9
        per_clk = mufu_clk
    else:
        pipe, achieved = "fp32+int", (ops["fp32"] + ops["int"]) * ci_s / 1e9
        peak = sms * fp32_clk * f_max / 1e9
        per_clk = fp32_clk
    f_med = (clocks.get("sm_mhz") or 0) * 1e6
    direct = {"pipe": pipe, "count": "direct-form", "achieved": achieved, "peak": peak, "unit": "Gop/s",
              "ratio": achieved / peak,
              "peak_basis": f"{sms} SMs x {per_clk:.2f}/clk ({rate_basis}) x {f_max / 1e6:.0f} MHz (max SM clock)"}
    if meas.get("warp_instr"):
        issue_peak = sms * ISSUE_PER_CLK_SM * f_max * 32 / 1e9  # thread-instructions / s, in G
        ach = meas["warp_instr"] * ci_s / 1e9  # thread-instructions / s (warp_instr per 32 units x 32 / 32)
        return {"bound": "alu", "pipe": "issue", "count": "executed (ncu: warp instructions per 32 chain-"
                "iterations, all pipes)", "achieved": ach, "peak": issue_peak, "unit": "Ginstr/s",
                "frac": ach / issue_peak, "frac_at_sampled_clock": (ach / issue_peak * f_max / f_med) if f_med else None,
                "peak_basis": f"{sms} SMs x {ISSUE_PER_CLK_SM} warp-instructions/clk x 32 lanes x "
                              f"{f_max / 1e6:.0f} MHz (max SM clock)",
                "warp_instr_per_32_units": meas["warp_instr"], "direct_form_equivalent": direct}
    return {"bound": "alu", "pipe": pipe, "count": "direct-form (no executed count for these sources)",
            "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
            "frac_at_sampled_clock": (achieved / peak * f_max / f_med) if f_med else None,
            "peak_basis": direct["peak_basis"], "direct_form_equivalent": direct}


def _device_inputs(gac, w, mid, dev, stream, base=0):
    """Seeded truths and noise of voxels [base, base + N); the signal from the
    library's own forward model on the device (FP64)."""
    import torch
    N, M = w.n_vox, w.n_meas
    th = torch.from_numpy(W.truths(w, base, N)).to(dev)
    sig = torch.from_numpy(W.sigma(w, th.cpu().numpy())).to(dev)
    s = torch.empty((N, M), dtype=torch.float64, device=dev)
    gac.gac_forward(mid, th, N, gac.PREC_FP64, s, stream)
    z = torch.from_numpy(W.noise(w, base, N)).to(dev)
    y = (s + sig.double()[:, None] * z).float().contiguous()
    return y, sig


def time_workload(gac, name, dev, stream, rates, steps=5, warmup=3):
    """One more single-GPU workload of the sampler, timed like the headline
    (inputs resident in HBM, samples stored, CUDA events on the launching
    stream, clocks sampled during the timed region); its own line's figures."""
    import torch
    w = W.WORKLOADS[name]
    N, C, P, S = w.n_vox, w.n_chains, w.n_par, w.n_samples
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    y, sig = _device_inputs(gac, w, mid, dev, stream)
    out = dict(mean=torch.empty((P, N), dtype=torch.float64, device=dev),
               std=torch.empty((P, N), dtype=torch.float64, device=dev),
               samples=torch.empty((S, C, P, N), dtype=torch.float32, device=dev),
               accept_rate=torch.empty((C, N), dtype=torch.float32, device=dev),
               nonfinite=torch.empty((C, N), dtype=torch.int32, device=dev))
    opts = gac.make_opts(w.iterations, w.burnin, w.thin, C, w.mcmc_seed)
    for _ in range(warmup):
        gac.gac_mcmc_run(mid, y, N, sig, 0.0, None, opts, out, stream)
    torch.cuda.synchronize()
    # a short workload runs more steps, so that the clocks are sampled (every
    # 200 ms) while it runs: at least ~1.5 s of timed kernel time
    t0 = time.perf_counter()
    gac.gac_mcmc_run(mid, y, N, sig, 0.0, None, opts, out, stream)
    torch.cuda.synchronize()
    steps = int(min(4000, max(steps, np.ceil(1.5 / max(time.perf_counter() - t0, 1e-6)))))
    # buffers that fit in L2 (129 MB) are evicted before every step by writing
    # a larger buffer outside the timed events
    touched = sum(t.numel() * t.element_size() for t in (y, sig, *out.values()))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if touched < (256 << 20) else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(dev.index or 0) as clk:
        torch.cuda.synchronize()
        for e0, e1 in ev:
            if flush is not None:
                flush.fill_(1)
            e0.record(stream)
            gac.gac_mcmc_run(mid, y, N, sig, 0.0, None, opts, out, stream)
            e1.record(stream)
        torch.cuda.synchronize()
    kernel_s = sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3 / steps
    ci = w.chain_iterations
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    roof = _roofline(name, "mh", ci / kernel_s, rates, sms, clocks, _measured(name, "mh"))
    l2 = ("flushed before every step (256 MB write outside the timed events)" if flush is not None else
          f"inputs + outputs {touched / 1e9:.1f} GB per step > 129 MB L2")
    del out, y, sig, flush
    torch.cuda.empty_cache()
    return {"value": ci / kernel_s, "unit": UNIT, "ms_per_step": kernel_s * 1e3, "steps": steps,
            "warmup": warmup, "config": {"n_vox": N, "n_chains": C, "iterations": w.iterations,
                                         "burnin": w.burnin, "thin": w.thin, "samples_stored": True, "l2": l2},
            "roofline": roof, "clocks": clocks, "gpu_launches": steps}


def run_ours(args, w):
    import torch
    from paper_2511_22094_gb300 import build
    build.build()
    from paper_2511_22094_gb300 import gac

    group = RankGroup("nccl")
    world, rank, local = group.world, group.rank, group.local
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream()

    from paper_2511_22094_gb300 import shard
    N, C, P, M = w.n_vox, w.n_chains, w.n_par, w.n_meas
    S = w.n_samples
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    base, _ = shard.weak_range(N, rank)  # this rank's slice of a volume of world * N voxels

    # synthetic inputs: seeded truths and noise; the signal from the library's
    # own forward model on the device
    y, sig = _device_inputs(gac, w, mid, dev, stream, base)
    out = dict(mean=torch.empty((P, N), dtype=torch.float64, device=dev),
               std=torch.empty((P, N), dtype=torch.float64, device=dev),
               samples=torch.empty((S, C, P, N), dtype=torch.float32, device=dev),
               accept_rate=torch.empty((C, N), dtype=torch.float32, device=dev),
               nonfinite=torch.empty((C, N), dtype=torch.int32, device=dev))
    if args.rhat and args.sampler == "mh":
        out["rhat"] = torch.empty((P, N), dtype=torch.float64, device=dev)
        out["step_scale"] = torch.empty((C, N), dtype=torch.float32, device=dev)
    prec = {"mixed": gac.PREC_MIXED, "fp32": gac.PREC_FP32, "fp64": gac.PREC_FP64}[args.precision]
    opts = gac.make_opts(w.iterations, w.burnin, w.thin, C, w.mcmc_seed, voxel_base=base, precision=prec,
                         moments_mode=gac.MOMENTS_ALL_POSTBURNIN if args.moments == "all" else gac.MOMENTS_THINNED,
                         adapt_window=args.adapt_window, adapt_target=args.adapt_target if args.adapt_window else 0.0,
                         lanes_per_chain=args.lanes)

    def step():
        if args.sampler == "ensemble":
            gac.gac_ensemble_run(mid, y, N, sig, 0.0, None, opts, args.stretch, out, stream)
        else:
            gac.gac_mcmc_run(mid, y, N, sig, 0.0, None, opts, out, stream)

    barrier = group.barrier

    rates = _pipe_rates(gac, stream)  # the roofline's denominators, before any timing
    for _ in range(args.warmup):
        step()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        for e0, e1 in ev:
            e0.record(stream)
            step()
            e1.record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    per_step = [e0.elapsed_time(e1) / 1e3 for e0, e1 in ev]
    t_total = group.max_time(sum(per_step), dev)
    ci_per_step = N * C * w.iterations
    value = weak_value(world, ci_per_step, args.steps, t_total)
    kernel_s = t_total / args.steps

    # end to end through the same public call with pinned host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        hy = y.cpu().pin_memory()
        hs = sig.cpu().pin_memory()
        hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
        h2d = hy.numel() * 4 + hs.numel() * 4
        d2h = sum(v.numel() * v.element_size() for v in hout.values())
        run = (lambda o: gac.gac_ensemble_run(mid, hy, N, hs, 0.0, None, opts, args.stretch, o, stream)) \
            if args.sampler == "ensemble" else (lambda o: gac.gac_mcmc_run(mid, hy, N, hs, 0.0, None, opts, o, stream))
        run(hout)  # warm the allocator
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(reps):
            run(hout)
            _ = float(hout["accept_rate"][0, 0])  # read the result on the host
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / reps
        e2e = {"value": ci_per_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3}

    if rank != 0:
        group.close()
        return
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    base_name = w.name.replace("_ensemble", "")
    meas = _measured(base_name, args.sampler) if (world == 1 and args.precision == "mixed") else {}
    roof = _roofline(base_name, args.sampler, ci_per_step / kernel_s, rates, sms, clocks, meas)
    roof["traffic"] = (meas.get("traffic_bytes") if N == W.WORKLOADS[base_name].n_vox and not args.rhat
                       and not args.adapt_window and args.moments == "thinned" else None)
    roof["kernel_ms"] = kernel_s * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "fp32": "f32", "fp64": "f64"}[args.precision],
            "data": "synthetic (seeded truths + Gaussian noise, signal from the library's forward model)",
            "config": {"workload": w.name, "sampler": args.sampler, "n_vox": N,
                       ("n_walkers" if args.sampler == "ensemble" else "n_chains"): C, "iterations": w.iterations,
                       "burnin": w.burnin, "thin": w.thin, "samples_stored": True,
                       "precision": args.precision, "parallelism": f"voxel-shard x{world}",
                       "adapt_window": args.adapt_window, "moments": args.moments,
                       "rhat_and_step_scale": bool(args.rhat and args.sampler == "mh"),
                       "lanes_per_chain": args.lanes or "library's choice",
                       "l2": f"inputs {y.numel() * 4 / 1e6:.0f} MB + samples {S * C * P * N * 4 / 1e9:.1f} GB written per step > 129 MB L2"},
            "roofline": roof, "pipe_rates_per_sm_clk": rates, "clocks": clocks, "gpu_launches": args.steps,
            "wall_s": t_wall}
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline:
        rate, threads, sample = cpu_oracle_rate(w, sampler=args.sampler, stretch=args.stretch)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": sample}
    if world == 1 and not args.no_extras and args.sampler == "mh" and w.name == "mwi3_1m" \
            and args.n_vox is None and args.iterations is None:
        # the other single-GPU workloads and the serving trace, measured in the
        # same run (after the headline's timed region, which they do not touch)
        del out, y, sig
        torch.cuda.empty_cache()
        line["workloads"] = {name: time_workload(gac, name, dev, stream, rates)
                             for name in ("monoexp_4k", "smt_1p5m")}
        line["serving"] = serving_study(gac, dev, 200, saturated=True)
    print(json.dumps(line), flush=True)
    group.close()


def run_serving(args):
    """The serving study alone (see serving_study), as its own JSON line."""
    import torch
    from paper_2511_22094_gb300 import build
    build.build()
    from paper_2511_22094_gb300 import gac

    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    print(json.dumps(serving_study(gac, dev, args.serving_jobs, args.serving_saturated)), flush=True)


def serving_study(gac, dev, n_jobs=200, saturated=True):
    """Serving trace: 200 jobs with Poisson arrivals (mean gap 0.2 s), mixed
    models, 10k-2M voxels, 1-4 chains, 1k-5k iterations, under a 120 GB HBM
    budget.  Continuous batching (gac_server_*) against the plain form: the
    same jobs run one gac_mcmc_run after another in arrival order.  Inputs
    start in pinned host memory and results end there in both forms.  With
    `saturated`, the same jobs also all arrive at t = 0.  Each pass carries
    the clocks sampled while it ran."""
    import torch
    trace = W.serving_trace(n_jobs=n_jobs)
    mids = {}
    jobs = []
    t_prep = time.perf_counter()
    for tj in trace:
        w = tj.workload
        key = w.kind
        if key not in mids:
            mids[key] = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
        mid = mids[key]
        th = torch.from_numpy(W.truths(w, tj.first_voxel, w.n_vox)).to(dev)
        sig = torch.from_numpy(W.sigma(w, th.cpu().numpy())).to(dev)
        s = torch.empty((w.n_vox, w.n_meas), dtype=torch.float64, device=dev)
        gac.gac_forward(mid, th, w.n_vox, gac.PREC_FP64, s)
        g = torch.Generator(device=dev).manual_seed(1_000_003 * (tj.index + 1))
        z = torch.randn((w.n_vox, w.n_meas), dtype=torch.float64, device=dev, generator=g)
        y = (s + sig.double()[:, None] * z).float()
        hy = torch.empty(y.shape, dtype=torch.float32).pin_memory()
        hy.copy_(y)
        hs = torch.empty(sig.shape, dtype=torch.float32).pin_memory()
        hs.copy_(sig)
        opts = gac.make_opts(w.iterations, w.burnin, w.thin, w.n_chains, w.mcmc_seed)
        jobs.append(dict(tj=tj, mid=mid, y=hy, sig=hs, opts=opts, ci=w.chain_iterations,
                         P=w.n_par, N=w.n_vox, C=w.n_chains))
        del th, sig, s, z, y
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t_prep

    def outs(j):
        return dict(mean=np.empty((j["P"], j["N"])), std=np.empty((j["P"], j["N"])),
                    accept_rate=np.empty((j["C"], j["N"]), np.float32),
                    nonfinite=np.empty((j["C"], j["N"]), np.int32))

    def summarize(lat, makespan):
        lat = np.asarray(lat)
        ci = sum(j["ci"] for j in jobs)
        return {"throughput": ci / makespan, "unit": UNIT, "makespan_s": makespan,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean())}

    def serve_pass(compress):
        srv = gac.gac_server_create(120 << 30, 64)
        ids, lat = [], [None] * len(jobs)
        done_t = [0.0] * len(jobs)
        t0 = time.perf_counter()

        def waiter():
            for i, jid in enumerate(ids_q):
                while jid[0] is None:
                    time.sleep(0.0005)
                lat[i] = gac.gac_server_wait(srv, jid[0], 3600.0, outs(jobs[i]))
                done_t[i] = time.perf_counter() - t0
        ids_q = [[None] for _ in jobs]
        th = threading.Thread(target=waiter)
        th.start()
        for i, j in enumerate(jobs):
            at = j["tj"].arrival_s * compress
            dt = t0 + at - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids_q[i][0] = gac.gac_server_submit(srv, j["mid"], j["y"], j["N"], j["sig"], 0.0, j["opts"])
        th.join()
        st = gac.gac_server_get_stats(srv)
        gac.gac_server_destroy(srv)
        r = summarize(lat, max(done_t))
        r["rounds"] = st["rounds"]
        r["scheduler_s"] = {"gpu_wait": st["gpu_s"], "round_prep": st["round_host_s"], "admit_retire": st["admit_s"]}
        return r

    def sequential_pass(compress):
        lat, t0 = [], time.perf_counter()
        end = 0.0
        for j in jobs:
            at = j["tj"].arrival_s * compress
            dt = t0 + at - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            gac.gac_mcmc_run(j["mid"], j["y"], j["N"], j["sig"], 0.0, None, j["opts"], outs(j))
            end = time.perf_counter() - t0
            lat.append(end - at)
        return summarize(lat, end)

    def clocked(fn, compress):
        with ClockSampler(dev.index or 0) as clk:
            r = fn(compress)
        r["clocks"] = clk.summary()
        return r

    # warm up both paths on the first few jobs
    for j in jobs[:3]:
        gac.gac_mcmc_run(j["mid"], j["y"], j["N"], j["sig"], 0.0, None, j["opts"], outs(j))
    res = {"continuous_batching": clocked(serve_pass, 1.0), "sequential": clocked(sequential_pass, 1.0)}
    if saturated:
        res["continuous_batching_all_at_t0"] = clocked(serve_pass, 0.0)
        res["sequential_all_at_t0"] = clocked(sequential_pass, 0.0)
    for a, b in (("continuous_batching", "sequential"), ("continuous_batching_all_at_t0", "sequential_all_at_t0")):
        if a in res:
            res[a]["vs_sequential"] = {"throughput": res[a]["throughput"] / res[b]["throughput"],
                                       "p50_speedup": res[b]["p50_s"] / res[a]["p50_s"],
                                       "p99_speedup": res[b]["p99_s"] / res[a]["p99_s"],
                                       "mean_speedup": res[b]["mean_s"] / res[a]["mean_s"]}
    return {"metric": "serving trace: throughput and job latency", "unit": UNIT,
            "trace": {"jobs": len(jobs), "arrivals": "Poisson, mean gap 0.2 s",
                      "span_s": trace[-1].arrival_s,
                      "chain_iterations": sum(j["ci"] for j in jobs),
                      "budget_bytes": 120 << 30, "max_resident": 64, "prep_s": t_prep},
            **res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="mwi3_1m", choices=sorted(W.WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=("mixed", "fp32", "fp64"), default="mixed")
    ap.add_argument("--sampler", choices=("mh", "ensemble"), default="mh")
    ap.add_argument("--stretch", type=float, default=2.0, help="ensemble stepSize a")
    ap.add_argument("--n-vox", type=int, default=None, help="smaller case (profiling only)")
    ap.add_argument("--iterations", type=int, default=None, help="smaller case (profiling only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, default=0, choices=(0, 1, 2, 4),
                    help="lanes per chain (0: the library chooses; results do not depend on it)")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline workload only (skip the other workloads and the serving trace)")
    ap.add_argument("--serving", action="store_true", help="run the serving trace instead")
    ap.add_argument("--serving-jobs", type=int, default=200)
    ap.add_argument("--serving-saturated", action="store_true")
    ap.add_argument("--fit", action="store_true", help="whole-volume Adam fit instead of MCMC")
    ap.add_argument("--fit-iterations", type=int, default=100)
    ap.add_argument("--adapt-window", type=int, default=0, help="burn-in step adaptation window (0: off)")
    ap.add_argument("--adapt-target", type=float, default=0.3, help="adaptation's target acceptance rate")
    ap.add_argument("--moments", choices=("thinned", "all"), default="thinned",
                    help="moments over the thinned samples or over every post-burn-in state")
    ap.add_argument("--rhat", action="store_true", help="also write R-hat and the final step multipliers")
    ap.add_argument("--oracle-study", action="store_true",
                    help="time the CPU oracle on all cores and on one core for every workload")
    args = ap.parse_args()
    if args.oracle_study:
        run_oracle_study(args)
        return
    if args.serving:
        run_serving(args)
        return
    if args.fit:
        run_fit(args)
        return
    w = W.WORKLOADS[args.workload]
    if args.sampler == "ensemble":
        # Table 1: 50 walkers x 2,000 iterations, 10% burn-in, thinning 100, at the
        # paper's largest speed-test size (2.5e5 voxels)
        w = w.with_(name=w.name + "_ensemble", n_vox=min(w.n_vox, 250_000), n_chains=50,
                    iterations=2000, burnin=200, thin=100)
    if args.n_vox is not None:
        w = w.with_(n_vox=args.n_vox)
    if args.iterations is not None:
        w = w.with_(iterations=args.iterations, burnin=min(w.burnin, args.iterations // 5))
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
