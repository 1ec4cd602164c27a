"""Continuous-batching server on the device.

Each job's result in a mix of concurrently resident jobs (different models,
voxel counts, chains and iteration counts, sliced into rounds) equals the same
job run alone through gac_mcmc_run: the random numbers depend only on (seed,
t, voxel, chain) and a slice resumes from the exact saved state.  Jobs that
do not fit the HBM budget wait and are admitted as memory frees up.
"""
import numpy as np
import pytest

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _jobs(orc, gac):
    specs = [  # (workload, voxels, chains, I, B, T, burn-in adaptation window)
        (W.MONOEXP_4K, 3000, 1, 700, 100, 5, 0),
        (W.MWI3_1M, 1500, 4, 600, 60, 20, 15),
        (W.SMT_1P5M, 2500, 3, 900, 90, 30, 0),
        (W.MONOEXP_4K, 257, 2, 1200, 120, 10, 0),
        (W.MWI3_1M, 333, 1, 400, 40, 40, 0),
        (W.SMT_1P5M, 64, 4, 350, 35, 7, 5),
        (W.MWI3_1M, 120_000, 4, 1500, 150, 50, 25),  # large: sliced over many rounds
    ]
    jobs = []
    for i, (w, n, C, I, B, T, Wa) in enumerate(specs):
        mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
        th, sig, y = make_voxels(orc, w, 1000 * i, n)
        opts = gac.make_opts(I, B, T, C, 77 + i, adapt_window=Wa, adapt_target=0.3 if Wa else 0.0)
        jobs.append((w, mid, y, sig, opts))
    return jobs


def _alone(gac, mid, y, sig, opts):
    return gac.run_host(mid, y, sig, iterations=opts.iterations, burnin=opts.burnin, thin=opts.thin,
                        n_chains=opts.n_chains, seed=opts.seed, adapt_window=opts.adapt_window,
                        adapt_target=opts.adapt_target)


def _out_like(ref):
    return {k: np.empty_like(v) for k, v in ref.items() if v is not None and k != "trace"}


def test_mix_equals_alone(gac, orc):
    jobs = _jobs(orc, gac)
    refs = [_alone(gac, mid, y, sig, opts) for (_, mid, y, sig, opts) in jobs]
    srv = gac.gac_server_create(8 << 30, 64)
    try:
        ids = [gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, opts, keep_samples=True)
               for (_, mid, y, sig, opts) in jobs]
        for jid, ref in zip(ids, refs):
            out = _out_like(ref)
            lat = gac.gac_server_wait(srv, jid, 300.0, out)
            assert lat > 0
            for k in ("samples", "accept_rate", "nonfinite", "step_scale"):
                np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
            np.testing.assert_allclose(out["mean"], ref["mean"], rtol=1e-12, atol=0)
            np.testing.assert_allclose(out["std"], ref["std"], rtol=1e-9, atol=0)
            np.testing.assert_allclose(out["rhat"], ref["rhat"], rtol=1e-9, atol=0)
        st = gac.gac_server_get_stats(srv)
        assert st["finished"] == len(jobs) and st["rounds"] > 1 and st["bytes_in_use"] == 0
    finally:
        gac.gac_server_destroy(srv)


def test_budget_queues_and_admits_as_memory_frees(gac, orc):
    jobs = _jobs(orc, gac)
    need = [gac.gac_server_job_bytes(mid, y.shape[0], opts, False, True) for (_, mid, y, sig, opts) in jobs]
    budget = max(need) + min(need)  # never room for all at once
    srv = gac.gac_server_create(budget, 64)
    try:
        ids = [gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, opts)
               for (_, mid, y, sig, opts) in jobs]
        st = gac.gac_server_get_stats(srv)
        assert st["bytes_in_use"] <= budget
        for jid, (_, mid, y, sig, opts) in zip(ids, jobs):
            ref = _alone(gac, mid, y, sig, opts)
            out = {"mean": np.empty_like(ref["mean"])}
            gac.gac_server_wait(srv, jid, 300.0, out)
            np.testing.assert_allclose(out["mean"], ref["mean"], rtol=1e-12)
    finally:
        gac.gac_server_destroy(srv)


def test_cancel_and_poll(gac, orc):
    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 20_000)
    srv = gac.gac_server_create(8 << 30, 8)
    try:
        # long enough (~0.6 s alone) that no single round can take it to the end,
        # so the cancel always lands before its last round is queued
        long_job = gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, gac.make_opts(200_000, 2000, 1000, 4, 1))
        short = gac.gac_server_submit(srv, mid, y[:100], 100, sig[:100], 0.0, gac.make_opts(200, 20, 10, 1, 2))
        gac.gac_server_cancel(srv, long_job)
        gac.gac_server_wait(srv, short, 120.0, {})
        with pytest.raises(gac.GacError) as e:
            gac.gac_server_wait(srv, long_job, 120.0, {})
        assert e.value.status == 8  # CANCELLED
        with pytest.raises(gac.GacError):
            gac.gac_server_poll(srv, short)  # already delivered and forgotten
        # poll of a running job reports not done
        j = gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, gac.make_opts(3000, 300, 100, 4, 3))
        done, _ = gac.gac_server_poll(srv, j)
        assert not done
        gac.gac_server_wait(srv, j, 300.0, {})
    finally:
        gac.gac_server_destroy(srv)


def test_destroy_with_jobs_in_flight(gac, orc):
    w = W.SMT_1P5M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 50_000)
    srv = gac.gac_server_create(8 << 30, 8)
    for i in range(3):
        gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, gac.make_opts(2000, 200, 100, 4, i))
    gac.gac_server_destroy(srv)  # must return without waiting for the jobs to finish


def test_cancel_while_rounds_are_in_flight(gac, orc):
    """Cancelling running jobs while later rounds are already queued: their
    memory returns only after those rounds, so jobs admitted into it and the
    job that keeps running all equal their runs alone."""
    import time
    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 40_000)
    srv = gac.gac_server_create(8 << 30, 16)
    try:
        # three jobs of ~0.1 s each alone, so the cancels land mid-run
        big = [gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, gac.make_opts(20000, 2000, 1000, 4, 10 + i))
               for i in range(3)]
        time.sleep(0.05)
        gac.gac_server_cancel(srv, big[0])
        gac.gac_server_cancel(srv, big[1])
        small = []
        for i in range(3):
            opts = gac.make_opts(800, 80, 20, 2, 20 + i)
            ys, ss = y[2000 * i:2000 * (i + 1)], sig[2000 * i:2000 * (i + 1)]
            small.append((gac.gac_server_submit(srv, mid, ys, 2000, ss, 0.0, opts, keep_samples=True), ys, ss, opts))
        for jid, ys, ss, opts in small:
            ref = _alone(gac, mid, ys, ss, opts)
            out = _out_like(ref)
            gac.gac_server_wait(srv, jid, 300.0, out)
            np.testing.assert_array_equal(out["samples"], ref["samples"])
            np.testing.assert_allclose(out["mean"], ref["mean"], rtol=1e-12, atol=0)
        opts = gac.make_opts(20000, 2000, 1000, 4, 12)
        ref = _alone(gac, mid, y, sig, opts)
        out = {"mean": np.empty_like(ref["mean"]), "accept_rate": np.empty_like(ref["accept_rate"])}
        gac.gac_server_wait(srv, big[2], 300.0, out)
        np.testing.assert_array_equal(out["accept_rate"], ref["accept_rate"])
        np.testing.assert_allclose(out["mean"], ref["mean"], rtol=1e-12, atol=0)
        for jid in big[:2]:
            with pytest.raises(gac.GacError):
                gac.gac_server_wait(srv, jid, 60.0, {})
    finally:
        gac.gac_server_destroy(srv)


def test_large_job_is_not_starved_by_small_arrivals(gac, orc):
    """A stream of small jobs, each finishing within one round, keeps arriving
    while a large job runs: small jobs take at most half of a round, so the
    large job still finishes within a few times its time alone."""
    import time
    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 60_000)
    big_opts = gac.make_opts(6000, 600, 100, 4, 1)
    t0 = time.perf_counter()
    gac.run_host(mid, y, sig, iterations=6000, burnin=600, thin=100, n_chains=4, seed=1, want_samples=False)
    alone = time.perf_counter() - t0
    srv = gac.gac_server_create(8 << 30, 64)
    try:
        big = gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, big_opts)
        small = []
        t_start = time.perf_counter()
        while True:
            done, lat = gac.gac_server_poll(srv, big)
            if done:
                break
            small.append(gac.gac_server_submit(srv, mid, y[:500], 500, sig[:500], 0.0,
                                               gac.make_opts(400, 40, 20, 2, 100 + len(small))))
            time.sleep(0.002)
            assert time.perf_counter() - t_start < 60.0
        for jid in small:
            gac.gac_server_wait(srv, jid, 60.0, {})
        print(f"large job alone {alone:.3f} s, in the stream {lat:.3f} s, {len(small)} small jobs")
        assert lat < 5.0 * alone + 1.0
        assert len(small) > 10
    finally:
        gac.gac_server_destroy(srv)


def test_all_postburnin_moments_jobs_equal_alone(gac, orc):
    """Moments over every post-burn-in state: the FP32 block partials carried
    between the server's slices give the same moments as one launch."""
    jobs = []
    for i, (w, n, C, I, B) in enumerate([(W.MWI3_1M, 3000, 4, 900, 100), (W.SMT_1P5M, 4000, 2, 1100, 150),
                                         (W.MONOEXP_4K, 2000, 1, 800, 80)]):
        mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
        th, sig, y = make_voxels(orc, w, 700 * i, n)
        jobs.append((mid, y, sig, gac.make_opts(I, B, 10, C, 300 + i, moments_mode=1)))
    srv = gac.gac_server_create(8 << 30, 64)
    try:
        ids = [gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, opts) for (mid, y, sig, opts) in jobs]
        for jid, (mid, y, sig, opts) in zip(ids, jobs):
            ref = gac.run_host(mid, y, sig, iterations=opts.iterations, burnin=opts.burnin, thin=opts.thin,
                               n_chains=opts.n_chains, seed=opts.seed, moments_mode=1, want_samples=False)
            out = {k: np.empty_like(ref[k]) for k in ("mean", "std", "accept_rate")}
            gac.gac_server_wait(srv, jid, 300.0, out)
            np.testing.assert_array_equal(out["accept_rate"], ref["accept_rate"])
            np.testing.assert_allclose(out["mean"], ref["mean"], rtol=1e-12, atol=0)
            np.testing.assert_allclose(out["std"], ref["std"], rtol=1e-9, atol=0)
    finally:
        gac.gac_server_destroy(srv)


def test_zero_iteration_job_completes(gac, orc):
    """A job with no iterations takes one empty round: its chains are
    initialised and its outputs written as gac_mcmc_run writes them."""
    w = W.SMT_1P5M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 300)
    srv = gac.gac_server_create(1 << 30, 8)
    try:
        opts = gac.make_opts(0, 0, 1, 2, 9)
        jid = gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, opts)
        ref = gac.run_host(mid, y, sig, iterations=0, burnin=0, thin=1, n_chains=2, seed=9, want_samples=False)
        out = {k: np.empty_like(ref[k]) for k in ("mean", "std", "accept_rate", "nonfinite")}
        gac.gac_server_wait(srv, jid, 60.0, out)
        for k in out:
            np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
    finally:
        gac.gac_server_destroy(srv)


def test_two_waiters_on_one_job(gac, orc):
    """Two host threads wait for the same job: one receives the results, the
    other UNKNOWN_JOB (the job was collected while it slept); neither hangs."""
    import threading

    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 4000)
    srv = gac.gac_server_create(8 << 30, 8)
    try:
        jid = gac.gac_server_submit(srv, mid, y, y.shape[0], sig, 0.0, gac.make_opts(3000, 300, 100, 4, 5))
        statuses = []

        def waiter():
            try:
                gac.gac_server_wait(srv, jid, 120.0, {})
                statuses.append(0)
            except gac.GacError as e:
                statuses.append(e.status)

        ts = [threading.Thread(target=waiter) for _ in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join(180.0)
        assert not any(t.is_alive() for t in ts)
        assert sorted(statuses) == [0, 9], statuses
    finally:
        gac.gac_server_destroy(srv)
