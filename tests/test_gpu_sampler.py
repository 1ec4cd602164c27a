"""The MH sampler on the device against the FP64 oracle (mcmc.m, Sec. 2.2.2).

Lock-step checks (every recorded step of traced chains):
  - the acceptance word is the oracle's word, bit for bit;
  - the proposal is clamp(theta + step z) with the oracle's normals, to the
    FP32 error of Box-Muller;
  - each state follows from the previous record's decision, exactly;
  - the decision equals the oracle's FP64 decision recomputed from the
    recorded theta and theta' in >= 99.9% of steps (>= 99.99% for FP64);
  - the kernel's L' equals the oracle's within 1e-3 after burn-in.
Free-running checks (same seed): posterior means within 0.05 posterior SD;
bit-exact determinism, tiling and split invariance, host/device pointers.
"""
import numpy as np
import pytest
import torch

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _register(gac, w, acq=None):
    return gac.gac_model_register(w.kind, w.acq if acq is None else acq, w.lb, w.ub, w.step)


def _lockstep_check(gac, orc, w, tr, y, sig, seed, prec, n_tr, C, I, B, min_agree):
    P = w.n_par
    lb, ub, step = map(np.array, (w.lb, w.ub, w.step))
    nw = orc.n_words(P)
    agree = total = 0
    dL = []
    for v in range(n_tr):
        for c in range(C):
            rec = tr[v, c]
            th, pr = rec["theta"][:, :P], rec["prop"][:, :P]
            # words: bit-exact
            t = np.arange(1, I + 1, dtype=np.uint32)
            words = orc.words_many(seed, t, np.full(I, v, np.uint32), np.full(I, c, np.uint32), nw)
            np.testing.assert_array_equal(rec["w_acc"], words[:, nw - 1])
            # proposal from the oracle's normals
            z = orc.normals_many(words, P)
            want = np.clip(th + step * z, lb, ub)
            tol = 3e-3 * step + 3e-7 * np.abs(want) if prec != gac.PREC_FP64 else 1e-12 * (1 + np.abs(want))
            assert (np.abs(pr - want) <= tol).all(), (v, c, np.abs(pr - want).max())
            # chain continuity
            acc = rec["accepted"] != 0
            nxt = np.where(acc[:-1, None], pr[:-1], th[:-1])
            np.testing.assert_array_equal(th[1:], nxt)
            # decisions
            L, Lp, dec = orc.lockstep(w.kind, w.acq, w.lb, w.ub, w.step, y[v], float(sig[v]), th, pr,
                                      rec["w_acc"])
            agree += int((dec == acc).sum())
            total += I
            # L' at posterior-typical states (chi^2 <= 2M, i.e. |L'| <= M) in
            # absolute terms; elsewhere relative to |L'| (chains still far
            # from the fit, where FP32 errors grow with |L'|)
            typical = np.abs(Lp) <= w.n_meas
            dL.append(np.abs(rec["Lp"] - Lp)[typical])
            rel = np.abs(rec["Lp"] - Lp) / np.maximum(np.abs(Lp), 1.0)
            # FP64: 1e-12 (AxCaliberSMT: its series stops at 64 terms, the oracle's at 100)
            tol64 = 1e-9 if w.kind == W.AXCAL else 1e-12
            assert rel.max() <= (tol64 if prec == gac.PREC_FP64 else 1e-4), (v, c, rel.max())
    dL = np.concatenate(dL) if dL else np.zeros(1)
    frac = agree / total
    print(f"{w.name} prec={prec}: agreement {agree}/{total} = {frac:.6f}; posterior-typical "
          f"|dL'| ({dL.size} steps) max {dL.max():.2e} p99.9 {np.quantile(dL, 0.999):.2e}")
    assert frac >= min_agree
    return frac, dL


LOCKSTEP = [
    (W.MONOEXP_4K, 4096, 64, 0, 0.999),
    (W.MWI3_1M, 256, 8, 0, 0.999),
    (W.SMT_1P5M, 256, 8, 0, 0.999),
    (W.AXCAL_250K.with_(name="axcal_2k", iterations=2000, burnin=200, thin=20), 256, 8, 0, 0.999),
    (W.AXCAL_250K.with_(name="axcal_1k", iterations=1000, burnin=100, thin=20), 64, 4, 2, 0.9999),
    (W.MWI3_1M, 64, 4, 2, 0.9999),
    (W.MONOEXP_4K, 256, 32, 2, 0.9999),
    (W.MWI3_1M.with_(name="mwi3_fp32"), 64, 4, 1, 0.99),
]


@pytest.mark.parametrize("w,n,n_tr,prec,min_agree", LOCKSTEP,
                         ids=[f"{c[0].name}-p{c[3]}" for c in LOCKSTEP])
def test_lockstep(gac, orc, w, n, n_tr, prec, min_agree):
    mid = _register(gac, w)
    th, sig, y = make_voxels(orc, w, 0, n)
    C, I, B, T = w.n_chains, w.iterations, w.burnin, w.thin
    out = gac.run_host(mid, y, sig, iterations=I, burnin=B, thin=T, n_chains=C, seed=w.mcmc_seed,
                       precision=prec, trace_n_vox=n_tr)
    tr = out["trace"]
    frac, dL = _lockstep_check(gac, orc, w, tr, y, sig, w.mcmc_seed, prec, n_tr, C, I, B, min_agree)
    tol_L = 1e-3 if prec == gac.PREC_MIXED else (2e-3 if prec == gac.PREC_FP32 else 1e-8)
    assert np.quantile(dL, 0.999) <= tol_L
    # the initial state is the uniform-prior draw of counter iteration 0xFFFFFFFF
    lb, ub = np.array(w.lb), np.array(w.ub)
    for v in range(min(n_tr, 4)):
        wi = orc.words(w.mcmc_seed, 0xFFFFFFFF, v, 0, w.n_par)
        init = lb + (ub - lb) * np.array([orc.u01(x) for x in wi])
        assert np.allclose(tr[v, 0, 0]["theta"][:w.n_par], init, rtol=2e-7, atol=1e-6 * (ub - lb).max())


def _posterior_gap(gpu, ref):
    sd = ref["std"]
    ok = sd > 0
    return np.abs(gpu["mean"] - ref["mean"])[ok] / sd[ok]


FREE = [(W.MONOEXP_4K, 4096), (W.MWI3_1M, 512), (W.SMT_1P5M, 512),
        (W.AXCAL_250K.with_(name="axcal_3k", iterations=3000, burnin=300, thin=30), 512)]


@pytest.mark.parametrize("w,n", FREE, ids=[c[0].name for c in FREE])
def test_free_running_posterior_parity(gac, orc, w, n):
    mid = _register(gac, w)
    th, sig, y = make_voxels(orc, w, 0, n)
    kw = dict(iterations=w.iterations, burnin=w.burnin, thin=w.thin, n_chains=w.n_chains,
              seed=w.mcmc_seed)
    g = gac.run_host(mid, y, sig, **kw)
    r = orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, **kw)
    gap = _posterior_gap(g, r)
    same = np.all(g["samples"] == r["samples"].astype(np.float32), axis=(0, 1))  # [P][N]
    print(f"{w.name}: |dmean|/SD median {np.median(gap):.2e} p99 {np.quantile(gap, 0.99):.2e} "
          f"max {gap.max():.2e}; within 0.05 SD: {(gap <= 0.05).mean():.4f}; "
          f"accept rate gpu {g['accept_rate'].mean():.4f} oracle {r['accept_rate'].mean():.4f}")
    assert (gap <= 0.05).mean() >= 0.99
    assert abs(g["accept_rate"].mean() - r["accept_rate"].mean()) < 0.01
    assert np.all(g["nonfinite"] == 0)


def test_moments_match_stored_samples(gac, orc):
    w = W.MWI3_1M
    mid = _register(gac, w)
    th, sig, y = make_voxels(orc, w, 0, 300)
    # MIXED: FP64 Welford over the FP32 states that are also stored -> FP64
    # agreement.  FP64: states are doubles, samples are stored rounded to
    # float (2^-24 relative).  FP32: Welford in float.
    for prec, rtol in ((gac.PREC_MIXED, 1e-10), (gac.PREC_FP64, 2 ** -23), (gac.PREC_FP32, 1e-5)):
        g = gac.run_host(mid, y, sig, iterations=1200, burnin=200, thin=10, n_chains=4, seed=3,
                         precision=prec)
        s = g["samples"].astype(np.float64)  # [S][C][P][N]
        pooled = s.transpose(2, 3, 0, 1).reshape(w.n_par, 300, -1)
        scale = np.abs(pooled).max(-1)
        assert (np.abs(g["mean"] - pooled.mean(-1)) <= rtol * scale + 1e-300).all(), prec
        sd = pooled.std(-1, ddof=1)
        assert (np.abs(g["std"] - sd) <= 10 * rtol * scale + 1e-3 * sd * (prec == gac.PREC_FP32)).all(), prec


def test_all_postburnin_moments(gac, orc):
    w = W.MONOEXP_4K
    mid = _register(gac, w)
    th, sig, y = make_voxels(orc, w, 0, 256)
    kw = dict(iterations=800, burnin=200, thin=50, n_chains=2, seed=4, moments_mode=1)
    g = gac.run_host(mid, y, sig, precision=gac.PREC_FP64, **kw)
    r = orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, **kw)
    gap = _posterior_gap(g, r)
    assert (gap <= 1e-6).mean() >= 0.99


def test_determinism_tiling_split_and_pointer_kinds(gac, orc):
    w = W.MWI3_1M.with_(n_chains=3)
    mid = _register(gac, w)
    n = 777  # ragged against 85 voxels per block
    th, sig, y = make_voxels(orc, w, 0, n)
    kw = dict(iterations=300, burnin=100, thin=20, n_chains=3, seed=99)
    a = gac.run_host(mid, y, sig, **kw)
    b = gac.run_host(mid, y, sig, **kw)
    for k in ("mean", "std", "samples", "accept_rate", "nonfinite"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    # split with voxel_base reproduces the whole run
    k0 = 301
    p1 = gac.run_host(mid, y[:k0], sig[:k0], **kw)
    p2 = gac.run_host(mid, y[k0:], sig[k0:], voxel_base=k0, **kw)
    np.testing.assert_array_equal(np.concatenate([p1["mean"], p2["mean"]], 1), a["mean"])
    np.testing.assert_array_equal(np.concatenate([p1["samples"], p2["samples"]], 3), a["samples"])
    # a single voxel
    one = gac.run_host(mid, y[5:6], sig[5:6], voxel_base=5, **kw)
    np.testing.assert_array_equal(one["mean"][:, 0], a["mean"][:, 5])
    # device buffers (and an unaligned data pointer) give the same bits
    dev = torch.device("cuda:0")
    P, S, C = w.n_par, gac.n_samples(300, 100, 20), 3
    yd = torch.zeros(n * w.n_meas + 1, dtype=torch.float32, device=dev)
    yd[1:] = torch.from_numpy(y.ravel()).to(dev)
    out = dict(mean=torch.empty((P, n), dtype=torch.float64, device=dev),
               samples=torch.empty((S, C, P, n), dtype=torch.float32, device=dev))
    opts = gac.make_opts(300, 100, 20, 3, 99)
    gac.gac_mcmc_run(mid, yd.data_ptr() + 4, n, torch.from_numpy(sig).to(dev), 0.0, None, opts, out,
                     torch.cuda.current_stream())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["mean"].cpu().numpy(), a["mean"])
    np.testing.assert_array_equal(out["samples"].cpu().numpy(), a["samples"])
    # page-locked host buffers (read and written in place by the kernel) too
    hy = torch.from_numpy(y).pin_memory()
    hs = torch.from_numpy(sig).pin_memory()
    hout = dict(mean=torch.empty((P, n), dtype=torch.float64).pin_memory(),
                std=torch.empty((P, n), dtype=torch.float64).pin_memory(),
                samples=torch.empty((S, C, P, n), dtype=torch.float32).pin_memory(),
                accept_rate=torch.empty((C, n), dtype=torch.float32).pin_memory())
    gac.gac_mcmc_run(mid, hy, n, hs, 0.0, None, opts, hout, torch.cuda.current_stream())
    for k, v in hout.items():
        np.testing.assert_array_equal(v.numpy(), a[k], err_msg=f"pinned {k}")


def test_degenerate_options(gac, orc):
    w = W.MONOEXP_4K
    mid = _register(gac, w)
    th, sig, y = make_voxels(orc, w, 0, 40)
    g = gac.run_host(mid, y, sig, iterations=100, burnin=100, thin=5, n_chains=2, seed=1)
    assert np.isnan(g["mean"]).all() and np.isnan(g["std"]).all()
    g = gac.run_host(mid, y, sig, iterations=105, burnin=100, thin=5, n_chains=1, seed=1)
    assert (g["std"] == 0).all()
    np.testing.assert_array_equal(g["mean"], g["samples"][0, 0].astype(np.float64))
    g = gac.run_host(mid, y, sig, iterations=0, burnin=0, thin=1, n_chains=1, seed=1)
    assert (g["accept_rate"] == 0).all() and np.isnan(g["mean"]).all()
    # a parameter fixed by lb = ub
    fixed = gac.gac_model_register(w.kind, w.acq, [1.0, 10.0], [1.0, 80.0], [0.3, 1.0])
    g = gac.run_host(fixed, y, sig, iterations=200, burnin=0, thin=1, n_chains=1, seed=1)
    assert (g["samples"][:, :, 0, :] == 1.0).all() and (g["std"][0] == 0).all()
    # scalar sigma equals a constant per-voxel sigma
    a = gac.run_host(mid, y, None, sigma_scalar=0.01, iterations=200, burnin=50, thin=5, n_chains=1, seed=2)
    b = gac.run_host(mid, y, np.full(40, 0.01, np.float32), iterations=200, burnin=50, thin=5,
                     n_chains=1, seed=2)
    np.testing.assert_array_equal(a["mean"], b["mean"])
    # x0 given: the chain starts there (clamped into the bounds)
    x0 = np.tile(np.array([[2.0, 30.0]], np.float32), (40, 1, 1))
    g = gac.run_host(mid, y, sig, iterations=10, burnin=0, thin=1, n_chains=1, seed=2, x0=x0,
                     trace_n_vox=3)
    assert np.allclose(g["trace"][0, 0, 0]["theta"][:2], [1.5, 30.0])


def test_linear_gaussian_posterior_on_device(gac, orc):
    """The GPU sampler's stationary distribution is the exact posterior of
    the linear-Gaussian test model (checked across many identical voxels)."""
    t = np.linspace(0.0, 1.0, 12)
    X = np.stack([np.ones(12), t], 1)
    sig = 0.1
    y0 = (X @ np.array([0.5, -1.0]) + sig * np.random.default_rng(11).standard_normal(12)).astype(np.float32)
    XtX = X.T @ X
    mu = np.linalg.solve(XtX, X.T @ y0.astype(np.float64))
    cov = sig ** 2 * np.linalg.inv(XtX)
    sd = np.sqrt(np.diag(cov))
    mid = gac.gac_model_register(100, t, mu - 100 * sd, mu + 100 * sd, 1.2 * sd)
    n = 4096
    y = np.tile(y0, (n, 1))
    x0 = np.tile(mu.astype(np.float32), (n, 1, 1))
    g = gac.run_host(mid, y, np.full(n, sig, np.float32), iterations=3000, burnin=500, thin=25,
                     n_chains=1, seed=5, x0=x0)
    s = g["samples"][:, 0].astype(np.float64)  # [S][P][N], voxels independent
    m = s.mean(axis=(0, 2))
    # voxel means are independent; their spread gives the MC error
    se = s.mean(axis=0).std(axis=1) / np.sqrt(n)
    assert np.all(np.abs(m - mu) < 5 * se), (m, mu, se)
    var = np.array([np.mean((s[:, p] - mu[p]) ** 2) for p in range(2)])
    assert np.allclose(var, np.diag(cov), rtol=0.03)


def test_small_and_full_tiles_give_the_same_bits(gac, orc):
    """A volume too small to fill every resident block runs in tiles of one
    warp of chains; a large one in full blocks.  The random numbers depend
    only on (seed, t, voxel, chain), so the first voxels of a large run equal
    the same voxels run alone, bit for bit."""
    w = W.MWI3_1M
    mid = _register(gac, w)
    n_big, n_small = 60_000, 700  # 240,000 chains fill full blocks; 2,800 do not
    th, sig, y = make_voxels(orc, w, 0, n_big)
    kw = dict(iterations=300, burnin=100, thin=20, n_chains=4, seed=5)
    big = gac.run_host(mid, y, sig, **kw)
    small = gac.run_host(mid, y[:n_small], sig[:n_small], **kw)
    tail = gac.run_host(mid, y[-n_small:], sig[-n_small:], voxel_base=n_big - n_small, **kw)
    for k in ("samples", "accept_rate", "mean", "std"):
        np.testing.assert_array_equal(small[k], big[k][..., :n_small], err_msg=k)
        np.testing.assert_array_equal(tail[k], big[k][..., -n_small:], err_msg=k)


def test_mixed_all_postburnin_moments_blocked(gac, orc):
    """MIXED moments over every post-burn-in state come from FP32 sums over
    blocks of 64 states merged into the FP64 Welford state; with thinning 1 the
    thinned mode's per-state FP64 Welford sees the same states of the same
    chains, so the two must agree to the FP32 rounding of the block sums."""
    w = W.MWI3_1M
    mid = _register(gac, w)
    th, sig, y = make_voxels(orc, w, 0, 500)
    kw = dict(iterations=1300, burnin=300, thin=1, n_chains=4, seed=17)  # 15 full blocks + 40 states
    per_state = gac.run_host(mid, y, sig, moments_mode=0, **kw)
    blocked = gac.run_host(mid, y, sig, moments_mode=1, want_samples=False, **kw)
    np.testing.assert_array_equal(blocked["accept_rate"], per_state["accept_rate"])
    sd = per_state["std"]
    ok = sd > 0
    dm = np.abs(blocked["mean"] - per_state["mean"])[ok] / sd[ok]
    ds = np.abs(blocked["std"] - sd)[ok] / sd[ok]
    print(f"blocked vs per-state moments: |dmean|/SD max {dm.max():.2e}, |dSD|/SD max {ds.max():.2e}")
    assert dm.max() <= 1e-5 and ds.max() <= 1e-4
    assert np.all(blocked["std"][~ok] <= 1e-6)


LANE_CASES = [
    # (workload, echoes kept, voxels, chains, lane counts compared with one lane)
    ("monoexp", 12, 1000, 1, (2, 4)),
    ("monoexp", 12, 333, 3, (2, 4)),
    ("mwi3", 24, 301, 4, (4,)),
    ("mwi3", 12, 257, 2, (2, 4)),
    ("mwi3", 22, 150, 4, (4,)),  # a partial last block
]


@pytest.mark.parametrize("case", LANE_CASES, ids=[f"{c[0]}_{c[1]}echo_{c[2]}x{c[3]}" for c in LANE_CASES])
def test_lane_split_gives_the_same_bits(gac, orc, case):
    """Lanes per chain (each lane one block of six echoes, the block sums
    combined by warp shuffles in the one-thread kernel's Kahan order, random
    numbers drawn a round ahead by rotating lanes) give the one-thread
    kernel's results bit for bit: samples, moments, R-hat, acceptance rates
    and step multipliers, with thinned moments and with moments over every
    post-burn-in state, burn-in adaptation, a start x0, ragged tiles and
    several chains per voxel."""
    name, n_echo, n, C, lanes = case
    base = W.MONOEXP_4K if name == "monoexp" else W.MWI3_1M
    w = base.with_(acq=base.acq[:n_echo])
    mid = _register(gac, w)
    th, sig, y = make_voxels(orc, w, 0, n)
    x0 = np.repeat(th[:, None, :], C, axis=1).astype(np.float32)
    keys = ("samples", "mean", "std", "rhat", "accept_rate", "nonfinite", "step_scale")
    runs = [dict(iterations=600, burnin=200, thin=5, n_chains=C, seed=21),
            dict(iterations=700, burnin=300, thin=7, n_chains=C, seed=22, adapt_window=50, adapt_target=0.3,
                 moments_mode=gac.MOMENTS_ALL_POSTBURNIN, x0=x0)]
    for kw in runs:
        one = gac.run_host(mid, y, sig, lanes_per_chain=1, **kw)
        for g in lanes:
            split = gac.run_host(mid, y, sig, lanes_per_chain=g, **kw)
            for k in keys:
                np.testing.assert_array_equal(split[k], one[k], err_msg=f"{k} with {g} lanes")
        assert np.isfinite(one["mean"]).all()
