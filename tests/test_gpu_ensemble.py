"""Affine-invariant ensemble sampler on the device against the FP64 oracle
(Sec. 2.2.2, Table 1: 50 walkers x 2000 iterations, 10% burn-in, thinning
100).

Lock-step (every recorded walker move of traced voxels): the acceptance word
is the oracle's; the proposal is X_j + z (X_k - X_j) with the partner j and
stretch z the oracle derives from the same words, j's position taken from
the trace; states follow the recorded decisions exactly; decisions equal the
oracle's FP64 decisions in >= 99.9% of moves.  Free-running: the FP64 kernel
shadows the oracle (posterior means within 0.05 posterior SD for >= 99% of
voxel-parameters); the MIXED kernel matches it in distribution with
independent streams (the paper's Demo 2 design); determinism and voxel_base
split invariance; the exact linear-Gaussian posterior.
"""
import numpy as np
import pytest

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TABLE1 = dict(iterations=2000, burnin=200, thin=100, n_walkers=50)


def _ens(w):
    return w.with_(n_chains=50, iterations=2000, burnin=200, thin=100)


def _lockstep(gac, orc, w, tr, y, sig, seed, L, I, stretch, n_tr, prec):
    P = w.n_par
    H = L // 2
    lb, ub = np.array(w.lb), np.array(w.ub)
    agree = total = 0
    for v in range(n_tr):
        rec = tr[v]  # [L][I]
        th = rec["theta"][:, :, :P]
        pr = rec["prop"][:, :, :P]
        acc = rec["accepted"] != 0
        after = np.where(acc[..., None], pr, th)  # state after each walker's own move
        # continuity: a walker's next record starts from its state after its move
        np.testing.assert_array_equal(th[:, 1:], after[:, :-1])
        for k in range(L):
            h = 0 if k < H else 1
            t = np.arange(1, I + 1, dtype=np.uint32)
            wds = orc.words_many(seed, t, np.full(I, v, np.uint32), np.full(I, k, np.uint32), 3)
            np.testing.assert_array_equal(rec["w_acc"][k], wds[:, 2])
            j = (1 - h) * H + ((wds[:, 0].astype(np.uint64) * H) >> 32).astype(np.int64)
            z = np.array([orc.stretch_z(int(x), stretch) for x in wds[:, 1]])
            # partner position when k moves: half 0 sees j after t-1 (= j's record
            # theta at t), half 1 sees j after its move at t
            xj = (th if h == 0 else after)[j, np.arange(I)]
            want = xj + z[:, None] * (th[k] - xj)
            tol = 2e-6 * (np.abs(want) + np.abs(xj) + 1) if prec != gac.PREC_FP64 else 1e-12 * (1 + np.abs(want))
            assert (np.abs(pr[k] - want) <= tol).all(), (v, k, np.abs(pr[k] - want).max())
            inside = np.all((pr[k] >= lb) & (pr[k] <= ub), axis=1)
            L0, L1, _ = orc.lockstep(w.kind, w.acq, w.lb, w.ub, w.step, y[v], float(sig[v]), th[k],
                                     np.where(inside[:, None], pr[k], th[k]), rec["w_acc"][k])
            logu = np.log((rec["w_acc"][k].astype(np.float64) + 0.5) * 2.0 ** -32)
            dec = inside & (logu < (P - 1) * np.log(z) + L1 - L0)
            agree += int((dec == acc[k]).sum())
            total += I
    return agree / total


CASES = [(W.MONOEXP_4K, 512, 8, 0, 0.999), (W.MWI3_1M, 64, 2, 0, 0.999), (W.SMT_1P5M, 128, 4, 0, 0.999),
         (W.MWI3_1M, 32, 2, 2, 0.9999)]


@pytest.mark.parametrize("w,n,n_tr,prec,min_agree", CASES, ids=[f"{c[0].name}-p{c[3]}" for c in CASES])
def test_ensemble_lockstep(gac, orc, w, n, n_tr, prec, min_agree):
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, n)
    I, L, stretch, seed = 600, 50, 2.0, w.mcmc_seed + 7
    g = gac.run_ensemble_host(mid, y, sig, iterations=I, burnin=60, thin=30, n_walkers=L, seed=seed,
                              stretch=stretch, precision=prec, trace_n_vox=n_tr)
    frac = _lockstep(gac, orc, w, g["trace"], y, sig, seed, L, I, stretch, n_tr, prec)
    print(f"ensemble {w.name} prec={prec}: lock-step agreement {frac:.6f}")
    assert frac >= min_agree


ENS_PARITY = [(W.MONOEXP_4K, 1024), (W.MWI3_1M, 128), (W.SMT_1P5M, 256)]


@pytest.mark.parametrize("w,n", ENS_PARITY, ids=["monoexp", "mwi3", "smt"])
def test_ensemble_fp64_shadows_oracle(gac, orc, w, n):
    """Same seed, FP64 kernel: the walkers follow the oracle's (a decision
    flips only if FP64 rounding straddles log u), so posterior means agree to
    0.05 SD for >= 99% of voxel-parameters.  (In FP32 one near-tie flip in any
    of a voxel's ~10^5 moves reroutes all its walkers, since each walker's
    partner comes from the other half; the MIXED path is checked with
    independent streams below.)"""
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, n)
    kw = dict(TABLE1, seed=w.mcmc_seed + 11)
    g = gac.run_ensemble_host(mid, y, sig, stretch=2.0, precision=gac.PREC_FP64, **kw)
    r = orc.ensemble_run(w.kind, w.acq, w.lb, w.ub, y, sig, stretch=2.0, **kw)
    assert g["samples"].shape[0] * g["samples"].shape[1] == 900  # Table 1
    ok = r["std"] > 0
    gap = np.abs(g["mean"] - r["mean"])[ok] / r["std"][ok]
    print(f"ensemble FP64 {w.name}: |dmean|/SD median {np.median(gap):.2e} p99 {np.quantile(gap, 0.99):.2e}; "
          f"within 0.05 SD {(gap <= 0.05).mean():.4f}")
    assert (gap <= 0.05).mean() >= 0.99
    assert abs(g["accept_rate"].mean() - r["accept_rate"].mean()) < 0.005


@pytest.mark.parametrize("w,n", ENS_PARITY, ids=["monoexp", "mwi3", "smt"])
def test_ensemble_mixed_independent_seeds(gac, orc, w, n):
    """MIXED kernel against the oracle with independent random streams, the
    paper's Demo 2 design (GPU-minus-CPU against CPU-minus-CPU)."""
    from test_gpu_precision_study import paired_seed_check
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 4 * n)
    kw = dict(TABLE1, stretch=2.0, want_samples=False)
    runs = {s: orc.ensemble_run(w.kind, w.acq, w.lb, w.ub, y, sig, seed=s, **kw) for s in (11, 22, 44)}
    runs[33] = gac.run_ensemble_host(mid, y, sig, seed=33, **kw)
    paired_seed_check(runs, ((11, 22), (33, 44)), f"ensemble {w.name}")
    assert abs(runs[33]["accept_rate"].mean() - runs[44]["accept_rate"].mean()) < 0.01


def test_ensemble_determinism_and_split(gac, orc):
    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    n = 37  # ragged against 10 voxels per block
    th, sig, y = make_voxels(orc, w, 0, n)
    kw = dict(iterations=300, burnin=30, thin=30, n_walkers=20, seed=5, stretch=1.7)
    a = gac.run_ensemble_host(mid, y, sig, **kw)
    b = gac.run_ensemble_host(mid, y, sig, **kw)
    for k in ("mean", "std", "samples", "accept_rate"):
        np.testing.assert_array_equal(a[k], b[k])
    p2 = gac.run_ensemble_host(mid, y[13:], sig[13:], voxel_base=13, **kw)
    np.testing.assert_array_equal(p2["samples"], a["samples"][..., 13:])
    with pytest.raises(gac.GacError):
        gac.run_ensemble_host(mid, y, sig, iterations=10, burnin=0, thin=1, n_walkers=7, seed=1)
    with pytest.raises(gac.GacError):
        gac.run_ensemble_host(mid, y, sig, iterations=10, burnin=0, thin=1, n_walkers=8, seed=1, stretch=1.0)


def test_ensemble_linear_gaussian_posterior_on_device(gac, orc):
    t = np.linspace(0.0, 1.0, 12)
    X = np.stack([np.ones(12), t], 1)
    sig = 0.1
    y0 = (X @ np.array([0.5, -1.0]) + sig * np.random.default_rng(11).standard_normal(12)).astype(np.float32)
    XtX = X.T @ X
    mu = np.linalg.solve(XtX, X.T @ y0.astype(np.float64))
    cov = sig ** 2 * np.linalg.inv(XtX)
    sd = np.sqrt(np.diag(cov))
    mid = gac.gac_model_register(100, t, mu - 100 * sd, mu + 100 * sd, [0.0, 0.0])
    n, L = 1024, 32
    x0 = (mu + 0.5 * sd * np.random.default_rng(3).standard_normal((n, L, 2))).astype(np.float32)
    g = gac.run_ensemble_host(mid, np.tile(y0, (n, 1)), np.full(n, sig, np.float32), iterations=1500,
                              burnin=300, thin=50, n_walkers=L, seed=8, x0=x0)
    s = g["samples"].astype(np.float64)  # [S][L][P][N]
    vm = s.mean(axis=(0, 1))             # per-voxel means [P][N], independent voxels
    m = vm.mean(axis=1)
    se = vm.std(axis=1) / np.sqrt(n)
    assert np.all(np.abs(m - mu) < 5 * se), (m, mu, se)
    var = np.array([np.mean((s[:, :, p] - mu[p]) ** 2) for p in range(2)])
    assert np.allclose(var, np.diag(cov), rtol=0.04)


def test_ensemble_mixed_all_postburnin_moments_blocked(gac, orc):
    """MIXED ensemble moments over every post-burn-in state use the blocked
    FP32 accumulation; with thinning 1 the thinned mode's per-state FP64
    Welford sees the same walkers, so the two agree to FP32 rounding."""
    w = W.SMT_1P5M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 200)
    kw = dict(iterations=900, burnin=100, thin=1, n_walkers=20, seed=8)  # 12 full blocks + 32 states
    per_state = gac.run_ensemble_host(mid, y, sig, moments_mode=0, **kw)
    blocked = gac.run_ensemble_host(mid, y, sig, moments_mode=1, want_samples=False, **kw)
    np.testing.assert_array_equal(blocked["accept_rate"], per_state["accept_rate"])
    sd = per_state["std"]
    ok = sd > 0
    dm = np.abs(blocked["mean"] - per_state["mean"])[ok] / sd[ok]
    ds = np.abs(blocked["std"] - sd)[ok] / sd[ok]
    print(f"ensemble blocked vs per-state moments: |dmean|/SD max {dm.max():.2e}, |dSD|/SD max {ds.max():.2e}")
    assert dm.max() <= 1e-5 and ds.max() <= 1e-4
