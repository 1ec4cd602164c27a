"""Burn-in step adaptation and R-hat on the device against the FP64 oracle.

Lock-step (every recorded step of traced chains, steps started 8x too wide):
the multiplier 2^(e/4) each proposal used, with e re-derived from the
recorded decisions by the documented window rule; the proposal
clamp(theta + step 2^(e/4) z) with the oracle's normals; the decisions against
the oracle's FP64 decisions; the reported final multiplier.  Free-running:
the FP64 kernel reproduces the oracle's final multipliers, moments and R-hat;
the MIXED kernel's R-hat is that of its own returned samples (the definition
applied to them) and agrees with the oracle's.
"""
import numpy as np
import pytest

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EMIN, EMAX = -48, 16


def _exponents(acc, W_a, B, target):
    """e in force at each iteration t = 1..I, and the final e."""
    e, a0, n = 0, 0, 0
    used = np.empty(len(acc), np.int64)
    for t in range(1, len(acc) + 1):
        used[t - 1] = e
        n += int(acc[t - 1])
        if W_a > 0 and t <= B and t % W_a == 0:
            a = n - a0
            if a > target * W_a and e < EMAX:
                e += 1
            if a < target * W_a and e > EMIN:
                e -= 1
            a0 = n
    return used, e


CASES = [(W.MONOEXP_4K, 512, 16, 0), (W.MWI3_1M, 64, 4, 0), (W.SMT_1P5M, 128, 8, 0),
         (W.MWI3_1M, 32, 2, 2)]


@pytest.mark.parametrize("w,n,n_tr,prec", CASES, ids=[f"{c[0].name}-p{c[3]}" for c in CASES])
def test_adaptive_lockstep(gac, orc, w, n, n_tr, prec):
    step = 8.0 * np.array(w.step)
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, step)
    th, sig, y = make_voxels(orc, w, 0, n)
    C, I, B, T, Wa, tgt, seed = w.n_chains, 700, 400, 50, 25, 0.25, w.mcmc_seed + 3
    g = gac.run_host(mid, y, sig, iterations=I, burnin=B, thin=T, n_chains=C, seed=seed, precision=prec,
                     trace_n_vox=n_tr, adapt_window=Wa, adapt_target=tgt)
    P, nw = w.n_par, orc.n_words(w.n_par)
    lb, ub = np.array(w.lb), np.array(w.ub)
    agree = total = 0
    e_final = []
    for v in range(n_tr):
        for c in range(C):
            rec = g["trace"][v, c]
            acc = rec["accepted"] != 0
            used, e_end = _exponents(acc, Wa, B, tgt)
            e_final.append(e_end)
            assert g["step_scale"][c, v] == pytest.approx(2.0 ** (e_end / 4.0), rel=3e-7)
            t = np.arange(1, I + 1, dtype=np.uint32)
            words = orc.words_many(seed, t, np.full(I, v, np.uint32), np.full(I, c, np.uint32), nw)
            z = orc.normals_many(words, P)
            lam = 2.0 ** (used / 4.0)
            th_r, pr = rec["theta"][:, :P], rec["prop"][:, :P]
            want = np.clip(th_r + step * lam[:, None] * z, lb, ub)
            tol = (3e-3 * step * lam[:, None] + 3e-7 * np.abs(want)) if prec != gac.PREC_FP64 \
                else 1e-12 * (1 + np.abs(want))
            assert (np.abs(pr - want) <= tol).all(), (v, c, np.abs(pr - want).max())
            L, Lp, dec = orc.lockstep(w.kind, w.acq, w.lb, w.ub, step, y[v], float(sig[v]), th_r, pr,
                                      rec["w_acc"])
            agree += int((dec == acc).sum())
            total += I
    frac = agree / total
    e_final = np.array(e_final)
    print(f"{w.name} prec={prec}: agreement {frac:.6f}; final e min {e_final.min()} median "
          f"{np.median(e_final)} max {e_final.max()}")
    assert frac >= (0.9999 if prec == gac.PREC_FP64 else 0.999)
    assert e_final.min() < -2  # the 8x steps were narrowed
    # every chain's reported multiplier is a power 2^(e/4) within the range
    e_all = np.round(4 * np.log2(g["step_scale"].astype(np.float64)))
    assert np.allclose(g["step_scale"], 2.0 ** (e_all / 4.0), rtol=3e-7)
    assert (e_all >= EMIN).all() and (e_all <= EMAX).all()


def test_adaptive_fp64_reproduces_oracle(gac, orc):
    w = W.MONOEXP_4K
    step = 8.0 * np.array(w.step)
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, step)
    th, sig, y = make_voxels(orc, w, 0, 256)
    kw = dict(iterations=2000, burnin=1000, thin=10, n_chains=4, seed=91, adapt_window=50, adapt_target=0.3)
    g = gac.run_host(mid, y, sig, precision=gac.PREC_FP64, **kw)
    r = orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, step, y, sig, **kw)
    e_g = np.round(4 * np.log2(g["step_scale"].astype(np.float64)))
    e_r = np.round(4 * np.log2(r["step_scale"]))
    same = (e_g == e_r).mean()
    gap = np.abs(g["mean"] - r["mean"]) / r["std"]
    dr = np.abs(g["rhat"] - r["rhat"]) / r["rhat"]
    print(f"FP64 adaptive: same final e {same:.4f}; |dmean|/SD max {gap.max():.2e}; "
          f"|dR-hat|/R-hat median {np.median(dr):.2e} max {dr.max():.2e}")
    assert same >= 0.999
    assert (e_r != 0).mean() > 0.5
    assert np.quantile(gap, 0.99) <= 1e-9
    assert np.quantile(dr, 0.99) <= 1e-9


def test_rhat_of_returned_samples_and_oracle(gac, orc):
    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 256)
    kw = dict(iterations=3000, burnin=500, thin=25, n_chains=4, seed=w.mcmc_seed)
    g = gac.run_host(mid, y, sig, **kw)
    # the definition applied to the kernel's own thinned samples
    s = g["samples"].astype(np.float64)  # [S][C][P][N]
    n = s.shape[0]
    cm = s.mean(axis=0)                                  # [C][P][N]
    Wv = s.var(axis=0, ddof=1).mean(axis=0)              # [P][N]
    Bn = cm.var(axis=0, ddof=1)                          # [P][N]
    want = np.sqrt(((n - 1) / n * Wv + Bn) / Wv)
    np.testing.assert_allclose(g["rhat"], want, rtol=1e-9)
    r = orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, **kw)
    d = np.abs(g["rhat"] - r["rhat"])
    print(f"R-hat MIXED vs oracle: median |d| {np.median(d):.2e}, p99 {np.quantile(d, 0.99):.2e}; "
          f"median R-hat {np.median(r['rhat']):.3f}")
    assert np.median(d) < 1e-4
    assert (d < 0.05).mean() >= 0.98
    one = gac.run_host(mid, y[:8], sig[:8], iterations=300, burnin=50, thin=10, n_chains=1, seed=1)
    assert np.isnan(one["rhat"]).all()
