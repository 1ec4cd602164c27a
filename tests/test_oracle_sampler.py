"""Pins of the oracle's Metropolis-Hastings sampler (mcmc.m, Sec. 2.2.2).

- Table 1's sample-count arithmetic (golden fixture);
- the thinning grid t in {B+T, B+2T, ...}, the initial state and every
  transition of a chain against the documented construction;
- moments = mean / SD (n-1) of the pooled thinned samples;
- stationary distribution: an exact linear-Gaussian posterior, and brute-force
  grid posteriors of 1- and 2-parameter mono-exponential voxels (Eq. 3), each
  within 4 Monte-Carlo standard errors (batch means).
"""
import os

import numpy as np
import pytest

MONOEXP, MWI3, SMT, LINEAR = 1, 2, 3, 100
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TE12 = np.array([2.0 + 3 * k for k in range(12)])


def test_table1_sample_counts(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_sample_counts.txt"))
            if l.strip() and not l.startswith("#")]
    assert rows
    for chains, iters, ratio, thin, total in rows:
        iters, thin = int(iters), int(thin)
        burnin = int(np.floor(float(ratio) * iters))  # burn-in given as a ratio of iterations
        assert int(chains) * orc.n_samples(iters, burnin, thin) == int(total)


def test_sample_count_edges(orc):
    assert orc.n_samples(2000, 500, 5) == 300
    assert orc.n_samples(500, 500, 5) == 0
    assert orc.n_samples(100, 500, 5) == 0
    assert orc.n_samples(504, 500, 5) == 0
    assert orc.n_samples(505, 500, 5) == 1


def _voxel(orc, kind, acq, theta, sigma, seed=3):
    s = orc.forward(kind, acq, np.asarray(theta, float))
    rng = np.random.default_rng(seed)
    return (s + sigma * rng.standard_normal(s.shape)).astype(np.float32)


MONO = dict(kind=MONOEXP, acq=TE12, lb=[0.5, 10.0], ub=[1.5, 80.0], step=[0.01, 1.0])


def test_chain_init_and_every_transition(orc):
    y = _voxel(orc, MONOEXP, TE12, [1.0, 35.0], 0.01)
    seed, v, c, I = 0xABCDEF0123, 17, 2, 400
    path, acc = orc.chain_path(**MONO, y=y, sigma=0.01, iterations=I, seed=seed, voxel=v, chain=c)
    lb, ub, step = map(np.array, (MONO["lb"], MONO["ub"], MONO["step"]))
    # initial state: uniform prior draw from counter iteration 0xFFFFFFFF
    w0 = orc.words(seed, 0xFFFFFFFF, v, c, 2)
    np.testing.assert_array_equal(path[0], lb + (ub - lb) * np.array([orc.u01(x) for x in w0]))
    n_acc = 0
    for t in range(1, I + 1):
        w = orc.words(seed, t, v, c, orc.n_words(2))
        z = orc.normals_from_words(w, 2)
        prop = np.minimum(np.maximum(path[t - 1] + step * z, lb), ub)
        L, Lp = orc.loglik(MONOEXP, TE12, np.stack([path[t - 1], prop]), np.stack([y, y]), [0.01, 0.01])
        accept = np.log(orc.u01(int(w[-1]))) < Lp - L
        n_acc += accept
        np.testing.assert_array_equal(path[t], prop if accept else path[t - 1])
    assert acc == n_acc / I
    assert 0 < n_acc < I


def test_thinning_grid_and_moments(orc):
    th = np.array([[1.2, 30.0], [0.7, 60.0], [1.0, 15.0]])
    sig = np.array([0.012, 0.007, 0.01], np.float32)
    y = np.concatenate([_voxel(orc, MONOEXP, TE12, th[i:i + 1], sig[i], seed=i) for i in range(3)])
    I, B, T, C, seed = 700, 200, 7, 3, 99
    r = orc.mcmc_run(**MONO, data=y, sigma=sig, iterations=I, burnin=B, thin=T, n_chains=C,
                     seed=seed)
    S = orc.n_samples(I, B, T)
    assert r["samples"].shape == (S, C, 2, 3) and S == 71
    for v in range(3):
        for c in range(C):
            path, acc = orc.chain_path(**MONO, y=y[v], sigma=float(sig[v]), iterations=I,
                                       seed=seed, voxel=v, chain=c)
            grid = B + T * np.arange(1, S + 1)          # t = B+T, B+2T, ... <= I
            np.testing.assert_array_equal(r["samples"][:, c, :, v], path[grid])
            assert r["accept_rate"][c, v] == acc
        pooled = r["samples"][:, :, :, v].transpose(2, 0, 1).reshape(2, -1)
        np.testing.assert_allclose(r["mean"][:, v], pooled.mean(1), rtol=1e-13)
        np.testing.assert_allclose(r["std"][:, v], pooled.std(1, ddof=1), rtol=1e-11)
    assert np.all(r["nonfinite"] == 0)


def test_all_postburnin_moments_mode(orc):
    y = _voxel(orc, MONOEXP, TE12, [1.1, 50.0], 0.01)[None]
    I, B, T, C = 600, 150, 50, 2
    r = orc.mcmc_run(**MONO, data=y, sigma=np.float32([0.01]), iterations=I, burnin=B, thin=T,
                     n_chains=C, seed=5, moments_mode=1)
    pooled = np.concatenate([orc.chain_path(**MONO, y=y[0], sigma=0.01, iterations=I, seed=5,
                                            chain=c)[0][B + 1:] for c in range(C)])
    np.testing.assert_allclose(r["mean"][:, 0], pooled.mean(0), rtol=1e-13)
    np.testing.assert_allclose(r["std"][:, 0], pooled.std(0, ddof=1), rtol=1e-11)


def test_degenerate_runs(orc):
    y = _voxel(orc, MONOEXP, TE12, [1.0, 30.0], 0.01)[None]
    r = orc.mcmc_run(**MONO, data=y, sigma=np.float32([0.01]), iterations=50, burnin=50, thin=5,
                     n_chains=2, seed=1)
    assert r["samples"].shape[0] == 0 and np.all(np.isnan(r["mean"])) and np.all(np.isnan(r["std"]))
    r = orc.mcmc_run(**MONO, data=y, sigma=np.float32([0.01]), iterations=55, burnin=50, thin=5,
                     n_chains=1, seed=1)
    assert r["samples"].shape[0] == 1 and np.all(r["std"] == 0.0)
    np.testing.assert_array_equal(r["mean"][:, 0], r["samples"][0, 0, :, 0])
    # zero voxels
    r = orc.mcmc_run(**MONO, data=np.zeros((0, 12), np.float32), sigma=np.zeros(0, np.float32),
                     iterations=10, burnin=0, thin=1, n_chains=1, seed=1)
    assert r["mean"].shape == (2, 0)
    # a parameter fixed by lb = ub stays fixed
    r = orc.mcmc_run(kind=MONOEXP, acq=TE12, lb=[1.0, 10.0], ub=[1.0, 80.0], step=[0.5, 1.0],
                     data=y, sigma=np.float32([0.01]), iterations=300, burnin=0, thin=1,
                     n_chains=1, seed=2)
    assert np.all(r["samples"][:, :, 0, :] == 1.0)
    # invalid arguments are rejected
    with pytest.raises(ValueError):
        orc.mcmc_run(**MONO, data=y, sigma=None, iterations=10, burnin=0, thin=0, n_chains=1, seed=1)


def test_voxel_base_offsets_the_counter(orc):
    th = np.array([[1.2, 30.0], [0.7, 60.0], [1.0, 15.0], [0.9, 45.0]])
    y = np.concatenate([_voxel(orc, MONOEXP, TE12, th[i:i + 1], 0.01, seed=i) for i in range(4)])
    kw = dict(**MONO, sigma=None, sigma_scalar=0.01, iterations=300, burnin=100, thin=10,
              n_chains=2, seed=7)
    full = orc.mcmc_run(data=y, **kw)
    part = orc.mcmc_run(data=y[2:], voxel_base=2, **kw)
    np.testing.assert_array_equal(full["samples"][..., 2:], part["samples"])
    np.testing.assert_array_equal(full["mean"][:, 2:], part["mean"])


def test_openmp_thread_count_does_not_change_results(orc):
    th = np.array([[1.2, 30.0], [0.7, 60.0], [1.0, 15.0], [0.9, 45.0]] * 4)
    y = np.concatenate([_voxel(orc, MONOEXP, TE12, th[i:i + 1], 0.01, seed=i) for i in range(16)])
    kw = dict(**MONO, data=y, sigma=None, sigma_scalar=0.01, iterations=200, burnin=50, thin=5,
              n_chains=2, seed=8)
    a = orc.mcmc_run(n_threads=1, **kw)
    b = orc.mcmc_run(n_threads=4, **kw)
    assert a["threads"] == 1 and b["threads"] == 4
    for k in ("mean", "std", "samples", "accept_rate"):
        np.testing.assert_array_equal(a[k], b[k])


# ------------------------------------------------ stationary distributions
def _batch_mcse(x, n_batches=50):
    """x: [chains][n] -> Monte-Carlo SE of the pooled mean by batch means."""
    C, n = x.shape
    m = n // n_batches
    bm = x[:, :m * n_batches].reshape(C, n_batches, m).mean(2).ravel()
    return bm.std(ddof=1) / np.sqrt(bm.size)


def _check_moments(samples, mean_ref, cov_ref, k=4.0):
    """samples [S][C][P]: pooled mean and (co)variance within k MCSE."""
    S, C, P = samples.shape
    x = samples.transpose(1, 0, 2)  # [C][S][P]
    mu = x.reshape(-1, P).mean(0)
    for p in range(P):
        se = _batch_mcse(x[:, :, p])
        assert abs(mu[p] - mean_ref[p]) < k * se, (p, mu[p], mean_ref[p], se)
        for q in range(p, P):
            prod = (x[:, :, p] - mean_ref[p]) * (x[:, :, q] - mean_ref[q])
            se2 = _batch_mcse(prod)
            assert abs(prod.mean() - cov_ref[p, q]) < k * se2 + 1e-12, (p, q, prod.mean(), cov_ref[p, q], se2)


def test_linear_gaussian_posterior(orc):
    """s = a + c t with Gaussian noise and a flat prior: the posterior is
    N((X'X)^-1 X'y, sigma^2 (X'X)^-1) exactly (bounds 100 SD away)."""
    t = np.linspace(0.0, 1.0, 12)
    X = np.stack([np.ones(12), t], 1)
    sig = 0.1
    y = (X @ np.array([0.5, -1.0]) + sig * np.random.default_rng(11).standard_normal(12)).astype(np.float32)
    XtX = X.T @ X
    mu = np.linalg.solve(XtX, X.T @ y.astype(np.float64))
    cov = sig ** 2 * np.linalg.inv(XtX)
    sd = np.sqrt(np.diag(cov))
    r = orc.mcmc_run(kind=LINEAR, acq=t, lb=mu - 100 * sd, ub=mu + 100 * sd, step=1.2 * sd,
                     data=y[None], sigma=np.float32([sig]), iterations=250_000, burnin=2_000,
                     thin=1, n_chains=4, seed=2024, x0=np.tile(mu, (1, 4, 1)).astype(np.float32))
    _check_moments(r["samples"][:, :, :, 0], mu, cov)
    assert 0.15 < r["accept_rate"].mean() < 0.7


def _grid_posterior(y, sigma, s0_axis, r2_axis):
    S0, R2 = np.meshgrid(s0_axis, r2_axis, indexing="ij")
    s = S0[..., None] * np.exp(-R2[..., None] * TE12 * 1e-3)
    L = -0.5 * (((y.astype(np.float64) - s) / sigma) ** 2).sum(-1)
    w = np.exp(L - L.max())
    w /= w.sum()
    mean = np.array([(w * S0).sum(), (w * R2).sum()])
    d = [S0 - mean[0], R2 - mean[1]]
    cov = np.array([[(w * d[i] * d[j]).sum() for j in range(2)] for i in range(2)])
    return mean, cov


def test_grid_posterior_two_parameters(orc):
    sig = 0.01
    y = _voxel(orc, MONOEXP, TE12, [1.0, 40.0], sig, seed=12)
    mean0, cov0 = _grid_posterior(y, sig, np.linspace(0.9, 1.1, 400), np.linspace(30, 50, 400))
    sd = np.sqrt(np.diag(cov0))
    mean, cov = _grid_posterior(y, sig, np.linspace(mean0[0] - 9 * sd[0], mean0[0] + 9 * sd[0], 2000),
                                np.linspace(mean0[1] - 9 * sd[1], mean0[1] + 9 * sd[1], 2000))
    r = orc.mcmc_run(**dict(MONO, step=list(1.5 * sd)), data=y[None], sigma=np.float32([sig]),
                     iterations=200_000, burnin=2_000, thin=1, n_chains=4, seed=77,
                     x0=np.tile(mean, (1, 4, 1)).astype(np.float32))
    _check_moments(r["samples"][:, :, :, 0], mean, cov)


def test_grid_posterior_one_parameter(orc):
    """S0 fixed by lb = ub; R2* alone, 1-D grid of 20,000 points."""
    sig = 0.02
    y = _voxel(orc, MONOEXP, TE12, [1.0, 25.0], sig, seed=13)
    r2 = np.linspace(15, 35, 20_000)
    s = np.exp(-r2[:, None] * TE12 * 1e-3)
    L = -0.5 * (((y.astype(np.float64) - s) / sig) ** 2).sum(-1)
    w = np.exp(L - L.max())
    w /= w.sum()
    m = (w * r2).sum()
    v = (w * (r2 - m) ** 2).sum()
    r = orc.mcmc_run(kind=MONOEXP, acq=TE12, lb=[1.0, 10.0], ub=[1.0, 80.0],
                     step=[0.0, 1.5 * np.sqrt(v)], data=y[None], sigma=np.float32([sig]),
                     iterations=200_000, burnin=2_000, thin=1, n_chains=4, seed=78,
                     x0=np.tile([1.0, m], (1, 4, 1)).astype(np.float32))
    _check_moments(r["samples"][:, :, 1:, 0], [m], np.array([[v]]))
    assert np.all(r["samples"][:, :, 0, 0] == 1.0)
