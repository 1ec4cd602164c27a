"""Pins of the oracle's affine-invariant ensemble sampler (Sec. 2.2.2).

- the stretch factor z has density proportional to 1/sqrt(z) on [1/a, a]
  (closed-form CDF, Kolmogorov-Smirnov);
- every walker move of a path follows the documented construction (two
  halves, partner from the other half, proposal X_j + z (X_k - X_j), prior
  box, acceptance with the z^(P-1) factor);
- affine invariance (Goodman & Weare): the same random numbers on an affinely
  reparametrised target give the affinely mapped walker paths;
- stationary distribution: the exact linear-Gaussian posterior and a
  brute-force grid posterior, within 4 Monte-Carlo standard errors.
"""
import numpy as np
import pytest
from scipy import stats

from test_oracle_sampler import _batch_mcse, _grid_posterior, _voxel

LINEAR, MONOEXP = 100, 1
TE12 = np.array([2.0 + 3 * k for k in range(12)])


@pytest.mark.parametrize("a", [1.5, 2.0, 3.0])
def test_stretch_distribution(orc, a):
    rng = np.random.default_rng(int(a * 10))
    w = rng.integers(0, 2 ** 32, 200_000, dtype=np.uint64)
    z = np.array([orc.stretch_z(int(x), a) for x in w[:200_000]])
    assert z.min() >= 1 / a and z.max() <= a
    cdf = lambda x: (np.sqrt(x) - 1 / np.sqrt(a)) / (np.sqrt(a) - 1 / np.sqrt(a))
    assert stats.kstest(z, cdf).pvalue > 1e-3
    assert orc.stretch_z(0, a) == pytest.approx(1 / a, rel=1e-8)
    assert orc.stretch_z(0xFFFFFFFF, a) == pytest.approx(a, rel=1e-8)


def _linear_problem(seed=11, sig=0.1):
    t = np.linspace(0.0, 1.0, 12)
    X = np.stack([np.ones(12), t], 1)
    y = (X @ np.array([0.5, -1.0]) + sig * np.random.default_rng(seed).standard_normal(12)).astype(np.float32)
    XtX = X.T @ X
    mu = np.linalg.solve(XtX, X.T @ y.astype(np.float64))
    cov = sig ** 2 * np.linalg.inv(XtX)
    return t, y, sig, mu, cov


def test_every_walker_move(orc):
    t, y, sig, mu, cov = _linear_problem()
    sd = np.sqrt(np.diag(cov))
    lb, ub = mu - 1.5 * sd, mu + 1.5 * sd  # tight: proposals often leave the box
    L, I, a, seed, v = 8, 60, 2.0, 77, 5
    path, acc = orc.ensemble_path(LINEAR, t, lb, ub, y, sig, iterations=I, n_walkers=L, seed=seed,
                                  stretch=a, voxel=v)
    H = L // 2
    X = path[0].copy()
    # initial walkers: the uniform-prior draw of counter iteration 0xFFFFFFFF
    for k in range(L):
        w0 = orc.words(seed, 0xFFFFFFFF, v, k, 2)
        np.testing.assert_array_equal(X[k], lb + (ub - lb) * np.array([orc.u01(x) for x in w0]))
    LL = orc.loglik(LINEAR, t, X, np.tile(y, (L, 1)), np.full(L, sig, np.float32))
    n_acc = np.zeros(L)
    outside = 0
    for it in range(1, I + 1):
        for h in (0, 1):
            other = (1 - h) * H
            for i in range(H):
                k = h * H + i
                w = orc.words(seed, it, v, k, 3)
                j = other + (int(w[0]) * H >> 32)
                z = orc.stretch_z(int(w[1]), a)
                Y = X[j] + z * (X[k] - X[j])
                if np.any(Y < lb) or np.any(Y > ub):
                    outside += 1
                    continue
                Ly = orc.loglik(LINEAR, t, Y[None], y[None], [sig])[0]
                if np.log(orc.u01(int(w[2]))) < (2 - 1) * np.log(z) + Ly - LL[k]:
                    X[k], LL[k] = Y, Ly
                    n_acc[k] += 1
        np.testing.assert_array_equal(X, path[it], err_msg=f"iteration {it}")
    np.testing.assert_array_equal(acc, n_acc / I)
    assert outside > 0 and n_acc.sum() > 0


def test_affine_invariance(orc):
    """Reparametrise the linear model s = a + c t as c' = kappa c with
    acquisitions t / kappa.  With the same random numbers, walker k of the new
    problem is the image (a, kappa c) of walker k of the old one; for
    kappa = 4 every operation scales exactly, so the paths map bit for bit.
    A general affine change (also shifting a by beta through the data) maps
    them up to rounding, checked over a short run."""
    t, y, sig, mu, cov = _linear_problem()
    sd = np.sqrt(np.diag(cov))
    lb, ub = mu - 200 * sd, mu + 200 * sd
    L, seed = 16, 9
    x0 = (mu + sd * np.random.default_rng(2).standard_normal((L, 2))).astype(np.float32).astype(np.float64)
    A = np.array([1.0, 4.0])
    p1, a1 = orc.ensemble_path(LINEAR, t, lb, ub, y, sig, iterations=300, n_walkers=L, seed=seed,
                               x0=x0.astype(np.float32))
    p2, a2 = orc.ensemble_path(LINEAR, t / 4.0, lb * A, ub * A, y, sig, iterations=300, n_walkers=L,
                               seed=seed, x0=(x0 * A).astype(np.float32))
    np.testing.assert_array_equal(p2, p1 * A)
    np.testing.assert_array_equal(a1, a2)
    assert a1.mean() > 0.1
    # general affine change: c' = 3 c, a' = a - 0.25, over 20 iterations
    A3, shift = np.array([1.0, 3.0]), np.array([0.25, 0.0])
    x0b = ((x0 * A3 - shift).astype(np.float32).astype(np.float64) + shift) / A3
    q1, _ = orc.ensemble_path(LINEAR, t, lb, ub, y, sig, iterations=20, n_walkers=L, seed=seed,
                              x0=x0b.astype(np.float32))
    q2, _ = orc.ensemble_path(LINEAR, t / 3.0, lb * A3 - shift, ub * A3 - shift, y - np.float32(0.25),
                              sig, iterations=20, n_walkers=L, seed=seed,
                              x0=(x0b.astype(np.float32).astype(np.float64) * A3 - shift).astype(np.float32))
    assert np.abs(q2 - (q1 * A3 - shift)).max() < 1e-5


def _check(samples, mean_ref, cov_ref, k=4.0):
    """samples [S][L][P]: pooled mean and covariance within k MCSE, the MCSE
    from batch means of the walker-averaged series."""
    xs = samples.mean(axis=1)  # [S][P] ensemble average per iteration
    S, L, P = samples.shape
    for p in range(P):
        se = _batch_mcse(xs[None, :, p], n_batches=40)
        m = samples[:, :, p].mean()
        assert abs(m - mean_ref[p]) < k * se, (p, m, mean_ref[p], se)
        for q in range(p, P):
            prod = ((samples[:, :, p] - mean_ref[p]) * (samples[:, :, q] - mean_ref[q])).mean(axis=1)
            se2 = _batch_mcse(prod[None], n_batches=40)
            assert abs(prod.mean() - cov_ref[p, q]) < k * se2 + 1e-12, (p, q, prod.mean(), cov_ref[p, q], se2)


def test_linear_gaussian_posterior(orc):
    t, y, sig, mu, cov = _linear_problem()
    sd = np.sqrt(np.diag(cov))
    L = 32
    x0 = (mu + 0.5 * sd * np.random.default_rng(3).standard_normal((1, L, 2))).astype(np.float32)
    r = orc.ensemble_run(LINEAR, t, mu - 100 * sd, mu + 100 * sd, y[None], np.float32([sig]),
                         iterations=40_000, burnin=1_000, thin=1, n_walkers=L, seed=2025, x0=x0)
    _check(r["samples"][:, :, :, 0], mu, cov)
    assert 0.2 < r["accept_rate"].mean() < 0.9


def test_grid_posterior_two_parameters(orc):
    sig = 0.01
    y = _voxel(orc, MONOEXP, TE12, [1.0, 40.0], sig, seed=12)
    mean0, cov0 = _grid_posterior(y, sig, np.linspace(0.9, 1.1, 400), np.linspace(30, 50, 400))
    sd = np.sqrt(np.diag(cov0))
    mean, cov = _grid_posterior(y, sig, np.linspace(mean0[0] - 9 * sd[0], mean0[0] + 9 * sd[0], 2000),
                                np.linspace(mean0[1] - 9 * sd[1], mean0[1] + 9 * sd[1], 2000))
    L = 24
    x0 = (mean + sd * np.random.default_rng(4).standard_normal((1, L, 2))).astype(np.float32)
    r = orc.ensemble_run(MONOEXP, TE12, [0.5, 10.0], [1.5, 80.0], y[None], np.float32([sig]),
                         iterations=30_000, burnin=1_000, thin=1, n_walkers=L, seed=78, x0=x0)
    _check(r["samples"][:, :, :, 0], mean, cov)


def test_table1_ensemble_sample_count(orc):
    """Table 1: 50 walkers x 2000 iterations, 10% burn-in, thinning 100 -> 900."""
    t, y, sig, mu, cov = _linear_problem()
    sd = np.sqrt(np.diag(cov))
    r = orc.ensemble_run(LINEAR, t, mu - 100 * sd, mu + 100 * sd, y[None], np.float32([sig]),
                         iterations=2000, burnin=200, thin=100, n_walkers=50, seed=1)
    assert r["samples"].shape[0] * r["samples"].shape[1] == 900


def test_rejects_bad_ensembles(orc):
    t, y, sig, mu, cov = _linear_problem()
    for L, a in ((7, 2.0), (2, 2.0), (8, 1.0)):
        with pytest.raises(ValueError):
            orc.ensemble_run(LINEAR, t, [-9, -9], [9, 9], y[None], np.float32([sig]), iterations=10,
                             burnin=0, thin=1, n_walkers=L, seed=1, stretch=a)
