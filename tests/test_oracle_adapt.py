"""Pins of the oracle's convergence diagnostic and burn-in step adaptation.

R-hat (Gelman & Rubin 1992, no chain splitting): hand-computed values of two
small examples, its exact value for identical chains, invariance under affine
maps of the parameter and permutations of chains and of samples within a
chain, R-hat -> 1 for long i.i.d. chains, and the degenerate cases.

Step adaptation during burn-in (an extension; the paper's steps are fixed):
the multiplier each proposal uses, read back from the path of a chain whose
every proposal is accepted (a flat likelihood); the multiplier reached when
every proposal is rejected; the freeze after burn-in; and the exact
linear-Gaussian posterior of the post-burn-in states with adaptation on.
"""
import numpy as np
import pytest

from test_oracle_sampler import LINEAR, _check_moments

T12 = np.linspace(0.0, 1.0, 12)


# ------------------------------------------------------------------ R-hat --
def test_rhat_hand_examples(orc):
    # chains (0, 2) and (1, 3): chain means 1 and 2, within variances 2 and 2
    # -> W = 2; variance of the means (1 - 1.5)^2 + (2 - 1.5)^2 = 1/2 -> B/n = 1/2;
    # var+ = (1/2) 2 + 1/2 = 3/2; R-hat = sqrt(3/4)
    assert orc.rhat([[0.0, 2.0], [1.0, 3.0]]) == pytest.approx(np.sqrt(3.0) / 2.0, rel=1e-15)
    # chains (1,2,3), (2,3,4), (6,6,6): within variances 1, 1, 0 -> W = 2/3;
    # means 2, 3, 6 around 11/3: squared deviations 25/9 + 4/9 + 49/9 = 26/3,
    # over C - 1 = 2 -> B/n = 13/3; var+ = (2/3)(2/3) + 13/3 = 43/9;
    # R-hat = sqrt((43/9) / (2/3)) = sqrt(43/6)
    assert orc.rhat([[1.0, 2.0, 3.0], [2.0, 3.0, 4.0], [6.0, 6.0, 6.0]]) == \
        pytest.approx(np.sqrt(43.0 / 6.0), rel=1e-15)


def test_rhat_identical_chains_and_invariances(orc):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(37)
    # B = 0: R-hat = sqrt((n - 1) / n)
    assert orc.rhat(np.tile(x, (4, 1))) == pytest.approx(np.sqrt(36.0 / 37.0), rel=1e-14)
    ch = rng.standard_normal((5, 40)) + rng.standard_normal((5, 1))
    r = orc.rhat(ch)
    assert r > 1.0
    assert orc.rhat(-3.5 * ch + 11.0) == pytest.approx(r, rel=1e-12)
    assert orc.rhat(ch[[3, 0, 4, 1, 2]]) == pytest.approx(r, rel=1e-13)
    assert orc.rhat(ch[:, rng.permutation(40)]) == pytest.approx(r, rel=1e-13)


def test_rhat_long_iid_chains_near_one(orc):
    ch = np.random.default_rng(6).standard_normal((4, 200_000))
    assert abs(orc.rhat(ch) - 1.0) < 1e-4


def test_rhat_degenerate(orc):
    assert np.isnan(orc.rhat([[1.0, 2.0, 3.0]]))          # one chain
    assert np.isnan(orc.rhat([[1.0], [2.0]]))             # one sample per chain
    assert np.isnan(orc.rhat([[1.0, 1.0], [1.0, 1.0]]))   # W = B = 0
    assert np.isinf(orc.rhat([[1.0, 1.0], [2.0, 2.0]]))   # W = 0 < B


def test_sampler_rhat_is_that_of_its_moment_values(orc):
    t, y, sig, mu, sd = _linear()
    data = np.stack([y, y[::-1]])
    r = orc.mcmc_run(kind=LINEAR, acq=t, lb=mu - 50 * sd, ub=mu + 50 * sd, step=sd, data=data,
                     sigma=np.float32([sig, sig]), iterations=3000, burnin=500, thin=10,
                     n_chains=3, seed=4)
    for v in range(2):
        for p in range(2):
            assert r["rhat"][p, v] == pytest.approx(orc.rhat(r["samples"][:, :, p, v].T), rel=1e-12)
    one = orc.mcmc_run(kind=LINEAR, acq=t, lb=mu - 50 * sd, ub=mu + 50 * sd, step=sd, data=data,
                       sigma=np.float32([sig, sig]), iterations=300, burnin=50, thin=10,
                       n_chains=1, seed=4)
    assert np.isnan(one["rhat"]).all()


# ------------------------------------------------------- step adaptation --
def _linear(seed=11, sig=0.1):
    X = np.stack([np.ones(12), T12], 1)
    y = (X @ np.array([0.5, -1.0]) + sig * np.random.default_rng(seed).standard_normal(12)).astype(np.float32)
    XtX = X.T @ X
    mu = np.linalg.solve(XtX, X.T @ y.astype(np.float64))
    sd = np.sqrt(np.diag(sig ** 2 * np.linalg.inv(XtX)))
    return T12, y, sig, mu, sd


def _multipliers_used(orc, path, seed, v, c, step):
    """(theta_t - theta_{t-1}) / (step z_t) for every iteration of a chain that
    accepted everything and was never clamped."""
    I = path.shape[0] - 1
    lam = np.empty((I, path.shape[1]))
    for t in range(1, I + 1):
        z = orc.normals_from_words(orc.words(seed, t, v, c, orc.n_words(2)), 2)
        lam[t - 1] = (path[t] - path[t - 1]) / (step * z)
    return lam


@pytest.mark.parametrize("B,W,e_final", [(100, 10, 10), (95, 10, 9), (300, 10, 16), (0, 10, 0)])
def test_adaptation_when_every_proposal_is_accepted(orc, B, W, e_final):
    """Flat likelihood (sigma = 1e30): every proposal is accepted, so each
    window ending at t <= B raises e by one, up to 16; iteration t proposes with
    2^(e/4), e = the windows completed before t."""
    step = np.array([0.1, 0.2])
    seed, v, c, I = 31, 3, 1, B + 60
    path, acc, scale = orc.chain_path(LINEAR, T12, [-1e6, -1e6], [1e6, 1e6], step, np.zeros(12, np.float32),
                                      1e30, iterations=I, burnin=B, seed=seed, voxel=v, chain=c,
                                      x0=np.zeros(2, np.float32), adapt_window=W, adapt_target=0.5,
                                      want_scale=True)
    assert acc == 1.0
    lam = _multipliers_used(orc, path, seed, v, c, step)
    t = np.arange(1, I + 1)
    e = np.minimum(np.minimum((t - 1) // W, B // W), 16)
    np.testing.assert_allclose(lam, np.tile(2.0 ** (e / 4.0), (2, 1)).T, rtol=1e-9)
    assert scale == 2.0 ** (e_final / 4.0)


@pytest.mark.parametrize("B,e_final", [(200, -20), (400, -40), (700, -48)])
def test_adaptation_when_every_proposal_is_rejected(orc, B, e_final):
    """A noise-free voxel with sigma = 1e-9 started at its exact parameters:
    every move is rejected, so e falls by one per window, down to -48."""
    par = np.array([0.5, -1.0])
    y = (par[0] + par[1] * T12).astype(np.float32)
    path, acc, scale = orc.chain_path(LINEAR, T12, [-5, -5], [5, 5], [0.1, 0.1], y, 1e-9,
                                      iterations=B + 20, burnin=B, seed=8,
                                      x0=par.astype(np.float32), adapt_window=10, adapt_target=0.25,
                                      want_scale=True)
    assert acc == 0.0
    assert (path == path[0]).all()
    assert scale == 2.0 ** (e_final / 4.0)


def test_adaptation_off_is_the_fixed_step_sampler(orc):
    t, y, sig, mu, sd = _linear()
    kw = dict(kind=LINEAR, acq=t, lb=mu - 50 * sd, ub=mu + 50 * sd, step=sd, data=y[None],
              sigma=np.float32([sig]), iterations=800, burnin=200, thin=5, n_chains=2, seed=12)
    a, b = orc.mcmc_run(**kw), orc.mcmc_run(**kw, adapt_window=0, adapt_target=0.3)
    for k in ("samples", "mean", "std", "accept_rate"):
        np.testing.assert_array_equal(a[k], b[k])
    assert (a["step_scale"] == 1.0).all()
    for bad in (dict(adapt_window=-1, adapt_target=0.3), dict(adapt_window=10, adapt_target=0.0),
                dict(adapt_window=10, adapt_target=1.0)):
        with pytest.raises(ValueError):
            orc.mcmc_run(**kw, **bad)


def test_adapted_chain_samples_the_exact_posterior(orc):
    """Steps 30 SD wide at the start; adaptation shrinks them during the
    burn-in only, so the post-burn-in states are draws of the exact
    linear-Gaussian posterior (within 4 Monte-Carlo SE)."""
    t, y, sig, mu, sd = _linear()
    X = np.stack([np.ones(12), t], 1)
    cov = sig ** 2 * np.linalg.inv(X.T @ X)
    r = orc.mcmc_run(kind=LINEAR, acq=t, lb=mu - 100 * sd, ub=mu + 100 * sd, step=30 * sd,
                     data=y[None], sigma=np.float32([sig]), iterations=250_000, burnin=5_000, thin=1,
                     n_chains=4, seed=2026, x0=np.tile(mu, (1, 4, 1)).astype(np.float32),
                     adapt_window=50, adapt_target=0.3)
    e = np.round(4 * np.log2(r["step_scale"]))
    assert (e < -8).all() and (e > -24).all()  # from 30 SD down to about 1-3 SD
    _check_moments(r["samples"][:, :, :, 0], mu, cov)
    post = r["accept_rate"] * 250_000  # accepted moves, dominated by the post-burn-in ones
    assert (0.15 < post / 250_000).all() and (post / 250_000 < 0.5).all()
