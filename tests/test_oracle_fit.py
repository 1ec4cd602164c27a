"""Pins of the oracle's whole-volume gradient fit (askadam.m, Sec. 2.2.1,
Eq. 2, 4, 5).

- dg/dx against 40-digit quadrature of -int_0^1 u^2 exp(-x u^2) du;
- every model's hand-written Jacobian against central finite differences of
  the (separately pinned) forward model;
- the loss gradient, data and total-variation terms together, against
  central finite differences of the loss the oracle reports: with Adam's
  epsilon far above the gradient the update is plain gradient descent with
  step lr/eps, which exposes the gradient's size, not only its sign;
- Adam's first step moves every free parameter by lr against the gradient;
- the window slope against numpy's least-squares fit, and both stopping rules
  at the iteration the full loss history predicts;
- L2 on the linear model converges to the exact parameters of noise-free
  data; the mask leaves outside voxels untouched.
"""
import mpmath as mp
import numpy as np
import pytest

MONOEXP, MWI3, SMT, LINEAR = 1, 2, 3, 100
TE12 = np.array([2.0 + 3 * k for k in range(12)])
TE24 = np.array([2.0 + 44.0 * k / 23 for k in range(24)])
BVALS = np.array([0.0, 1.0, 2.5, 5.0, 7.5, 10.0])
MODELS = {
    MONOEXP: (TE12, [0.5, 10.0], [1.5, 80.0]),
    MWI3: (TE24, [0.0, 0.0, 0.0, 3.0, 40.0, 30.0, -10.0, -10.0, -np.pi], [1.0, 1.0, 1.0, 20.0, 80.0, 60.0, 20.0, 20.0, np.pi]),
    SMT: (BVALS, [0.0, 1.0, 0.5, 0.0], [1.0, 3.0, 3.0, 1.5]),
    LINEAR: (np.linspace(0, 1, 12), [-2.0, -3.0], [2.0, 3.0]),
}


@pytest.mark.parametrize("x", [-10.0, -1.0, -0.3, 0.0, 0.5, 1.0, 3.0, 20.0])
def test_dg_against_quadrature(orc, x):
    mp.mp.dps = 40
    want = -mp.quad(lambda u: u * u * mp.exp(-mp.mpf(x) * u * u), [0, 1])
    assert orc.dg(x) == pytest.approx(float(want), rel=1e-13, abs=1e-16)


@pytest.mark.parametrize("kind", list(MODELS))
def test_jacobian_against_finite_differences(orc, kind):
    acq, lb, ub = MODELS[kind]
    rng = np.random.default_rng(kind)
    lb, ub = np.array(lb), np.array(ub)
    for _ in range(20):
        th = rng.uniform(lb + 0.1 * (ub - lb), ub - 0.1 * (ub - lb))
        s, J = orc.jacobian(kind, acq, th)
        np.testing.assert_allclose(s, orc.forward(kind, acq, th), rtol=1e-15, atol=1e-15)
        for p in range(len(th)):
            h = 1e-6 * (ub[p] - lb[p])
            e = np.zeros_like(th)
            e[p] = h
            fd = (orc.forward(kind, acq, th + e) - orc.forward(kind, acq, th - e)) / (2 * h)
            np.testing.assert_allclose(J[:, p], fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max(initial=1e-30))


def _volume(orc, kind, shape, seed=5, noise=0.01):
    acq, lb, ub = MODELS[kind]
    rng = np.random.default_rng(seed)
    lb, ub = np.array(lb), np.array(ub)
    N = int(np.prod(shape))
    truth = rng.uniform(lb + 0.2 * (ub - lb), ub - 0.2 * (ub - lb), (N, len(lb)))
    y = orc.forward(kind, acq, truth)
    y = (y + noise * rng.standard_normal(y.shape)).astype(np.float32)
    theta0 = rng.uniform(lb + 0.3 * (ub - lb), ub - 0.3 * (ub - lb), (N, len(lb)))
    return acq, lb, ub, y, truth, theta0


def _loss(orc, kind, acq, lb, ub, y, theta, **kw):
    th, hist, done = orc.fit_run(kind, acq, lb, ub, y, theta, iterations=1, **kw)
    return hist[0]


@pytest.mark.parametrize("kind,loss,lam", [(MONOEXP, 2, 0.0), (MWI3, 2, 0.0), (SMT, 1, 0.0), (SMT, 2, 0.3),
                                           (LINEAR, 1, 0.05)])
def test_loss_gradient_against_finite_differences(orc, kind, loss, lam):
    shape = (3, 2, 2)
    acq, lb, ub, y, truth, theta0 = _volume(orc, kind, shape)
    kw = dict(shape=shape, loss=loss, lam=lam, tv_params=0b1 if lam else 0, tv_dims=3)
    eps, lr = 1e3, 1.0  # Adam with epsilon >> |gradient|: u <- u - lr g / (|g| + eps)
    th1, hist, _ = orc.fit_run(kind, acq, lb, ub, y, theta0, iterations=1, lr=lr, eps=eps, **kw)
    step = -(th1 - theta0) / (ub - lb)
    g = step * eps / (lr - np.abs(step))  # gradient with respect to u
    rng = np.random.default_rng(1)
    for v, p in zip(rng.integers(0, theta0.shape[0], 6), rng.integers(0, len(lb), 6)):
        h = 1e-5 * (ub[p] - lb[p])
        tp, tm = theta0.copy(), theta0.copy()
        tp[v, p] += h
        tm[v, p] -= h
        fd = (_loss(orc, kind, acq, lb, ub, y, tp, **kw) - _loss(orc, kind, acq, lb, ub, y, tm, **kw)) / (2 * h)
        fd *= ub[p] - lb[p]
        assert g[v, p] == pytest.approx(fd, rel=1e-4, abs=1e-9), (v, p)


def test_adam_first_step_is_lr_against_the_gradient(orc):
    shape = (4, 3, 1)
    acq, lb, ub, y, truth, theta0 = _volume(orc, SMT, shape)
    lr = 1e-3
    th1, _, _ = orc.fit_run(SMT, acq, lb, ub, y, theta0, shape=shape, iterations=1, lr=lr, loss=2)
    du = (th1 - theta0) / (ub - lb)
    # the gradient, from a plain gradient step (Adam with epsilon >> |g|)
    th_gd, _, _ = orc.fit_run(SMT, acq, lb, ub, y, theta0, shape=shape, iterations=1, lr=1.0, eps=1e3, loss=2)
    step = -(th_gd - theta0) / (ub - lb)
    g = step * 1e3 / (1.0 - np.abs(step))
    # bias-corrected first moments are g and g^2: the step is lr g / (|g| + 1e-8), downhill
    np.testing.assert_allclose(du, -lr * g / (np.abs(g) + 1e-8), rtol=1e-6)
    assert (np.abs(du) > 0.99 * lr).mean() > 0.9


def test_window_slope_and_stopping_rules(orc):
    rng = np.random.default_rng(3)
    for n in (2, 5, 20):
        y = rng.standard_normal(n)
        assert orc.window_slope(y) == pytest.approx(np.polyfit(np.arange(n), y, 1)[0], rel=1e-12, abs=1e-15)
    shape = (4, 4, 1)
    acq, lb, ub, y, truth, theta0 = _volume(orc, MONOEXP, shape)
    kw = dict(shape=shape, loss=1, lr=0.02)
    _, full, done = orc.fit_run(MONOEXP, acq, lb, ub, y, theta0, iterations=300, **kw)
    assert done == 300
    tol = float(np.quantile(full, 0.3))
    _, h_tol, d_tol = orc.fit_run(MONOEXP, acq, lb, ub, y, theta0, iterations=300, tol=tol, **kw)
    assert d_tol == int(np.argmax(full < tol)) + 1
    np.testing.assert_array_equal(h_tol, full[:d_tol])
    W = 20
    slopes = np.array([abs(np.polyfit(np.arange(W), full[t - W:t], 1)[0]) for t in range(W, 301)])
    cv = float(np.quantile(slopes, 0.2))
    _, h_cv, d_cv = orc.fit_run(MONOEXP, acq, lb, ub, y, theta0, iterations=300, conv_value=cv, conv_window=W, **kw)
    assert d_cv == W + int(np.argmax(slopes < cv))
    # a threshold just above the first window's slope stops at t = W exactly
    _, _, d_first = orc.fit_run(MONOEXP, acq, lb, ub, y, theta0, iterations=300, conv_value=slopes[0] * 1.0001,
                                conv_window=W, **kw)
    assert d_first == W


def test_l2_linear_model_recovers_noise_free_parameters(orc):
    shape = (5, 1, 1)
    acq, lb, ub, y, truth, theta0 = _volume(orc, LINEAR, shape, noise=0.0)
    th, hist, done = orc.fit_run(LINEAR, acq, lb, ub, y, theta0, shape=shape, iterations=6000, lr=0.003, loss=2)
    np.testing.assert_allclose(th, truth, atol=2e-3)
    assert hist[-1] < 1e-6 * hist[0]


def test_mask_and_total_variation(orc):
    shape = (6, 1, 1)
    acq, lb, ub, y, truth, theta0 = _volume(orc, MONOEXP, shape, noise=0.02)
    mask = np.array([1, 1, 0, 1, 1, 1], np.uint8)
    th, _, _ = orc.fit_run(MONOEXP, acq, lb, ub, y, theta0, shape=shape, mask=mask, iterations=50, lr=0.01)
    np.testing.assert_array_equal(th[2], theta0[2])
    assert (th[mask == 1] != theta0[mask == 1]).all()
    # a strong TV on S0 along x makes the masked S0 values nearly equal
    th_tv, _, _ = orc.fit_run(MONOEXP, acq, lb, ub, y, theta0, shape=shape, mask=mask, iterations=3000, lr=0.003,
                              lam=5.0, tv_params=0b1, tv_dims=2)
    s0 = th_tv[mask == 1, 0]
    assert np.ptp(s0) < 0.2 * np.ptp(truth[mask == 1, 0])
