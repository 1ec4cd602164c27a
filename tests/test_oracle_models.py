"""Pins of the oracle's forward models and likelihood against closed forms,
library special functions and quadrature, and invariants of each model.

Mono-exponential decay is Eq. 3; the 3-pool myelin-water and spherical-mean
Standard Model forms are the closed forms stated in the oracle's source.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy import special, stats

MONOEXP, MWI3, SMT, LINEAR = 1, 2, 3, 100
TE12 = np.array([2.0 + 3 * k for k in range(12)])
TE24 = np.array([2.0 + k * 44 / 23 for k in range(24)])
BVALS = np.array([0.0, 1.0, 2.5, 5.0, 7.5, 10.0])


# ----------------------------------------------------------- mono-exponential
def test_monoexp_closed_form_limits(orc):
    rng = np.random.default_rng(1)
    th = np.stack([rng.uniform(0.5, 1.5, 50), rng.uniform(10, 80, 50)], 1)
    s0 = orc.forward(MONOEXP, [0.0], th)[:, 0]
    np.testing.assert_allclose(s0, th[:, 0], rtol=0, atol=0)  # S(TE = 0) = S0
    s = orc.forward(MONOEXP, TE12, th)
    assert (s > 0).all()  # a mono-exponential never reaches 0 at these TE
    for i in range(50):  # log S is linear in TE with slope -R2* (TE in ms, R2* in 1/s)
        slope, icpt = np.polyfit(TE12, np.log(s[i]), 1)
        assert slope == pytest.approx(-th[i, 1] * 1e-3, rel=1e-12)
        assert np.exp(icpt) == pytest.approx(th[i, 0], rel=1e-12)


# ------------------------------------------------------------------ 3-pool
def _mwi3_theta(rng, n):
    return np.stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n),
                     rng.uniform(3, 20, n), rng.uniform(40, 80, n), rng.uniform(30, 60, n),
                     rng.uniform(-10, 20, n), rng.uniform(-10, 20, n),
                     rng.uniform(-np.pi, np.pi, n)], 1)


def _cplx(s):
    return s[..., 0::2] + 1j * s[..., 1::2]


def test_mwi3_at_t0_is_rotated_amplitude_sum(orc):
    th = _mwi3_theta(np.random.default_rng(2), 40)
    s = _cplx(orc.forward(MWI3, [0.0], th))[:, 0]
    np.testing.assert_allclose(s, th[:, :3].sum(1) * np.exp(1j * th[:, 8]), rtol=1e-14)


def test_mwi3_real_when_no_frequency_and_phase(orc):
    th = _mwi3_theta(np.random.default_rng(3), 40)
    th[:, 6:9] = 0.0
    s = _cplx(orc.forward(MWI3, TE24, th))
    assert np.abs(s.imag).max() == 0.0
    # then it is the sum of three mono-exponentials with R2* = 1000 / T2* [1/s]
    ref = sum(orc.forward(MONOEXP, TE24, np.stack([th[:, j], 1000.0 / th[:, 3 + j]], 1))
              for j in range(3))
    np.testing.assert_allclose(s.real, ref, rtol=1e-13)


def test_mwi3_single_pool_phase_and_modulus(orc):
    th = _mwi3_theta(np.random.default_rng(4), 40)
    th[:, 1:3] = 0.0  # only the myelin-water pool
    s = _cplx(orc.forward(MWI3, TE24, th))
    mod = th[:, :1] * np.exp(-TE24[None] / th[:, 3:4])
    np.testing.assert_allclose(np.abs(s), mod, rtol=1e-13)
    # arg S(t) = phi0 - 2 pi df t  (t in ms, df in Hz)
    want = th[:, 8:9] - 2 * np.pi * th[:, 6:7] * TE24[None] * 1e-3
    d = np.angle(s * np.exp(-1j * want))
    assert np.abs(d).max() < 1e-12
    # the extra-cellular pool has no frequency offset: a single EW pool is df-free
    th2 = th.copy()
    th2[:, 0] = 0.0
    th2[:, 2] = 0.7
    s2 = _cplx(orc.forward(MWI3, TE24, th2))
    np.testing.assert_allclose(np.angle(s2 * np.exp(-1j * th2[:, 8:9])), 0.0, atol=1e-12)


def test_mwi3_modulus_invariant_under_global_phase(orc):
    th = _mwi3_theta(np.random.default_rng(5), 40)
    a = orc.forward(MWI3, TE24, th)
    th2 = th.copy()
    th2[:, 8] = np.random.default_rng(6).uniform(-np.pi, np.pi, 40)
    b = orc.forward(MWI3, TE24, th2)
    np.testing.assert_allclose(np.abs(_cplx(a)), np.abs(_cplx(b)), rtol=1e-13)
    np.testing.assert_allclose(_cplx(a) * np.exp(1j * (th2[:, 8:9] - th[:, 8:9])), _cplx(b),
                               rtol=1e-12, atol=1e-15)


# ------------------------------------------------- spherical-mean SM model
def _g_quadrature(x, n=400):
    u, w = leggauss(n)
    u = 0.5 * (u + 1.0)
    return 0.5 * np.sum(w * np.exp(-x * u * u))


G_POINTS = [-15.0, -10.0, -3.0, -1.0, -0.5, -1e-4, -1e-9, 0.0, 1e-9, 1e-4, 0.3, 0.999999, 1.0,
            1.000001, 2.0, 7.5, 30.0, 40.0]


@pytest.mark.parametrize("x", G_POINTS)
def test_smt_g_against_adaptive_quadrature(orc, x):
    """g(x) = integral_0^1 exp(-x u^2) du, by 40-digit adaptive quadrature."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    exact = mp.quad(lambda u: mp.exp(-x * u * u), [0, 1])
    assert orc.g(x) == pytest.approx(float(exact), rel=1e-14)


@pytest.mark.parametrize("x", G_POINTS)
def test_smt_g_against_gauss_legendre(orc, x):
    # 400-node Gauss-Legendre in double precision carries ~1e-13 of rounding
    assert orc.g(x) == pytest.approx(_g_quadrature(x), rel=1e-12)


def test_smt_g_against_erf_and_erfi(orc):
    for x in np.linspace(0.05, 40, 60):
        s = np.sqrt(x)
        assert orc.g(x) == pytest.approx(np.sqrt(np.pi) * special.erf(s) / (2 * s), rel=1e-13)
    for y in np.linspace(0.05, 15, 60):
        s = np.sqrt(y)  # g(-y) = sqrt(pi) erfi(sqrt y) / (2 sqrt y) = exp(y) D(sqrt y)/sqrt y
        assert orc.g(-y) == pytest.approx(np.sqrt(np.pi) * special.erfi(s) / (2 * s), rel=1e-12)
        assert orc.g(-y) == pytest.approx(np.exp(y) * special.dawsn(s) / s, rel=1e-12)


def test_smt_limits(orc):
    rng = np.random.default_rng(7)
    th = np.stack([rng.uniform(0, 1, 50), rng.uniform(1, 3, 50), rng.uniform(0.5, 3, 50),
                   rng.uniform(0, 1.5, 50)], 1)
    s = orc.forward(SMT, BVALS, th)
    np.testing.assert_allclose(s[:, 0], 1.0, rtol=1e-15)  # S(b = 0) = S0 = 1
    b = BVALS[1:]
    # f = 1: pure stick, sqrt(pi/(4 b Da)) erf(sqrt(b Da))
    th1 = th.copy()
    th1[:, 0] = 1.0
    s1 = orc.forward(SMT, b, th1)
    ref = np.sqrt(np.pi / (4 * b[None] * th1[:, 1:2])) * special.erf(np.sqrt(b[None] * th1[:, 1:2]))
    np.testing.assert_allclose(s1, ref, rtol=1e-13)
    # f = 0, De_par = De_perp = D: isotropic Gaussian exp(-b D)
    th2 = th.copy()
    th2[:, 0] = 0.0
    th2[:, 2] = th2[:, 3] = rng.uniform(0.2, 2.0, 50)
    np.testing.assert_allclose(orc.forward(SMT, b, th2), np.exp(-b[None] * th2[:, 2:3]), rtol=1e-14)
    # f = 0, De_perp = 0: a stick of diffusivity De_par (zeppelin limit)
    th3 = th.copy()
    th3[:, 0] = 0.0
    th3[:, 3] = 0.0
    ref3 = np.sqrt(np.pi / (4 * b[None] * th3[:, 2:3])) * special.erf(np.sqrt(b[None] * th3[:, 2:3]))
    np.testing.assert_allclose(orc.forward(SMT, b, th3), ref3, rtol=1e-13)


def test_smt_extra_term_by_orientation_quadrature(orc):
    """Extra-axonal term = spherical mean of an axisymmetric tensor signal,
    integral_0^1 exp(-b (De_perp + (De_par - De_perp) u^2)) du, by quadrature,
    including De_par < De_perp (the erfi branch)."""
    rng = np.random.default_rng(8)
    for _ in range(30):
        dpar, dperp = rng.uniform(0.5, 3), rng.uniform(0, 1.5)
        th = np.array([0.0, 2.0, dpar, dperp])
        s = orc.forward(SMT, BVALS, th)
        u, w = leggauss(400)
        u = 0.5 * (u + 1)
        ref = [0.5 * np.sum(w * np.exp(-bb * (dperp + (dpar - dperp) * u * u))) for bb in BVALS]
        np.testing.assert_allclose(s, ref, rtol=1e-12)


# ------------------------------------------------------------------ linear
def test_linear_model(orc):
    th = np.array([[0.3, -2.0], [1.5, 4.0]])
    t = np.linspace(0, 1, 12)
    np.testing.assert_array_equal(orc.forward(LINEAR, t, th), th[:, :1] + th[:, 1:] * t[None])


# -------------------------------------------------------------- likelihood
def test_loglik_is_gaussian_log_density_up_to_constant(orc):
    rng = np.random.default_rng(9)
    th = _mwi3_theta(rng, 30)
    s = orc.forward(MWI3, TE24, th)
    sig = rng.uniform(0.005, 0.05, 30).astype(np.float32)
    y = (s + sig[:, None] * rng.standard_normal(s.shape)).astype(np.float32)
    L = orc.loglik(MWI3, TE24, th, y, sig)
    sd = sig.astype(np.float64)
    ref = stats.norm.logpdf(y.astype(np.float64), s, sd[:, None]).sum(1) \
        + s.shape[1] * np.log(sd * np.sqrt(2 * np.pi))
    np.testing.assert_allclose(L, ref, rtol=1e-11)
    assert np.all(L <= 0)


def test_loglik_zero_at_exact_fit_and_scales_with_sigma(orc):
    t = np.arange(12) / 8.0
    th = np.array([[0.25, -0.5]])  # signal values exactly representable in float32
    y = orc.forward(LINEAR, t, th).astype(np.float32)
    assert np.all(y.astype(np.float64) == orc.forward(LINEAR, t, th))
    assert orc.loglik(LINEAR, t, th, y, [1.0])[0] == 0.0
    y2 = y + np.float32(0.125)
    l1 = orc.loglik(LINEAR, t, th, y2, [1.0])[0]
    l2 = orc.loglik(LINEAR, t, th, y2, [0.5])[0]
    assert l1 == pytest.approx(-0.5 * 12 * 0.125 ** 2, rel=1e-15)
    assert l2 == pytest.approx(4 * l1, rel=1e-15)
