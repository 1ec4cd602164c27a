"""Pins of the oracle's AxCaliberSMT model (Sec. 2.5; Fan et al. 2020).

- the zeros of J1' against scipy's jnp_zeros, and the sum rule
  sum_m 1/(x_m^4 (x_m^2 - 1)) = 7/192 behind Neuman's wide-pulse limit;
- the cylinder's Gaussian-phase attenuation kappa: Neuman's wide-pulse
  limit (7/48) gamma^2 G^2 delta R^4 / D with its 1/delta approach, the free
  diffusion bound kappa <= b D and the approach to it as R grows, exact
  proportionality to b at fixed timing;
- the restricted compartment's spherical mean e^{-k} g(b D - k) against a
  Gauss-Legendre orientation average of e^{-b D u^2 - k (1 - u^2)};
- compartment reductions: S(b=0) = 1, pure free water, the zeppelin and
  stick limits against the oracle's Standard Model.
"""
import numpy as np
import pytest
from scipy import special

SMT, AXCAL = 3, 4
DA, DEPAR, DCSF = 1.7, 1.7, 3.0


def test_j1p_zeros_against_scipy(orc):
    ref = special.jnp_zeros(1, 100)
    got = np.array([orc.j1p_zero(m) for m in range(1, 101)])
    np.testing.assert_allclose(got, ref, rtol=1e-13)


def test_neuman_sum_rule():
    x = special.jnp_zeros(1, 2000)
    assert np.sum(1.0 / (x ** 4 * (x ** 2 - 1.0))) == pytest.approx(7.0 / 192.0, rel=1e-12)


def _neuman(b, Delta, delta, R, D):
    g2 = b / (delta ** 2 * (Delta - delta / 3.0))  # gamma^2 G^2
    return 7.0 / 48.0 * g2 * delta * R ** 4 / D


@pytest.mark.parametrize("Delta_over_delta", [1.0, 2.0])
def test_wide_pulse_limit(orc, Delta_over_delta):
    """delta >> R^2/D: kappa -> Neuman's (7/48) gamma^2 G^2 delta R^4 / D, the
    relative gap shrinking as 1/delta."""
    R, D, b = 1.0, 1.7, 2.0
    gaps = []
    for delta in (50.0, 100.0, 200.0, 400.0):
        Delta = Delta_over_delta * delta
        k = orc.cyl_kappa(b, Delta, delta, R, D)
        gaps.append(1.0 - k / _neuman(b, Delta, delta, R, D))
    gaps = np.array(gaps)
    assert (gaps > 0).all() and gaps[-1] < 5e-3
    np.testing.assert_allclose(gaps[1:] / gaps[:-1], 0.5, rtol=0.02)


def test_free_diffusion_bound_and_limit(orc):
    b, Delta, delta, D = 6.0, 13.0, 6.0, DA
    Rs = np.array([0.5, 2.0, 8.0, 32.0, 64.0, 128.0, 256.0])
    ks = np.array([orc.cyl_kappa(b, Delta, delta, R, D) for R in Rs])
    assert (ks <= b * D * (1 + 1e-12)).all()
    assert (np.diff(ks) > 0).all()
    # wide cylinders: the deficit 1 - kappa/(b D) falls as 1/R (the surface-to-
    # volume law of restricted diffusion at short times)
    deficit = 1.0 - ks / (b * D)
    np.testing.assert_allclose(deficit[4:-1] / deficit[5:], 2.0, rtol=0.03)
    # exactly proportional to b (to G^2) at fixed timing
    for R in (1.0, 4.0):
        assert orc.cyl_kappa(3 * b, Delta, delta, R, D) == pytest.approx(3 * orc.cyl_kappa(b, Delta, delta, R, D),
                                                                          rel=1e-14)
    assert orc.cyl_kappa(0.0, Delta, delta, 2.0, D) == 0.0


def _acq(bs, Delta, delta):
    return np.array([[b, Delta, delta] for b in bs], float).ravel()


def test_restricted_spherical_mean_against_orientation_quadrature(orc):
    """f_n = 1, f_csf = 0: the signal is the orientation average of the
    cylinder, e^{-b Da u^2 - k (1 - u^2)} over u = cos(angle) in [0, 1]."""
    u, w = np.polynomial.legendre.leggauss(200)
    u, w = 0.5 * (u + 1.0), 0.5 * w
    for (b, Delta, delta, a) in ((0.8, 13.0, 6.0, 3.0), (6.0, 13.0, 6.0, 6.0), (17.8, 30.0, 6.0, 2.0),
                                 (4.25, 30.0, 6.0, 10.0)):
        k = orc.cyl_kappa(b, Delta, delta, a / 2, DA)
        want = np.sum(w * np.exp(-b * DA * u ** 2 - k * (1 - u ** 2)))
        s = orc.forward(AXCAL, _acq([b], Delta, delta), [a, 1.0, 0.0, 0.5])
        assert s[0] == pytest.approx(want, rel=1e-12), (b, a)


def test_compartment_reductions(orc):
    bs = [0.0, 0.05, 0.8, 2.4, 6.0, 9.85, 17.8]
    acq = _acq(bs, 30.0, 6.0)
    b = np.array(bs)
    # b = 0: S0 = 1 whatever the parameters
    assert orc.forward(AXCAL, _acq([0.0], 13.0, 6.0), [5.0, 0.4, 0.2, 0.7])[0] == 1.0
    # free water only
    np.testing.assert_allclose(orc.forward(AXCAL, acq, [4.0, 0.6, 1.0, 0.5]), np.exp(-b * DCSF), rtol=1e-15)
    # no neurite, no free water: the Standard Model's extra-axonal zeppelin
    der = 0.45
    zep = orc.forward(SMT, b, [0.0, 2.0, DEPAR, der])
    np.testing.assert_allclose(orc.forward(AXCAL, acq, [4.0, 0.0, 0.0, der]), zep, rtol=1e-14)
    # a vanishing radius: the restricted term becomes the stick g(b Da)
    stick = orc.forward(SMT, b, [1.0, DA, 1.0, 0.5])
    np.testing.assert_allclose(orc.forward(AXCAL, acq, [1e-3, 1.0, 0.0, der]), stick, rtol=1e-10)
    # mixture weights
    full = orc.forward(AXCAL, acq, [4.0, 0.3, 0.25, der])
    r = orc.forward(AXCAL, acq, [4.0, 1.0, 0.0, der])
    h = orc.forward(AXCAL, acq, [4.0, 0.0, 0.0, der])
    np.testing.assert_allclose(full, 0.75 * (0.3 * r + 0.7 * h) + 0.25 * np.exp(-b * DCSF), rtol=1e-14)
