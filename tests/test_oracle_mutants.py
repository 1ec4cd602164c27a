"""Plausible mistakes planted in copies of the oracle must fail a pin.

Each case rewrites one line of ``oracle/gac_oracle.c`` in a temporary copy
(never the oracle itself), builds it, and runs the pin that is meant to catch
that kind of mistake.  A pin that still passed would not be pinning anything.
"""
import numpy as np
import pytest

import test_oracle_adapt as A
import test_oracle_axcal as X
import test_oracle_ensemble as E
import test_oracle_fit as F
import test_oracle_models as M
import test_oracle_rng as R
import test_oracle_sampler as S


def _kat(orc):
    for ctr, key, exp in R.KAT:
        R.test_philox_known_answers(orc, ctr, key, exp)


def _g_pins(orc):
    for x in (-10.0, -1.0, 0.5, 7.5):
        M.test_smt_g_against_gauss_legendre(orc, x)


CASES = [
    # (name, old text, new text, pin)
    ("philox output word", "uint32_t n1 = lo1;", "uint32_t n1 = hi1;", _kat),
    ("philox key schedule", "k1 += weyl1;", "k1 += weyl0;", _kat),
    ("philox counter word 3", "uint32_t n2 = hi0 ^ x[3] ^ k1;", "uint32_t n2 = hi0 ^ x[1] ^ k1;", _kat),
    ("uniform offset", "((double)w + 0.5) * 0x1p-32", "((double)w) * 0x1p-32",
     R.test_u01_open_interval_and_exact),
    ("box-muller sin/cos swapped", "z[2 * j] = radius * cos(angle);",
     "z[2 * j] = radius * sin(angle);", R.test_box_muller_radius_and_angle),
    ("acceptance word", "log(orc_u01(w[nw - 1]))", "log(orc_u01(w[0]))",
     S.test_chain_init_and_every_transition),
    ("counter layout", "uint32_t ctr[4] = {t, v, (c << 8) | (uint32_t)k, 0u};",
     "uint32_t ctr[4] = {v, t, (c << 8) | (uint32_t)k, 0u};", R.test_word_layout),
    ("mono-exponential TE units", "exp(-theta[1] * acq[k] * 1e-3)", "exp(-theta[1] * acq[k])",
     M.test_monoexp_closed_form_limits),
    ("3-pool frequency sign", "theta[8] - 2.0 * ORC_PI * df", "theta[8] + 2.0 * ORC_PI * df",
     M.test_mwi3_single_pool_phase_and_modulus),
    ("3-pool EW frequency", "(j < 2) ? theta[6 + j] : 0.0", "theta[6 + (j % 2)]",
     M.test_mwi3_single_pool_phase_and_modulus),
    ("3-pool decay as rate", "exp(-t / theta[3 + j])", "exp(-t * theta[3 + j] * 1e-3)",
     M.test_mwi3_real_when_no_frequency_and_phase),
    ("SMT dropped perpendicular decay", "double extra = exp(-b * dperp) * orc_g(b * (dpar - dperp));",
     "double extra = orc_g(b * (dpar - dperp));", M.test_smt_limits),
    ("SMT series sign", "term *= -x / (double)n;", "term *= x / (double)n;", _g_pins),
    ("SMT erf branch factor", "return sqrt(ORC_PI) * erf(s) / (2.0 * s);",
     "return sqrt(ORC_PI) * erf(s) / s;", _g_pins),
    ("likelihood factor", "return -0.5 * sum;", "return -sum;",
     M.test_loglik_is_gaussian_log_density_up_to_constant),
    ("likelihood sigma", "double r = ((double)y[i] - s[i]) / sigma;",
     "double r = ((double)y[i] - s[i]) / (sigma * sigma);",
     M.test_loglik_zero_at_exact_fit_and_scales_with_sigma),
    ("thinning origin", "int s = (t - B) / T - 1;", "int s = (t - B) / T;",
     S.test_thinning_grid_and_moments),
    ("acceptance sign", "if (log_u < Lp - L)", "if (log_u < L - Lp)",
     S.test_chain_init_and_every_transition),
    ("no clamp", "prop[p] = clampd(theta[p] + m->step[p] * (lambda * z[p]), m->lb[p], m->ub[p]);",
     "prop[p] = theta[p] + m->step[p] * (lambda * z[p]);", S.test_degenerate_runs),
    ("SD divisor n", "sqrt(ss / (double)(n_all - 1))", "sqrt(ss / (double)n_all)",
     S.test_thinning_grid_and_moments),
    ("MH without acceptance test", "if (log_u < Lp - L) {", "if (1) {",
     S.test_linear_gaussian_posterior),
    ("ensemble z exponent", "(double)(P - 1) * log(z)", "(double)P * log(z)", E.test_every_walker_move),
    ("ensemble partner from own half", "int other = (1 - h) * H;", "int other = h * H;",
     E.test_every_walker_move),
    ("ensemble stretch law", "double s = (a - 1.0) * orc_u01(w) + 1.0;",
     "double s = (a - 1.0) * orc_u01(w) + 0.5;", lambda orc: E.test_stretch_distribution(orc, 2.0)),
    ("ensemble prior box ignored", "if (!inside) continue;", "(void)inside;", E.test_every_walker_move),
    ("ensemble stationary law (z^P)", "(double)(P - 1) * log(z)", "(double)P * log(z)",
     E.test_linear_gaussian_posterior),
    ("R-hat chain-mean divisor", "B_over_n /= (C - 1);", "B_over_n /= C;", A.test_rhat_hand_examples),
    ("R-hat within-chain divisor", "W += ss / (n - 1);", "W += ss / n;", A.test_rhat_hand_examples),
    ("adaptation after burn-in", "t <= B && t % o->adapt_window == 0", "t % o->adapt_window == 0",
     lambda orc: A.test_adaptation_when_every_proposal_is_accepted(orc, 100, 10, 10)),
    ("adaptation direction", "if (a > target && e < ORC_ADAPT_EMAX) ++e;",
     "if (a > target && e < ORC_ADAPT_EMAX) --e;",
     lambda orc: A.test_adaptation_when_every_proposal_is_accepted(orc, 100, 10, 10)),
    ("adaptation multiplier", "lambda = exp2(0.25 * (double)e);", "lambda = exp2(0.5 * (double)e);",
     lambda orc: A.test_adaptation_when_every_proposal_is_accepted(orc, 100, 10, 10)),
    ("cylinder radius power", "sum += (r2 * r2 * r2) / (D * D * x2 * x2 * x2 * (x2 - 1.0)) * N;",
     "sum += (r2 * r2) / (D * D * x2 * x2 * x2 * (x2 - 1.0)) * N;", X.test_free_diffusion_bound_and_limit),
    ("cylinder zero factor", "sum += (r2 * r2 * r2) / (D * D * x2 * x2 * x2 * (x2 - 1.0)) * N;",
     "sum += (r2 * r2 * r2) / (D * D * x2 * x2 * x2 * x2) * N;", lambda orc: X.test_wide_pulse_limit(orc, 1.0)),
    ("cylinder pulse-pair sign", "e_minus_one_plus(q * (Delta - delta)) - e_minus_one_plus(q * (Delta + delta));",
     "e_minus_one_plus(q * (Delta - delta)) + e_minus_one_plus(q * (Delta + delta));",
     X.test_free_diffusion_bound_and_limit),
    ("cylinder gradient timing", "double g2 = b / (delta * delta * (Delta - delta / 3.0));",
     "double g2 = b / (delta * delta * Delta);", lambda orc: X.test_wide_pulse_limit(orc, 2.0)),
    ("restricted orientation average", "double restricted = exp(-kap) * orc_g(b * ORC_AX_DA - kap);",
     "double restricted = exp(-kap) * orc_g(b * ORC_AX_DA);",
     X.test_restricted_spherical_mean_against_orientation_quadrature),
    ("free-water diffusivity", "fcsf * exp(-b * ORC_AX_DCSF);", "fcsf * exp(-b * ORC_AX_DA);",
     X.test_compartment_reductions),
    ("Adam second-moment bias correction", "(sqrt(mom2[i] / c2) + o->eps)", "(sqrt(mom2[i]) + o->eps)",
     F.test_adam_first_step_is_lr_against_the_gradient),
    ("TV subgradient sign", "grad[w2 * P + p] += o->lambda / (double)n_mask * sgn(diff);",
     "grad[w2 * P + p] -= o->lambda / (double)n_mask * sgn(diff);",
     lambda orc: F.test_loss_gradient_against_finite_differences(orc, 3, 2, 0.3)),
    ("L1 subgradient", "double drho_ds = (o->loss == 1) ? -w * sgn(r) : -2.0 * w * r;",
     "double drho_ds = (o->loss == 1) ? -w * r : -2.0 * w * r;",
     lambda orc: F.test_loss_gradient_against_finite_differences(orc, 3, 1, 0.0)),
    ("gradient in theta, not u", "grad[v * P + p] *= scale * (m->ub[p] - m->lb[p]); /* d/du */",
     "grad[v * P + p] *= scale; /* d/du */",
     lambda orc: F.test_loss_gradient_against_finite_differences(orc, 1, 2, 0.0)),
    ("SMT Jacobian De_perp", "J[k * P + 3] = -(1.0 - f) * bk * ex * (g_ex + dg_ex);",
     "J[k * P + 3] = -(1.0 - f) * bk * ex * (g_ex - dg_ex);",
     lambda orc: F.test_jacobian_against_finite_differences(orc, 3)),
    ("convergence window start", "o->conv_window > 1 && t >= o->conv_window &&", "o->conv_window > 1 && t > o->conv_window &&",
     F.test_window_slope_and_stopping_rules),
    ("adaptation floor", "if (a < target && e > ORC_ADAPT_EMIN) --e;", "if (a < target) --e;",
     lambda orc: A.test_adaptation_when_every_proposal_is_rejected(orc, 700, -48)),
]


@pytest.mark.parametrize("name,old,new,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(orc, name, old, new, pin):
    src = orc.source()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    so = orc.build_variant(src.replace(old, new), name.replace(" ", "_").replace("/", "_"))
    with orc.variant(so):
        with pytest.raises((AssertionError, ValueError)):
            pin(orc)
    # and the unmodified oracle passes the same pin
    pin(orc)
