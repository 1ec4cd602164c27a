"""Forward models and log-likelihood on the device against the FP64 oracle.

Tolerances: forward-model relative error <= 1e-5, measured norm-wise per
voxel (||s_gpu - s_ref|| / ||s_ref||, because elementwise relative error is
undefined where a complex component crosses zero); log-likelihood absolute
error <= 1e-3 at posterior-typical parameters (the truth and one-sigma
neighbourhoods of it, where |L| ~ M/2).  The FP64 variant is held to 1e-12
and 1e-8 (AxCaliberSMT: 1e-10 and 1e-7, its FP64 cylinder series stops at
64 terms where the oracle takes 100).
"""
import numpy as np
import pytest

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [W.MONOEXP_4K, W.MWI3_1M, W.SMT_1P5M, W.AXCAL_250K]
FP64_DEFAULT = (1e-12, 1e-8, 1e-12)   # forward, log-likelihood at the truth, relative far from it
FP64_TOL = {W.AXCAL: (1e-10, 1e-7, 1e-9)}


def _edge_thetas(w, rng, n):
    """Random points in the prior box plus its corners and faces."""
    lb, ub = np.array(w.lb), np.array(w.ub)
    th = rng.uniform(lb, ub, size=(n, w.n_par))
    P = w.n_par
    corners = np.array([[lb[p] if (i >> p) & 1 else ub[p] for p in range(P)] for i in range(min(2 ** P, 512))])
    faces = np.repeat(th[:P * 4], 1, axis=0)
    for i in range(faces.shape[0]):
        faces[i, i % P] = lb[i % P] if (i // P) % 2 == 0 else ub[i % P]
    return np.concatenate([th, corners, faces])


@pytest.mark.parametrize("w", CASES, ids=[w.name for w in CASES])
def test_forward_parity(gac, orc, w):
    rng = np.random.default_rng(w.kind)
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th = np.concatenate([W.truths(w, 0, 60_000), _edge_thetas(w, rng, 40_000)])
    ref = orc.forward(w.kind, w.acq, th)
    norm = np.linalg.norm(ref, axis=1)
    keep = norm > 1e-6 * norm.max()  # an all-zero signal (every amplitude 0) has no relative error
    for prec, tol in ((gac.PREC_MIXED, 1e-5), (gac.PREC_FP32, 1e-5),
                      (gac.PREC_FP64, FP64_TOL.get(w.kind, FP64_DEFAULT)[0])):
        s = gac.forward_host(mid, th, prec)
        rel = np.linalg.norm(s - ref, axis=1)[keep] / norm[keep]
        assert rel.max() <= tol, (w.name, prec, rel.max(), np.median(rel))
        assert np.abs(s[~keep] - ref[~keep]).max(initial=0) <= 1e-6


def test_forward_uneven_acquisitions(gac, orc):
    """Unevenly spaced echoes take the direct (non-recurrent) evaluation."""
    te = np.array([1.7, 2.9, 5.5, 6.0, 9.1, 14.0, 20.3, 26.1, 33.3, 40.0])
    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, te, w.lb, w.ub, w.step)
    th = W.truths(w, 0, 20_000)
    ref = orc.forward(w.kind, te, th)
    s = gac.forward_host(mid, th)
    rel = np.linalg.norm(s - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-5
    mono = gac.gac_model_register(1, te, [0.5, 10], [1.5, 80], [0.01, 1])
    th2 = W.truths(W.MONOEXP_4K, 0, 20_000)
    ref2 = orc.forward(1, te, th2)
    s2 = gac.forward_host(mono, th2)
    assert (np.linalg.norm(s2 - ref2, axis=1) / np.linalg.norm(ref2, axis=1)).max() <= 1e-5


def test_smt_g_both_branches(gac, orc):
    """x = b (De_par - De_perp) spans the erfi (x < 0), series/erf switch and
    erf branches; b = 0 gives S = 1 exactly in the FP64 path."""
    w = W.SMT_1P5M
    b = np.array([0.0, 1e-6, 0.1, 1.0, 2.5, 5.0, 7.5, 10.0])
    mid = gac.gac_model_register(w.kind, b, w.lb, w.ub, w.step)
    rng = np.random.default_rng(3)
    n = 50_000
    th = np.stack([rng.uniform(0, 1, n), rng.uniform(1, 3, n), rng.uniform(0.5, 3, n),
                   rng.uniform(0, 1.5, n)], 1)
    th[: n // 2, 3] = np.maximum(th[: n // 2, 3], th[: n // 2, 2])  # De_par <= De_perp
    ref = orc.forward(w.kind, b, th)
    for prec, tol in ((gac.PREC_MIXED, 1e-5), (gac.PREC_FP64, 1e-12)):
        s = gac.forward_host(mid, th, prec)
        rel = np.linalg.norm(s - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert rel.max() <= tol, (prec, rel.max())
        assert np.abs(s[:, 0] - 1.0).max() <= (1e-6 if prec != gac.PREC_FP64 else 1e-15)


def test_g_table_beyond_its_range(gac, orc):
    """b-values large enough that g's argument passes the end of the table:
    those arguments take the asymptote sqrt(pi)/2 x^-1/2 (both models), the
    rest the table."""
    rng = np.random.default_rng(11)
    n = 40_000
    w = W.SMT_1P5M
    b = np.array([0.0, 2.0, 10.0, 20.0, 40.0])
    lb, ub = [0.0, 1.0, 1.25, 0.0], [1.0, 3.0, 3.0, 1.5]  # b (De_par - De_perp) >= -12 at b = 40
    mid = gac.gac_model_register(w.kind, b, lb, ub, w.step)
    th = rng.uniform(lb, ub, (n, w.n_par))
    ref = orc.forward(w.kind, b, th)
    a = W.AXCAL_250K
    acq = np.array([[0.8, 13.0, 6.0], [6.0, 13.0, 6.0], [30.0, 30.0, 6.0], [60.0, 30.0, 6.0]]).ravel()
    mid_a = gac.gac_model_register(a.kind, acq, a.lb, a.ub, a.step)
    th_a = rng.uniform(a.lb, a.ub, (n, a.n_par))
    ref_a = orc.forward(a.kind, acq, th_a)
    for prec in (gac.PREC_MIXED, gac.PREC_FP32):
        for m, t, r in ((mid, th, ref), (mid_a, th_a, ref_a)):
            s = gac.forward_host(m, t, prec)
            rel = np.linalg.norm(s - r, axis=1) / np.linalg.norm(r, axis=1)
            assert rel.max() <= 1e-5, (m, prec, rel.max())


LOGLIK = [(W.MONOEXP_4K, 1e-3), (W.MWI3_1M, 1e-3), (W.SMT_1P5M, 1e-3), (W.AXCAL_250K, 1e-3),
          (W.MWI3_1M.with_(name="mwi3_snr50", snr=50.0), 1e-3),
          (W.MWI3_1M.with_(name="mwi3_snr300", snr=300.0), 1e-3)]


@pytest.mark.parametrize("w,tol", LOGLIK, ids=[c[0].name for c in LOGLIK])
def test_loglik_parity_at_posterior_typical_theta(gac, orc, w, tol):
    """|L_gpu - L_ref| at the true parameters, a typical posterior draw
    (|L| ~ M/2).  The FP32 forward model's error enters L as ~sqrt(M) x
    (relative error) x SNR, so the SNR-300 case is the tight one: the 3-pool
    recurrence in delta form with its double-float set-up keeps the relative
    error near 2.6e-7, i.e. |dL| ~ 5e-4 there (the FP64 path is exact to
    1e-8)."""
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    n = 100_000
    th, sig, y = make_voxels(orc, w, 0, n)
    th = th.astype(np.float32).astype(np.float64)  # the FP32 state holds float parameters
    ref = orc.loglik(w.kind, w.acq, th, y, sig)
    # away from the posterior, errors scale with |L|: check them relatively
    rng = np.random.default_rng(7)
    far = np.clip(th + np.array(w.step) * rng.standard_normal(th.shape), w.lb, w.ub)
    far = far.astype(np.float32).astype(np.float64)
    ref_far = orc.loglik(w.kind, w.acq, far, y, sig)
    res = {}
    _, t64, t64_far = FP64_TOL.get(w.kind, FP64_DEFAULT)
    for prec, t in ((gac.PREC_MIXED, tol), (gac.PREC_FP32, tol), (gac.PREC_FP64, t64)):
        L = gac.loglik_host(mid, th, y, sig, prec)
        err = np.abs(L - ref)
        res[prec] = (err.max(), np.quantile(err, 0.999), np.quantile(err, 0.99))
        assert err.max() <= t, (w.name, prec, res[prec])
        Lf = gac.loglik_host(mid, far, y, sig, prec)
        rel = np.abs(Lf - ref_far) / np.maximum(np.abs(ref_far), 1.0)
        assert rel.max() <= (t64_far if prec == gac.PREC_FP64 else 5e-5), (w.name, prec, rel.max())
    print(w.name, {k: tuple(f"{x:.2e}" for x in v) for k, v in res.items()})


def test_axcal_cylinder_regimes(gac, orc):
    """Axon diameters across the prior box, including the wide cylinders whose
    leading series terms take the Taylor forms (q delta < 1), with Delta =
    delta and Delta >> delta timings, and b = 0."""
    w = W.AXCAL_250K
    acq = np.array([[0.0, 13.0, 6.0], [1.5, 6.0, 6.0], [6.0, 13.0, 6.0], [17.8, 30.0, 6.0],
                    [3.0, 60.0, 4.0], [9.85, 30.0, 6.0]]).ravel()
    mid = gac.gac_model_register(w.kind, acq, w.lb, w.ub, w.step)
    rng = np.random.default_rng(11)
    n = 40_000
    th = np.stack([np.exp(rng.uniform(np.log(0.2), np.log(16.0), n)), rng.uniform(0, 1, n),
                   rng.uniform(0, 1, n), rng.uniform(0.05, 1.7, n)], 1)
    ref = orc.forward(w.kind, acq, th)
    for prec, tol in ((gac.PREC_MIXED, 1e-5), (gac.PREC_FP64, 1e-10)):
        s = gac.forward_host(mid, th, prec)
        rel = np.linalg.norm(s - ref, axis=1) / np.linalg.norm(ref, axis=1)
        print(f"axcal regimes prec={prec}: max {rel.max():.2e} median {np.median(rel):.2e}")
        assert rel.max() <= tol, (prec, rel.max())
        assert np.abs(s[:, 0] - 1.0).max() <= (1e-6 if prec != gac.PREC_FP64 else 1e-15)
