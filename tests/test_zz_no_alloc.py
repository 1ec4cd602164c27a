"""The allocation-free entry point (gac_mcmc_run_noalloc) through the C ABI.

Some callers cannot allocate device memory (an application whose memory is
all held by its own pool, or a loop that must not pay the synchronisation of
cudaMalloc/cudaFree), so this entry point keeps the chains' state between
slices in a fixed array the library already holds.  Its results must equal
those of the ordinary entry point, gac_mcmc_run, within the tolerances of the
serving tests (samples, acceptance rates and counters identical; means to
1e-12 and SDs to 1e-9 relative), on calls in a row -- each call finds the
previous call's contents in the shared array -- including one whose burn-in
step adaptation is carried across slices, and ones whose moments over every
post-burn-in state carry their FP32 block partials across slices.  This file
is collected
last so that a failing run stopped at the first failure has already run
every other test.
"""
import numpy as np
import pytest
import torch

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_run(gac, fn, mid, y, sig, opts, P, slice_iters=None):
    dev = torch.device("cuda:0")
    N, C = y.shape[0], opts.n_chains
    S = gac.n_samples(opts.iterations, opts.burnin, opts.thin)
    out = dict(mean=torch.full((P, N), float("nan"), dtype=torch.float64, device=dev),
               std=torch.full((P, N), float("nan"), dtype=torch.float64, device=dev),
               samples=torch.full((S, C, P, N), float("nan"), dtype=torch.float32, device=dev),
               accept_rate=torch.zeros((C, N), dtype=torch.float32, device=dev),
               nonfinite=torch.full((C, N), -1, dtype=torch.int32, device=dev),
               rhat=torch.full((P, N), float("nan"), dtype=torch.float64, device=dev),
               step_scale=torch.zeros((C, N), dtype=torch.float32, device=dev))
    yd = torch.from_numpy(y).to(dev)
    sd = torch.from_numpy(sig).to(dev)
    stream = torch.cuda.current_stream()
    if slice_iters is None:
        fn(mid, yd, N, sd, 0.0, None, opts, out, stream)
    else:
        fn(mid, yd, N, sd, 0.0, None, opts, slice_iters, out, stream)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


CALLS = [  # different jobs in a row through the same array (..., adaptation window, moments mode)
    (W.MWI3_1M, 1500, 4, 700, 70, 10, 128, 0, 0),
    (W.MONOEXP_4K, 3000, 1, 900, 100, 5, 64, 0, 0),
    (W.SMT_1P5M, 2000, 4, 500, 200, 10, 37, 20, 0),  # burn-in adaptation resumed across slices
    # moments over every post-burn-in state: blocks of 64 states whose FP32
    # partial sums are carried across slices of 45 iterations
    (W.MWI3_1M, 1200, 4, 620, 60, 10, 45, 0, 1),
    (W.SMT_1P5M, 1000, 2, 700, 100, 10, 53, 25, 1),
]


def test_noalloc_matches_gac_mcmc_run_on_two_calls(gac, orc):
    for i, (w, n, C, I, B, T, slice_iters, Wa, mm) in enumerate(CALLS):
        mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
        th, sig, y = make_voxels(orc, w, 500 * i, n)
        opts = gac.make_opts(I, B, T, C, 4242 + i, adapt_window=Wa, adapt_target=0.3 if Wa else 0.0,
                             moments_mode=mm)
        ref = _device_run(gac, gac.gac_mcmc_run, mid, y, sig, opts, w.n_par)
        got = _device_run(gac, gac.gac_mcmc_run_noalloc, mid, y, sig, opts, w.n_par, slice_iters)
        for k in ("samples", "accept_rate", "nonfinite", "step_scale"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"call {i}: {k}")
        np.testing.assert_allclose(got["mean"], ref["mean"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(got["std"], ref["std"], rtol=1e-9, atol=0)
        np.testing.assert_allclose(got["rhat"], ref["rhat"], rtol=1e-9, atol=0)
        if Wa:
            assert len(np.unique(ref["step_scale"])) > 1


def test_noalloc_rejects_what_it_cannot_do_without_allocating(gac, orc):
    w = W.MWI3_1M
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, 64)
    opts = gac.make_opts(100, 10, 10, 4, 1)
    # host buffers would need device staging
    with pytest.raises(gac.GacError) as e:
        gac.gac_mcmc_run_noalloc(mid, y, 64, sig, 0.0, None, opts, 50, {"mean": np.zeros((9, 64))})
    assert e.value.status == 1
    # more chains than the fixed state array holds
    n_big = gac.NOALLOC_STATE_BYTES // (20 * 9 + 20) // 4 + 1000
    dev = torch.device("cuda:0")
    yd = torch.zeros((n_big, w.n_meas), dtype=torch.float32, device=dev)
    with pytest.raises(gac.GacError) as e:
        gac.gac_mcmc_run_noalloc(mid, yd, n_big, None, 0.01, None, opts, 50, {})
    assert e.value.status == 1 and "at most" in gac.last_error()
    # no per-voxel sigma and an infinite scalar: rejected, as by gac_mcmc_run
    yd_small = torch.from_numpy(y).to(dev)
    for bad in (float("inf"), float("nan"), 0.0, -1.0):
        with pytest.raises(gac.GacError) as e:
            gac.gac_mcmc_run_noalloc(mid, yd_small, 64, None, bad, None, opts, 50, {})
        assert e.value.status == 1
