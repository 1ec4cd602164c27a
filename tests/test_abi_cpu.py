"""The C-ABI library loads without a GPU, exports every symbol that
include/gac.h declares, and rejects invalid arguments on the host (no compute
call needs a GPU here)."""
import ctypes as ct
import os
import re
import subprocess

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gac():
    from paper_2511_22094_gb300 import build
    build.build()
    from paper_2511_22094_gb300 import gac as g
    return g


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gac_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(gac):
    declared = _declared()
    assert {"gac_model_register", "gac_mcmc_run", "gac_forward", "gac_loglik"} <= declared
    lib = ct.CDLL(gac.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", gac.LIB_PATH], capture_output=True, text=True)
    if nm.returncode == 0:
        exported = set(re.findall(r"\sT\s(gac_\w+)", nm.stdout))
        assert declared <= exported
    assert set(gac.EXPORTS) <= declared


def test_version(gac):
    assert "sm_103a" in gac.version()


MONO = dict(kind=1, acq=[2.0 + 3 * k for k in range(12)], lb=[0.5, 10.0], ub=[1.5, 80.0],
            step=[0.01, 1.0])


def test_register_and_info(gac):
    mid = gac.gac_model_register(**MONO)
    assert gac.gac_model_info(mid) == (2, 12)
    mid2 = gac.gac_model_register(2, [2.0 + k * 44 / 23 for k in range(24)], [0, 0, 0, 3, 40, 30, -10, -10, -np.pi],
                                  [1, 1, 1, 20, 80, 60, 20, 20, np.pi], [0.01] * 9)
    assert gac.gac_model_info(mid2) == (9, 48)


@pytest.mark.parametrize("bad,status", [
    (dict(kind=7), 2),
    (dict(lb=[0.5, 10.0, 1.0], ub=[1.5, 80.0, 2.0], step=[0.1, 0.1, 0.1]), 1),
    (dict(lb=[1.6, 10.0]), 1),
    (dict(step=[-0.1, 1.0]), 1),
    (dict(acq=[]), 1),
    (dict(acq=[float("nan")] * 12), 1),
    (dict(acq=list(range(65))), 1),
])
def test_register_rejects(gac, bad, status):
    d = dict(MONO)
    d.update(bad)
    with pytest.raises(gac.GacError) as e:
        gac.gac_model_register(**d)
    assert e.value.status == status
    assert gac.last_error()


def test_register_rejects_model_specific_ranges(gac):
    with pytest.raises(gac.GacError):  # T2* lower bound 0
        gac.gac_model_register(2, [2.0, 3.0], [0, 0, 0, 0, 40, 30, -10, -10, -3], [1, 1, 1, 20, 80, 60, 20, 20, 3], [0.01] * 9)
    with pytest.raises(gac.GacError):  # SMT series range exceeded
        gac.gac_model_register(3, [0, 20.0], [0, 1, 0.5, 0], [1, 3, 3, 1.5], [0.02] * 4)
    with pytest.raises(gac.GacError):  # negative b
        gac.gac_model_register(3, [-1.0, 1.0], [0, 1, 0.5, 0], [1, 3, 3, 1.5], [0.02] * 4)


def test_run_argument_validation(gac):
    mid = gac.gac_model_register(**MONO)
    y = np.zeros((4, 12), np.float32)
    out = {}
    cases = [
        dict(iterations=-1), dict(burnin=-1), dict(thin=0), dict(n_chains=0), dict(n_chains=65),
        dict(precision=3), dict(moments_mode=2), dict(trace_n_vox=5),
        dict(adapt_window=-1), dict(adapt_window=10, adapt_target=0.0),
        dict(adapt_window=10, adapt_target=1.0), dict(adapt_window=10, adapt_target=float("nan")),
        dict(lanes_per_chain=-1), dict(lanes_per_chain=3), dict(lanes_per_chain=8),
        # lanes need MIXED precision, no trace, and no more blocks of six echoes than lanes
        dict(lanes_per_chain=2, precision=1), dict(lanes_per_chain=2, precision=2),
    ]
    for c in cases:
        kw = dict(iterations=10, burnin=0, thin=1, n_chains=1, seed=1)
        kw.update(c)
        opts = gac.make_opts(**kw)
        with pytest.raises(gac.GacError) as e:
            gac.gac_mcmc_run(mid, y, 4, None, 0.01, None, opts, out)
        assert e.value.status == 1, c
    opts = gac.make_opts(10, 0, 1, 1, 1)
    with pytest.raises(gac.GacError):  # no sigma and no scalar
        gac.gac_mcmc_run(mid, y, 4, None, 0.0, None, opts, out)
    with pytest.raises(gac.GacError):  # counter word overflow
        gac.gac_mcmc_run(mid, y, 4, None, 0.01, None, gac.make_opts(10, 0, 1, 1, 1, voxel_base=(1 << 32) - 2), out)
    with pytest.raises(gac.GacError) as e:
        gac.gac_mcmc_run(999, y, 4, None, 0.01, None, opts, out)
    assert e.value.status == 2
    with pytest.raises(gac.GacError):  # trace requested without a buffer
        gac.gac_mcmc_run(mid, y, 4, None, 0.01, None, gac.make_opts(10, 0, 1, 1, 1, trace_n_vox=1), out)
    uneven = gac.gac_model_register(**dict(MONO, acq=[1.0, 2.0, 4.0, 8.0] * 3))
    one_block = gac.gac_model_register(**dict(MONO, acq=[2.0, 5.0, 8.0, 11.0]))
    for m in (uneven, one_block):  # lanes split blocks of evenly spaced echoes: 2..4 of them
        with pytest.raises(gac.GacError) as e:
            gac.gac_mcmc_run(m, np.zeros((4, 4), np.float32) if m == one_block else y, 4, None, 0.01, None,
                             gac.make_opts(10, 0, 1, 1, 1, lanes_per_chain=2), out)
        assert e.value.status == 1
    # zero voxels: nothing to do, no GPU needed
    gac.gac_mcmc_run(mid, np.zeros((0, 12), np.float32), 0, None, 0.01, None, opts, out)
    gac.gac_mcmc_run(mid, np.zeros((0, 12), np.float32), 0, None, 0.01, None,
                     gac.make_opts(10, 0, 1, 1, 1, lanes_per_chain=2), out)


def test_result_sizes(gac):
    mid = gac.gac_model_register(**MONO)
    opts = gac.make_opts(2000, 500, 5, 3, 1, trace_n_vox=2)
    b = gac.gac_result_sizes(mid, 100, opts)
    assert b == dict(mean=2 * 100 * 8, std=2 * 100 * 8, samples=300 * 3 * 2 * 100 * 4,
                     accept_rate=3 * 100 * 4, nonfinite=3 * 100 * 4, trace=2 * 3 * 2000 * 216,
                     rhat=2 * 100 * 8, step_scale=3 * 100 * 4)
    b0 = gac.gac_result_sizes(mid, 100, gac.make_opts(400, 500, 5, 1, 1))
    assert b0["samples"] == 0


def test_server_host_side_checks(gac):
    """Creation, budget rejection and bad arguments need no GPU."""
    with pytest.raises(gac.GacError):
        gac.gac_server_create(0, 4)
    with pytest.raises(gac.GacError):
        gac.gac_server_create(1 << 30, 0)
    srv = gac.gac_server_create(1 << 20, 4)  # a 1 MiB budget
    try:
        mid = gac.gac_model_register(**MONO)
        opts = gac.make_opts(100, 10, 10, 2, 1)
        need = gac.gac_server_job_bytes(mid, 100_000, opts, False, True)
        assert need > 1 << 20
        y = np.zeros((100_000, 12), np.float32)
        with pytest.raises(gac.GacError) as e:
            gac.gac_server_submit(srv, mid, y, 100_000, np.ones(100_000, np.float32), 0.0, opts)
        assert e.value.status == 3  # BUDGET
        with pytest.raises(gac.GacError) as e:  # serving runs the MIXED path only
            gac.gac_server_submit(srv, mid, y[:10], 10, None, 0.01, gac.make_opts(100, 10, 10, 2, 1, precision=2))
        assert e.value.status == 1
        with pytest.raises(gac.GacError) as e:
            gac.gac_server_poll(srv, 12345)
        assert e.value.status == 9  # UNKNOWN_JOB
        with pytest.raises(gac.GacError):
            gac.gac_server_cancel(srv, 12345)
        for bad in (-1.0, float("nan")):  # the timeout is checked before the job
            with pytest.raises(gac.GacError) as e:
                gac.gac_server_wait(srv, 12345, bad)
            assert e.value.status == 1
        for ok in (0.0, float("inf")):
            with pytest.raises(gac.GacError) as e:
                gac.gac_server_wait(srv, 12345, ok)
            assert e.value.status == 9
        st = gac.gac_server_get_stats(srv)
        assert st["queued"] == 0 and st["budget"] == 1 << 20
    finally:
        gac.gac_server_destroy(srv)


def test_ensemble_rejects_mh_only_options(gac):
    mid = gac.gac_model_register(**MONO)
    y = np.zeros((4, 12), np.float32)
    for opts, out in ((gac.make_opts(10, 0, 1, 8, 1, adapt_window=5, adapt_target=0.3), {}),
                      (gac.make_opts(10, 0, 1, 8, 1), {"rhat": np.zeros((2, 4))}),
                      (gac.make_opts(10, 0, 1, 8, 1), {"step_scale": np.zeros((8, 4), np.float32)})):
        with pytest.raises(gac.GacError) as e:
            gac.gac_ensemble_run(mid, y, 4, None, 0.01, None, opts, 2.0, out)
        assert e.value.status == 1 and "MH sampler" in gac.last_error()


def test_register_same_description_returns_same_id(gac):
    a = gac.gac_model_register(**MONO)
    b = gac.gac_model_register(**MONO)
    d = dict(MONO)
    d["step"] = [0.02, 1.0]
    c = gac.gac_model_register(**d)
    assert a == b and c != a


def test_fit_argument_validation(gac):
    mid = gac.gac_model_register(**MONO)
    y, th = np.zeros((8, 12), np.float32), np.ones((8, 2))
    for bad in (dict(loss=3), dict(iterations=-1), dict(learning_rate=0.0), dict(beta1=1.0), dict(tv_dims=1),
                dict(convergence_value=1e-3, convergence_window=1), dict(precision=0), dict(tv_lambda=-1.0)):
        with pytest.raises(gac.GacError) as e:
            gac.fit_host(mid, y, th, shape=(2, 2, 2), **bad)
        assert e.value.status == 1, bad
    with pytest.raises(gac.GacError):  # no analytic gradient for AxCaliberSMT
        ax = gac.gac_model_register(4, [1.0, 13.0, 6.0], [0.2, 0, 0, 0.05], [16, 1, 1, 1.7], [0.1] * 4)
        gac.fit_host(ax, np.zeros((8, 1), np.float32), np.ones((8, 4)), shape=(2, 2, 2))
    # a grid of 2^31 / P voxels or more is rejected before any buffer is read
    with pytest.raises(gac.GacError) as e:
        gac.gac_fit_run(mid, y, None, None, gac.make_fit_opts((1 << 10, 1 << 10, 1 << 10), iterations=1), th)
    assert e.value.status == 1
    # zero iterations, or an empty mask: nothing to do, no GPU needed
    th2, hist, done = gac.fit_host(mid, y, th, shape=(2, 2, 2), iterations=0)
    assert done == 0 and (th2 == th).all()
    th3, hist, done = gac.fit_host(mid, y, th, shape=(2, 2, 2), mask=np.zeros(8, np.uint8))
    assert done == 0 and (th3 == th).all()


def test_pipe_probe_rejects_bad_arguments(gac):
    for op in (-1, 11, 99):
        with pytest.raises(gac.GacError) as e:
            gac.gac_pipe_rate(op)
        assert e.value.status == 1
    assert gac._lib.gac_pipe_rate(0, None, None) == 1
    assert set(gac.PIPE_OPS.values()) == set(range(11))


def test_binding_rejects_non_contiguous_buffers(gac):
    a = np.zeros((4, 12), np.float32)
    with pytest.raises(ValueError):
        gac._ptr(a[:, ::2])
    with pytest.raises(ValueError):
        gac._ptr(torch.zeros(4, 12).t())
    assert gac._ptr(a) == a.ctypes.data and gac._ptr(None) is None
