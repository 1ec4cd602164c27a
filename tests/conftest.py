import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libgac.so")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gac():
    """The CUDA library through its Python binding; no fallback."""
    import torch
    from paper_2511_22094_gb300 import build
    build.build()
    from paper_2511_22094_gb300 import gac as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return g


def make_voxels(orc, w, first=0, n=None):
    """Truths, sigma and noisy float32 data for voxels [first, first+n) of a
    workload; the noise-free signal comes from the oracle's forward model."""
    from paper_2511_22094_gb300 import workloads as W
    th = W.truths(w, first, n)
    sig = W.sigma(w, th)
    y = W.noisy_data(orc.forward(w.kind, w.acq, th), W.noise(w, first, n), sig)
    return th, sig, y
