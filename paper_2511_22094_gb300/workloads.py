"""Seeded synthetic workloads shaped like the paper's fitting problems.

This module holds no arithmetic of the sampler or of the forward models.  It
defines each workload's acquisition protocol, prior bounds, proposal steps and
sampler settings, and it draws the random inputs: ground-truth parameters from
the stated uniform ranges, standard-normal noise, and the per-voxel noise level
sigma fixed by the workload's SNR.  Whoever builds measured data evaluates the
forward model at the truths itself and adds ``sigma * noise``
(:func:`noisy_data`).  Both the CUDA path and the FP64 oracle read what this
module draws; neither imports the other.

The in-vivo data of the paper (Sec. 2.6) are not available, so these seeded
volumes stand in for them: protocols and parameter ranges follow the paper's
model list (Sec. 2.1) and speed-test design (Sec. 2.5), and the sampler
settings follow Table 1 (10% burn-in, thinning 100) unless a workload fixes
its own.

Draws are made in blocks of ``BLOCK`` voxels, each from its own
``numpy.random.Generator(PCG64(SeedSequence([seed, stream, block])))``, so that
any voxel range [first, first + n) of a volume is reproducible on its own.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MONOEXP, MWI3, SMT, AXCAL, LINEAR = 1, 2, 3, 4, 100
BLOCK = 65536
_STREAM_TRUTH, _STREAM_NOISE = 1, 2


@dataclass(frozen=True)
class Workload:
    name: str
    kind: int
    acq: tuple            # TE [ms], b [ms/um^2], or (b, Delta, delta) triplets (AxCaliberSMT)
    lb: tuple
    ub: tuple
    step: tuple
    n_vox: int
    n_chains: int
    iterations: int
    burnin: int
    thin: int
    snr: float
    data_seed: int
    mcmc_seed: int
    par_names: tuple = field(default=())

    @property
    def n_par(self) -> int:
        return len(self.lb)

    @property
    def n_meas(self) -> int:
        if self.kind == MWI3:
            return 2 * len(self.acq)
        return len(self.acq) // 3 if self.kind == AXCAL else len(self.acq)

    @property
    def n_samples(self) -> int:
        if self.iterations <= self.burnin:
            return 0
        return (self.iterations - self.burnin) // self.thin

    @property
    def chain_iterations(self) -> int:
        return self.n_vox * self.n_chains * self.iterations

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


_PI = float(np.pi)

#: Mono-exponential R2* decay (Eq. 3): 4,096 voxels, 12 echoes TE = 2:3:35 ms,
#: S0 ~ U(0.5, 1.5), R2* ~ U(10, 80) 1/s, SNR 100, 1 chain, 2,000 iterations,
#: 500 burn-in, thinning 5.
MONOEXP_4K = Workload(
    name="monoexp_4k", kind=MONOEXP, acq=tuple(2.0 + 3.0 * k for k in range(12)),
    lb=(0.5, 10.0), ub=(1.5, 80.0), step=(0.01, 1.0), n_vox=4096, n_chains=1,
    iterations=2000, burnin=500, thin=5, snr=100.0, data_seed=1, mcmc_seed=1001,
    par_names=("S0", "R2star"))

#: 3-pool complex myelin-water GRE model: 1,000,000 voxels, 24 echoes evenly
#: spaced over TE = 2..46 ms, SNR 150, 4 chains, 5,000 iterations, burn-in 10%
#: of the Table 1 setting kept as 500 iterations, thinning 100.
MWI3_1M = Workload(
    name="mwi3_1m", kind=MWI3, acq=tuple(2.0 + k * 44.0 / 23.0 for k in range(24)),
    lb=(0.0, 0.0, 0.0, 3.0, 40.0, 30.0, -10.0, -10.0, -_PI),
    ub=(1.0, 1.0, 1.0, 20.0, 80.0, 60.0, 20.0, 20.0, _PI),
    step=(0.01, 0.01, 0.01, 0.5, 1.0, 1.0, 0.5, 0.5, 0.02), n_vox=1_000_000, n_chains=4,
    iterations=5000, burnin=500, thin=100, snr=150.0, data_seed=2, mcmc_seed=1002,
    par_names=("A_MW", "A_IW", "A_EW", "T2s_MW", "T2s_IW", "T2s_EW", "df_MW", "df_IW", "phi0"))

#: Spherical-mean Standard Model: 1,500,000 voxels, b = {0, 1, 2.5, 5, 7.5, 10}
#: ms/um^2, f ~ U(0,1), Da ~ U(1,3), De_par ~ U(0.5,3), De_perp ~ U(0,1.5),
#: SNR 50, 4 chains, 5,000 iterations, 500 burn-in, thinning 100.
SMT_1P5M = Workload(
    name="smt_1p5m", kind=SMT, acq=(0.0, 1.0, 2.5, 5.0, 7.5, 10.0),
    lb=(0.0, 1.0, 0.5, 0.0), ub=(1.0, 3.0, 3.0, 1.5), step=(0.02, 0.05, 0.05, 0.05),
    n_vox=1_500_000, n_chains=4, iterations=5000, burnin=500, thin=100, snr=50.0,
    data_seed=3, mcmc_seed=1003, par_names=("f", "Da", "De_par", "De_perp"))

#: AxCaliberSMT, the paper's own speed-test model (Sec. 2.5): 250,000 voxels
#: (its largest sample count), the 16 b-values of Supplementary Table S1
#: (8 at Delta = 13 ms, 8 at Delta = 30 ms; pulse width delta = 6 ms, not
#: printed: chosen so that the largest b of each Delta needs 460-500 mT/m,
#: the scanner's gradient limit), SNR 30 at b = 0, and Table 1's MH settings
#: (4 chains x 25,000 iterations, 10% burn-in, thinning 100: 900 samples).
_AX_B13 = (0.05, 0.35, 0.8, 1.5, 2.4, 3.45, 4.75, 6.0)
_AX_B30 = (0.2, 0.95, 2.3, 4.25, 6.75, 9.85, 13.5, 17.8)
AXCAL_250K = Workload(
    name="axcal_250k", kind=AXCAL,
    acq=tuple(x for b in _AX_B13 for x in (b, 13.0, 6.0)) + tuple(x for b in _AX_B30 for x in (b, 30.0, 6.0)),
    lb=(0.2, 0.0, 0.0, 0.05), ub=(16.0, 1.0, 1.0, 1.7), step=(0.4, 0.02, 0.01, 0.04),
    n_vox=250_000, n_chains=4, iterations=25_000, burnin=2_500, thin=100, snr=30.0,
    data_seed=4, mcmc_seed=1004, par_names=("diameter", "f_neurite", "f_csf", "De_R"))

WORKLOADS = {w.name: w for w in (MONOEXP_4K, MWI3_1M, SMT_1P5M, AXCAL_250K)}


def _block_rng(seed: int, stream: int, block: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream, block])))


def _draw(w: Workload, first: int, n: int, stream: int, width: int, fill) -> np.ndarray:
    out = np.empty((n, width), np.float64)
    if n <= 0:
        return out
    for b in range(first // BLOCK, (first + n - 1) // BLOCK + 1):
        blk = fill(_block_rng(w.data_seed, stream, b), BLOCK)
        lo, hi = max(first, b * BLOCK), min(first + n, (b + 1) * BLOCK)
        out[lo - first:hi - first] = blk[lo - b * BLOCK:hi - b * BLOCK]
    return out


def truths(w: Workload, first: int = 0, n: int | None = None) -> np.ndarray:
    """Ground-truth parameters [n][P] (float64) for voxels [first, first+n)."""
    n = w.n_vox - first if n is None else n

    def fill(rng, m):
        if w.kind == MWI3:
            # amplitudes: A_IW, A_EW ~ U(0,1); myelin-water fraction ~ U(0, 0.3)
            a_iw, a_ew = rng.uniform(0.0, 1.0, m), rng.uniform(0.0, 1.0, m)
            mwf = rng.uniform(0.0, 0.3, m)
            a_mw = mwf * (a_iw + a_ew) / (1.0 - mwf)
            rest = [rng.uniform(lo, hi, m) for lo, hi in zip(w.lb[3:], w.ub[3:])]
            return np.stack([a_mw, a_iw, a_ew] + rest, axis=1)
        if w.kind == AXCAL:
            # inside the prior box: diameter ~ U(1, 10) um, f_neurite ~ U(0.3, 0.8),
            # f_csf ~ U(0, 0.2), De_R ~ U(0.3, 1.2) um^2/ms
            return np.stack([rng.uniform(1.0, 10.0, m), rng.uniform(0.3, 0.8, m), rng.uniform(0.0, 0.2, m),
                             rng.uniform(0.3, 1.2, m)], axis=1)
        return np.stack([rng.uniform(lo, hi, m) for lo, hi in zip(w.lb, w.ub)], axis=1)

    return _draw(w, first, n, _STREAM_TRUTH, w.n_par, fill)


def noise(w: Workload, first: int = 0, n: int | None = None) -> np.ndarray:
    """Standard-normal noise [n][M] (float64); complex data use (re, im) pairs."""
    n = w.n_vox - first if n is None else n
    return _draw(w, first, n, _STREAM_NOISE, w.n_meas,
                 lambda rng, m: rng.standard_normal((m, w.n_meas)))


def sigma(w: Workload, theta_true: np.ndarray) -> np.ndarray:
    """Per-voxel noise SD [n] (float32) from the workload's SNR at TE = 0 / b = 0:
    S0/SNR (mono-exponential), (A_MW + A_IW + A_EW)/SNR per real and imaginary
    channel (3-pool), 1/SNR (Standard Model and AxCaliberSMT, signals
    normalised to S(b=0) = 1)."""
    th = np.asarray(theta_true)
    if w.kind == MONOEXP:
        s = th[:, 0] / w.snr
    elif w.kind == MWI3:
        s = th[:, 0:3].sum(axis=1) / w.snr
    else:
        s = np.full(th.shape[0], 1.0 / w.snr)
    return s.astype(np.float32)


def noisy_data(signal: np.ndarray, z: np.ndarray, sig: np.ndarray) -> np.ndarray:
    """Measured data [n][M] float32 = noise-free signal + sigma * z (Gaussian noise)."""
    return (np.asarray(signal, np.float64) + np.asarray(sig, np.float64)[:, None] * z).astype(np.float32)


@dataclass(frozen=True)
class TraceJob:
    index: int
    arrival_s: float
    workload: Workload  # protocol, bounds, steps; n_vox, chains, iterations set per job
    first_voxel: int    # voxels drawn from this offset of the workload's volume


def serving_trace(seed: int = 6, n_jobs: int = 200, mean_interarrival_s: float = 0.2,
                  n_vox_range=(10_000, 2_000_000)) -> list:
    """Serving workload: Poisson arrivals (exponential gaps), each job's model
    drawn uniformly from the three protocols, voxel count log-uniform in
    n_vox_range, 1-4 chains, 1,000-5,000 iterations, burn-in 10% (Table 1),
    thinning 100."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7])))
    gaps = rng.exponential(mean_interarrival_s, n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    kinds = rng.integers(0, 3, n_jobs)
    lo, hi = np.log(n_vox_range[0]), np.log(n_vox_range[1])
    nv = np.exp(rng.uniform(lo, hi, n_jobs)).astype(np.int64)
    chains = rng.integers(1, 5, n_jobs)
    iters = rng.integers(1000, 5001, n_jobs)
    protos = (MONOEXP_4K, MWI3_1M, SMT_1P5M)
    jobs = []
    for i in range(n_jobs):
        base = protos[kinds[i]]
        w = base.with_(name=f"{base.name}-job{i}", n_vox=int(nv[i]), n_chains=int(chains[i]),
                       iterations=int(iters[i]), burnin=int(iters[i]) // 10, thin=100,
                       mcmc_seed=10_000 + i)
        first = int(rng.integers(0, max(1, base.n_vox - int(nv[i])))) if base.n_vox > nv[i] else 0
        jobs.append(TraceJob(i, float(arrivals[i]), w, first))
    return jobs
