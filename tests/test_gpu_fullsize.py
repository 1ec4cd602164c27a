"""Full-size runs in the benchmark's launch configuration -- one
gac_mcmc_run over the whole volume, MIXED precision, the workload's chains,
iterations, burn-in and thinning, device buffers -- against the FP64 oracle
on sampled voxels (mcmc.m, Sec. 2.2.2; Table 1 for the AxCaliberSMT run).

The oracle reruns contiguous blocks of sampled voxels -- the first block, one
in the middle, a seeded random one and the ragged end of the volume -- with
voxel_base set to their position, so both sides draw the same random numbers
(the inputs come from the seeded generators and the oracle's forward model).
Sampled outputs: posterior means within 0.05 posterior SD for >= 99% of
(voxel, parameter) pairs and acceptance rates within 0.01 on average; the
reported mean and SD equal those of the stored thinned samples.  Over the
whole volume (properties that hold at any size): no non-finite
log-likelihood, every stored sample and every mean inside the prior box,
SD >= 0, R-hat >= sqrt((n - 1) / n) wherever the within-chain variance is
positive (and not finite only where every chain is constant).  The ensemble
sampler runs at Table 1's settings over 250,000 voxels (the ensemble
benchmark) and is checked on sampled voxels by the paper's independent-seed
design.
"""
import numpy as np
import pytest
import torch

from conftest import make_voxels
from paper_2511_22094_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BLOCK = 16
CASES = [W.MWI3_1M, W.SMT_1P5M, W.AXCAL_250K]


def _blocks(N, seed):
    rng = np.random.default_rng(seed)
    return [0, N // 2 - BLOCK // 2, int(rng.integers(BLOCK, N - 2 * BLOCK)), N - BLOCK]


@pytest.mark.parametrize("w", CASES, ids=[w.name for w in CASES])
def test_full_size_against_oracle_on_sampled_voxels(gac, orc, w):
    N, C, P = w.n_vox, w.n_chains, w.n_par
    I, B, T, S = w.iterations, w.burnin, w.thin, w.n_samples
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, N)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    yd, sd = torch.from_numpy(y).to(dev), torch.from_numpy(sig).to(dev)
    out = dict(mean=torch.empty((P, N), dtype=torch.float64, device=dev),
               std=torch.empty((P, N), dtype=torch.float64, device=dev),
               samples=torch.empty((S, C, P, N), dtype=torch.float32, device=dev),
               accept_rate=torch.empty((C, N), dtype=torch.float32, device=dev),
               nonfinite=torch.empty((C, N), dtype=torch.int32, device=dev),
               rhat=torch.empty((P, N), dtype=torch.float64, device=dev))
    opts = gac.make_opts(I, B, T, C, w.mcmc_seed)
    gac.gac_mcmc_run(mid, yd, N, sd, 0.0, None, opts, out, stream)
    torch.cuda.synchronize()
    del yd, sd

    # whole volume: properties that hold at any size (the FP32 state lives in
    # the float-rounded prior box)
    lb = torch.tensor(np.float32(w.lb).astype(np.float64), device=dev)[:, None]
    ub = torch.tensor(np.float32(w.ub).astype(np.float64), device=dev)[:, None]
    assert int(out["nonfinite"].sum()) == 0
    for s in range(0, S, max(1, S // 8)):  # stored samples inside the box
        smp = out["samples"][s].double()  # [C][P][N]
        assert bool(((smp >= lb[None]) & (smp <= ub[None])).all()), s
    slack = 1e-12 * torch.maximum(lb.abs(), ub.abs())
    assert bool(((out["mean"] >= lb - slack) & (out["mean"] <= ub + slack)).all())
    assert bool((out["std"] >= 0).all())
    n = S * C
    # R-hat >= sqrt((n - 1) / n) where the within-chain variance W > 0; it is
    # not finite only where W = 0: every chain constant over its thinned
    # samples (a parameter that stayed on a clamp bound)
    rh = out["rhat"]
    fin = torch.isfinite(rh)
    assert float(rh[fin].min()) >= np.sqrt((S - 1) / S) * (1 - 1e-9)
    bad = (~fin).nonzero()
    if bad.numel():
        p_idx, v_idx = bad[:, 0], bad[:, 1]
        smp = out["samples"][:, :, p_idx, v_idx]  # [S][C][K]
        assert bool((smp.amax(0) == smp.amin(0)).all())
    print(f"{w.name}: R-hat not finite (W = 0) for {bad.shape[0]} of {rh.numel()} voxel-parameters")
    assert 0.0 < float(out["accept_rate"].mean()) < 1.0

    gaps, acc_g, acc_r = [], [], []
    for v0 in _blocks(N, w.data_seed):
        sl = slice(v0, v0 + BLOCK)
        r = orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y[sl], sig[sl], n_chains=C, iterations=I, burnin=B,
                         thin=T, seed=w.mcmc_seed, voxel_base=v0)
        g_mean = out["mean"][:, sl].cpu().numpy()
        g_std = out["std"][:, sl].cpu().numpy()
        ok = r["std"] > 0
        gaps.append((np.abs(g_mean - r["mean"]) / np.where(ok, r["std"], 1.0))[ok])
        acc_g.append(out["accept_rate"][:, sl].cpu().numpy())
        acc_r.append(r["accept_rate"])
        # the reported moments are those of the stored thinned samples
        smp = out["samples"][:, :, :, sl].double().cpu().numpy()  # [S][C][P][16]
        pooled = smp.transpose(2, 3, 0, 1).reshape(P, BLOCK, n)
        scale = np.abs(pooled).max(-1)
        assert (np.abs(g_mean - pooled.mean(-1)) <= 1e-10 * scale + 1e-300).all(), v0
        assert (np.abs(g_std - pooled.std(-1, ddof=1)) <= 1e-9 * scale + 1e-300).all(), v0
    gap = np.concatenate(gaps)
    dacc = abs(np.mean(np.concatenate(acc_g)) - np.mean(np.concatenate(acc_r)))
    print(f"{w.name} full size: |dmean|/SD median {np.median(gap):.2e} p99 {np.quantile(gap, 0.99):.2e}; "
          f"within 0.05 SD {(gap <= 0.05).mean():.4f}; accept-rate gap {dacc:.4f}")
    assert (gap <= 0.05).mean() >= 0.99
    assert dacc < 0.01


ENS_CASES = [W.MWI3_1M, W.SMT_1P5M]
ENS_BLOCK = 64


@pytest.mark.parametrize("w0", ENS_CASES, ids=[w.name for w in ENS_CASES])
def test_ensemble_full_size_on_sampled_voxels(gac, orc, w0):
    """The ensemble sampler in the benchmark's launch configuration: Table 1's
    50 walkers x 2,000 iterations (burn-in 200, thinning 100) over 250,000
    voxels in one gac_ensemble_run, MIXED, device buffers (the stored samples
    span more than 2^31 floats for the 3-pool model).  Whole volume: no
    non-finite log-likelihood, stored samples and means inside the prior box,
    SD >= 0.  On 512 sampled voxels (the first and last blocks and six seeded
    ones): the reported moments are those of the stored samples, and the
    posterior means agree with the FP64 oracle under independent random
    streams as closely as two oracle runs agree with each other (Demo 2's
    design, Sec. 2.6.2), with the same acceptance rate within 0.01."""
    from test_gpu_precision_study import paired_seed_check

    w = w0.with_(n_vox=250_000, n_chains=50, iterations=2000, burnin=200, thin=100)
    N, L, P = w.n_vox, w.n_chains, w.n_par
    I, B, T = w.iterations, w.burnin, w.thin
    S = gac.n_samples(I, B, T)
    mid = gac.gac_model_register(w.kind, w.acq, w.lb, w.ub, w.step)
    th, sig, y = make_voxels(orc, w, 0, N)
    dev = torch.device("cuda:0")
    out = dict(mean=torch.empty((P, N), dtype=torch.float64, device=dev),
               std=torch.empty((P, N), dtype=torch.float64, device=dev),
               samples=torch.empty((S, L, P, N), dtype=torch.float32, device=dev),
               accept_rate=torch.empty((L, N), dtype=torch.float32, device=dev),
               nonfinite=torch.empty((L, N), dtype=torch.int32, device=dev))
    opts = gac.make_opts(I, B, T, L, w.mcmc_seed)
    gac.gac_ensemble_run(mid, torch.from_numpy(y).to(dev), N, torch.from_numpy(sig).to(dev), 0.0, None, opts,
                         2.0, out, torch.cuda.current_stream())
    torch.cuda.synchronize()

    lb = torch.tensor(np.float32(w.lb).astype(np.float64), device=dev)[:, None]
    ub = torch.tensor(np.float32(w.ub).astype(np.float64), device=dev)[:, None]
    assert int(out["nonfinite"].sum()) == 0
    for s in range(S):  # every stored sample inside the box (walkers reject outside proposals)
        smp = out["samples"][s].double()  # [L][P][N]
        assert bool(((smp >= lb[None]) & (smp <= ub[None])).all()), s
    slack = 1e-12 * torch.maximum(lb.abs(), ub.abs())
    assert bool(((out["mean"] >= lb - slack) & (out["mean"] <= ub + slack)).all())
    assert bool((out["std"] >= 0).all())
    assert 0.0 < float(out["accept_rate"].mean()) < 1.0

    rng = np.random.default_rng(w.data_seed)
    blocks = rng.choice(np.arange(1, N // ENS_BLOCK - 1), 6, replace=False)
    starts = [0, N - ENS_BLOCK] + sorted(int(b) * ENS_BLOCK for b in blocks)
    idx = np.concatenate([np.arange(v0, v0 + ENS_BLOCK) for v0 in starts])
    assert np.unique(idx).size == idx.size == 8 * ENS_BLOCK
    it = torch.from_numpy(idx).to(dev)
    g = {k: out[k].index_select(out[k].dim() - 1, it).cpu().numpy() for k in ("mean", "std", "accept_rate")}
    smp = out["samples"].index_select(3, it).double().cpu().numpy()  # [S][L][P][512]
    del out
    # the reported moments are those of the stored samples, pooled over walkers
    pooled = smp.transpose(2, 3, 0, 1).reshape(P, idx.size, S * L)
    scale = np.abs(pooled).max(-1)
    assert (np.abs(g["mean"] - pooled.mean(-1)) <= 1e-10 * scale + 1e-300).all()
    assert (np.abs(g["std"] - pooled.std(-1, ddof=1)) <= 1e-9 * scale + 1e-300).all()

    kw = dict(iterations=I, burnin=B, thin=T, n_walkers=L, stretch=2.0, want_samples=False)
    runs = {s: orc.ensemble_run(w.kind, w.acq, w.lb, w.ub, y[idx], sig[idx], seed=s, **kw) for s in (11, 22, 44)}
    runs[33] = g
    paired_seed_check(runs, ((11, 22), (33, 44)), f"ensemble {w.name} full size")
    assert abs(g["accept_rate"].mean() - runs[44]["accept_rate"].mean()) < 0.01
