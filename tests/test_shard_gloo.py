"""Multi-rank path on the CPU: two gloo ranks each sample their voxel shard
(with voxel_base = the shard's first voxel) and gather; the result equals one
run over the whole volume bit for bit, for both the strong and the weak
split.  The oracle stands in for the per-rank sampler (no GPU here)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_22094_gb300 import shard
from paper_2511_22094_gb300 import workloads as W


def test_ranges_partition():
    for n in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            got = [shard.strong_range(n, r, world) for r in range(world)]
            assert sum(c for _, c in got) == n
            assert all(got[i][0] + got[i][1] == got[i + 1][0] for i in range(world - 1))
    assert shard.weak_range(1000, 3) == (3000, 1000)
    with pytest.raises(ValueError):
        shard.strong_range(10, 2, 2)


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


KW = dict(iterations=300, burnin=100, thin=20, n_chains=2, seed=5)


def _inputs(orc, w, first, n):
    th = W.truths(w, first, n)
    sig = W.sigma(w, th)
    return W.noisy_data(orc.forward(w.kind, w.acq, th), W.noise(w, first, n), sig), sig


def _rank(rank, world, port, n_total, mode, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = W.MWI3_1M
    if mode == "strong":
        first, n = shard.strong_range(n_total, rank, world)
    else:
        first, n = shard.weak_range(n_total // world, rank)
    y, sig = _inputs(oracle, w, first, n)
    r = oracle.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, voxel_base=first, n_threads=1, **KW)
    parts = [None] * world
    dist.all_gather_object(parts, (first, r["mean"], r["samples"]))
    if rank == 0:
        parts.sort(key=lambda p: p[0])
        out_q.put((np.concatenate([p[1] for p in parts], 1), np.concatenate([p[2] for p in parts], 3)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["strong", "weak"])
def test_two_rank_shards_reproduce_the_whole_run(orc, mode):
    n_total = 24
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, n_total, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    mean, samples = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = W.MWI3_1M
    y, sig = _inputs(orc, w, 0, n_total)
    whole = orc.mcmc_run(w.kind, w.acq, w.lb, w.ub, w.step, y, sig, **KW)
    np.testing.assert_array_equal(mean, whole["mean"])
    np.testing.assert_array_equal(samples, whole["samples"])
