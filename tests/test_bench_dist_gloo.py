"""The benchmark's multi-rank plumbing, as its GPU arm uses it under
torchrun, run with two gloo ranks on the CPU: the rank group from the
environment, the barrier around the timed region, the max-over-ranks time
that every rank gets, the whole-job (weak-scaling) value, and each rank's
disjoint voxel range."""
import importlib.util
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    bench = _load_bench()
    from paper_2511_22094_gb300 import shard
    g = bench.RankGroup("gloo")
    g.barrier(cuda=False)
    t_mine = 1.0 + 0.25 * rank  # this rank's timed region, seconds
    t_max = g.max_time(t_mine, "cpu")
    g.barrier(cuda=False)
    q.put((g.rank, g.world, t_max, bench.weak_value(g.world, 1000, 5, t_max), shard.weak_range(1000, g.rank)))
    g.close()


def test_two_gloo_ranks_time_and_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in got] == [0, 1] and all(r[1] == world for r in got)
    for _, _, t_max, value, _ in got:
        assert t_max == 1.25  # the slowest rank's time, on every rank
        assert value == world * 1000 * 5 / 1.25
    (b0, n0), (b1, n1) = got[0][4], got[1][4]
    assert (b0, n0, b1, n1) == (0, 1000, 1000, 1000)  # disjoint, contiguous voxel ranges


def test_single_process_group_is_a_no_op():
    os.environ.pop("WORLD_SIZE", None)
    bench = _load_bench()
    g = bench.RankGroup("gloo")
    assert g.world == 1 and g.pg is None
    assert g.max_time(3.0, "cpu") == 3.0
    g.barrier(cuda=False)
    g.close()
