"""The benchmark's multi-process path on CPU: two gloo ranks (world size 2, 127.0.0.1) run the same
host logic that the GPU ranks use under torchrun -- barrier, the max-over-ranks step time, the
whole-job value and the independent problem per rank (replicas only: there is no collective on the
data path)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    dist.barrier()
    ms = 100.0 + 50.0 * rank                      # ranks finish at different times
    mx = bench.max_over_ranks(ms, torch.device("cpu"), world)
    seed = bench.rank_seed(1004, rank)
    inp = synth.make_inputs(3, 4, seed)
    out.put((rank, mx, bench.job_value(5000, 42, world, mx), seed, float(inp.t2.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_independent_problems():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, v0, s0, t0), (r1, mx1, v1, s1, t1) = res
    assert mx0 == mx1 == 150.0                    # the slowest rank's time, on every rank
    assert v0 == v1 == pytest.approx(2 * 5000 * 42 / 0.150)
    assert s0 != s1 and t0 != t1                  # one independent problem per rank


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, 1) == 12.5
    assert bench.job_value(5000, 42, 1, 1000.0) == pytest.approx(210000.0)
