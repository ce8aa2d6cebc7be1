"""The N > 1 path of the benchmark on CPU: world-size-2 ``gloo`` ranks.

The method shards without exchange (independent volumes per GPU), so the
multi-GPU run is replicas only: every rank computes the moments of its own
volume, and the only collectives are the barrier and the max-over-ranks of
the step time.  Here two gloo ranks each run the multithreaded CPU DPMA on
their own seeded volume in place of the GPU step; the test checks that each
replica's moments equal the oracle's for that volume (no data crossed
ranks), that ``bench.max_over_ranks`` returns the slowest rank's time on
every rank, and that ``bench.whole_job_rate`` counts the units of all ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import cpu_dpma
        import oracle
        from paper_2012_08099_gb300 import synth
        vol = synth.uniform_volume((12, 10, 16), np.uint16, seed=100 + rank)
        got = cpu_dpma.moments(vol, 4, threads=2)
        ok = list(got) == list(oracle.moments(vol, 4, nthreads=1))
        # a slower second replica: the job's time is the slowest rank's
        my_ms = 1.0 + rank
        worst = bench.max_over_ranks(my_ms, dist, "cpu")
        rate = bench.whole_job_rate(float(vol.size), world, worst * 1e-3)
        out.put((rank, ok, worst, rate, vol.size))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, ok, worst, rate, nvox in res:
        assert ok, f"rank {rank}: replica moments differ from the oracle"
        assert worst == 2.0
        assert rate == pytest.approx(2 * nvox / 2.0e-3)
