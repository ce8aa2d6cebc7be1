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


def _slab_rank(rank: int, world: int, port: int, out):
    """One z-slab of a volume per rank: local moments, shifted to the volume's
    z origin (binomial expansion of (z' + z0)^r), summed over the ranks by
    one collective; rank 0 reports the sum."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from math import comb

        import cpu_dpma
        import oracle
        from paper_2012_08099_gb300 import synth
        vol = synth.uniform_volume((23, 11, 16), np.uint16, seed=7)
        K = 5
        h = 10  # rank 0: z < h, rank 1: z >= h
        z0 = 0 if rank == 0 else h
        slab = vol[:h] if rank == 0 else vol[h:]
        local = list(cpu_dpma.moments(np.ascontiguousarray(slab), K, threads=2))
        idx = {tr: i for i, tr in enumerate(oracle.graded_triples(K))}
        shifted = [0] * len(local)
        for (p, q, r), i in idx.items():
            shifted[i] = sum(comb(r, k) * z0 ** (r - k) * local[idx[(p, q, k)]]
                             for k in range(r + 1))
        parts = [None] * world
        dist.all_gather_object(parts, shifted)
        if rank == 0:
            total = [sum(col) for col in zip(*parts)]
            out.put(total == list(oracle.moments(vol, K, nthreads=1)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_one_volume():
    """The other way the method shards (one large volume cut along z): each
    rank computes its slab, the moments are exact integers, so one sum over
    the ranks gives the volume's moments bit for bit."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    ok = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ok


def _dead_peer_rank(rank: int, world: int, port: int, out):
    """Rank 1 leaves before the collective; rank 0's collective must end with
    an error after the process group's short timeout instead of hanging."""
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(0)  # dies without joining the collective
    t = torch.ones(4)
    try:
        dist.all_reduce(t)
        out.put("completed")
    except Exception as e:  # the dead peer is detected
        out.put("error: " + type(e).__name__)


def test_dead_rank_is_detected_on_the_host():
    """Failure detection without a GPU fault: a rank that dies between steps
    makes the survivor's next collective fail after its timeout."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dead_peer_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert res.startswith("error"), res
