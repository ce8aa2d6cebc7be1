"""GPU tests of the continuous-batching server (``dpma_server_*``).

* every result of a mixed, concurrent stream equals the result of the same
  request served alone (integers bit for bit; float32 within the stated
  tolerance 1e-6 * M_pqr(|V|)), and matches the oracle;
* admission under device-memory pressure: a small arena still serves every
  request, never holding more than it has;
* a request larger than the arena is refused; unknown tickets are reported;
* the counters (p50/p99, volumes/s) are filled in.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-6


@pytest.fixture(scope="module")
def dpma():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_08099_gb300 as d
    d.lib()
    return d


def requests():
    """Mixed sizes (fused and single-volume paths), element types and orders."""
    out = []
    for i, r in enumerate(synth.serving_stream(10, seed=5, xy_range=(32, 160), z_range=(16, 64))):
        out.append((r.volume, r.K))
    for i, (shape, dt, K) in enumerate([
        ((20, 30, 40), np.uint8, 4), ((5, 6, 7), np.uint16, 8), ((64, 64, 64), np.uint8, 3),
        ((17, 33, 300), np.uint16, 6), ((24, 20, 28), np.float32, 6), ((40, 48, 56), np.float32, 4),
        ((1, 1, 1), np.uint8, 0), ((3, 9, 2), np.uint16, 5),
    ]):
        out.append((synth.uniform_volume(shape, dt, seed=50 + i), K))
    return out


def check_close(a, b, vol, K):
    if isinstance(a, np.ndarray):
        ref = np.asarray(oracle.moments(vol, K, absolute=True), dtype=np.float64)
        assert np.all(np.abs(a - b) <= TOL * ref)
    else:
        assert a == b


def test_mixed_stream_equals_alone_and_oracle(dpma):
    reqs = requests()
    with dpma.Server(max_inflight=8, streams=3) as srv:
        alone = []
        for vol, K in reqs:                     # one at a time: nothing else in flight
            alone.append(srv.wait(srv.submit(vol, K)))
        # the same requests, submitted concurrently from 4 threads, 3 times over
        tickets = {}
        lock = threading.Lock()

        def producer(idx):
            for rep in range(3):
                for j in idx:
                    t = srv.submit(reqs[j][0], reqs[j][1])
                    with lock:
                        tickets[(rep, j)] = t

        parts = [list(range(k, len(reqs), 4)) for k in range(4)]
        th = [threading.Thread(target=producer, args=(p,)) for p in parts]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for (rep, j), t in sorted(tickets.items()):
            got = srv.wait(t)
            vol, K = reqs[j]
            check_close(got, alone[j], vol, K)
        st = srv.stats()
        assert st["completed"] == 4 * len(reqs) and st["failed"] == 0
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"] and st["volumes_per_s"] > 0
    for (vol, K), a in zip(reqs, alone):
        want = oracle.moments(vol, K)
        if isinstance(a, np.ndarray):
            ref = np.asarray(oracle.moments(vol, K, absolute=True), dtype=np.float64)
            assert np.all(np.abs(a - np.asarray(want)) <= TOL * ref)
        else:
            assert a == want


def test_admission_under_memory_pressure(dpma):
    vols = [synth.uniform_volume((60, 200, 200), np.uint16, seed=70 + i) for i in range(6)]
    need = vols[0].nbytes + dpma.workspace_size(200, 200, 60, dpma.U16, 6) + 4096
    arena = int(need * 2.5)  # at most two of them fit at once
    with dpma.Server(device_bytes=arena, max_inflight=16, streams=4) as srv:
        ts = [srv.submit(v, 6) for v in vols]
        got = [srv.wait(t) for t in ts]
        st = srv.stats()
        assert st["completed"] == len(vols)
        assert st["device_bytes_peak"] <= arena
        assert st["device_bytes_peak"] < 3 * need
    for v, g in zip(vols[:2], got[:2]):
        t = torch.from_numpy(v.view(np.int16)).cuda()
        assert g == dpma.moments_values(t, 6, dpma.U16)


def test_rejections_and_unknown_tickets(dpma):
    with dpma.Server(device_bytes=1 << 20) as srv:
        big = synth.uniform_volume((128, 128, 256), np.uint8, seed=1)  # 4 MiB > the arena
        with pytest.raises(dpma.DpmaError) as e:
            srv.submit(big, 3)
        assert e.value.status == 6
        assert srv.poll(12345) == -1
        small = synth.uniform_volume((4, 5, 6), np.uint8, seed=2)
        t = srv.submit(small, 3)
        assert srv.wait(t) == oracle.moments(small, 3)
        assert srv.stats()["rejected"] == 1


def test_wait_with_zero_timeout_polls(dpma):
    with dpma.Server() as srv:
        v = synth.uniform_volume((8, 8, 8), np.uint16, seed=3)
        t = srv.submit(v, 4)
        res = None
        for _ in range(100000):
            try:
                res = srv.wait(t, timeout_ms=0)
                break
            except dpma.DpmaError as e:
                assert e.status == 5  # not finished yet
        assert res == oracle.moments(v, 4)


def test_resident_projections_serve_lower_orders(dpma):
    """A keyed volume's images stay resident: requests for the same key at the
    same or a lower order skip the upload and the projection, and their
    results equal a fresh computation."""
    vol = synth.uniform_volume((40, 200, 300), np.uint16, seed=81)   # single-volume path
    t = torch.from_numpy(vol.view(np.int16)).cuda()
    with dpma.Server() as srv:
        first = srv.wait(srv.submit(vol, 8, key=42))
        assert first == dpma.moments_values(t, 8, dpma.U16)
        for K in (6, 4, 8, 0):
            got = srv.wait(srv.submit(vol, K, key=42))
            assert got == dpma.moments_values(t, K, dpma.U16), K
        st = srv.stats()
        assert st["cache_hits"] == 4 and st["resident_volumes"] == 1
        # a higher order than the resident one recomputes and replaces it
        srv2 = None
    with dpma.Server() as srv:
        srv.wait(srv.submit(vol, 3, key=5))
        got = srv.wait(srv.submit(vol, 6, key=5))
        assert got == dpma.moments_values(t, 6, dpma.U16)
        got = srv.wait(srv.submit(vol, 5, key=5))
        assert got == dpma.moments_values(t, 5, dpma.U16)
        st = srv.stats()
        assert st["cache_hits"] == 1 and st["resident_volumes"] == 1


def test_resident_images_are_evicted_under_pressure(dpma):
    vols = [synth.uniform_volume((30, 150, 260), np.uint16, seed=90 + i) for i in range(5)]
    ws = dpma.workspace_size(260, 150, 30, dpma.U16, 6)
    # room for one request in flight plus about two resident image sets
    arena = vols[0].nbytes + ws + 8192 + int(2.5 * ws)
    with dpma.Server(device_bytes=arena) as srv:
        for i, v in enumerate(vols):
            srv.wait(srv.submit(v, 6, key=100 + i))
        st = srv.stats()
        assert 1 <= st["resident_volumes"] < len(vols)  # older ones were evicted
        assert st["device_bytes_peak"] <= arena
        for i, v in enumerate(vols):                     # hits or recomputations: all exact
            t = torch.from_numpy(v.view(np.int16)).cuda()
            assert srv.wait(srv.submit(v, 4, key=100 + i)) == dpma.moments_values(t, 4, dpma.U16)


def test_keyed_float_volumes_are_recomputed(dpma):
    """Float32 images are limbs on the volume's own quantisation grid, so a
    keyed float32 volume keeps no resident images: a second request with the
    same key at a lower order is computed in full and meets the tolerance."""
    vol = synth.mri_like_f32(96, 80, 40, seed=83)
    with dpma.Server() as srv:
        for K in (6, 4, 6):
            got = np.asarray(srv.wait(srv.submit(vol, K, key=77)))
            want = oracle.moments(vol, K)
            mag = oracle.moments(vol, K, absolute=True)
            assert np.all(np.abs(got - want) <= 1e-6 * mag), K
        st = srv.stats()
        assert st["cache_hits"] == 0 and st["resident_volumes"] == 0
