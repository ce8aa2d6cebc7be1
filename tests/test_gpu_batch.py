"""GPU parity of the batched path (``dpma_batch_*``, ``dpma_moments_batched``).

Every volume of a batch must give exactly what the single-volume path gives
(integer volumes bit for bit, float volumes identical because they take that
very path), a sample must match the oracle, a run captured in a CUDA graph
must replay with new volume contents, and the batch of 4096 binary ROI masks
at K = 4 must equal the oracle (Eq. 2) for every ROI.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dpma():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_08099_gb300 as d
    d.lib()
    return d


def dev(vol):
    import paper_2012_08099_gb300 as d
    if vol.dtype == np.uint16:
        return torch.from_numpy(vol.view(np.int16)).cuda(), d.U16
    if vol.dtype == np.uint8:
        return torch.from_numpy(vol).cuda(), d.U8
    return torch.from_numpy(vol).cuda(), d.F32


def mixed_batch():
    """ROI masks plus odd sizes, orders 0..8, 16- and 32-bit pixels, and volumes
    that take the single-volume path (float32, a z-slice over 24 KB)."""
    vols, Ks = [], []
    for v in synth.roi_batch(40, seed=11).volumes:
        vols.append(v)
        Ks.append(4)
    cases = [
        ((20, 30, 40), np.uint16, 3), ((33, 17, 65), np.uint16, 6), ((9, 40, 100), np.uint16, 8),
        ((1, 1, 1), np.uint16, 0), ((2, 3, 1), np.uint8, 2), ((5, 7, 256), np.uint16, 5),
        ((12, 13, 14), np.uint8, 7), ((30, 20, 10), np.uint8, 8), ((64, 64, 64), np.uint8, 4),
        ((300, 4, 4), np.uint8, 4), ((4, 4, 300), np.uint16, 4), ((10, 11, 12), np.float32, 6),
        ((3, 1, 257), np.uint8, 3), ((1, 96, 1), np.uint8, 1), ((3, 100, 300), np.uint16, 4),
        ((7, 3, 255), np.uint8, 6), ((2, 5, 254), np.uint16, 8),
    ]
    for i, (shape, dt, K) in enumerate(cases):
        vols.append(synth.uniform_volume(shape, dt, seed=100 + i))
        Ks.append(K)
    return vols, Ks


def oracle_all(vols, K):
    """oracle.moments(v, K) for every volume, one oracle thread per volume on
    a pool of host threads (the oracle call releases the GIL)."""
    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 4)) as ex:
        return list(ex.map(lambda v: oracle.moments(v, K, nthreads=1), vols))


def single(dpma, t, K, dt):
    return dpma.moments_values(t, K, dt)


def same(a, b):
    if isinstance(a, np.ndarray):
        return np.array_equal(a, b)
    return a == b


def test_batched_matches_single_volume(dpma):
    vols, Ks = mixed_batch()
    tv = [dev(v) for v in vols]
    b = dpma.Batch([t for t, _ in tv], Ks, [d for _, d in tv])
    assert b.info(1) == 2                  # float32 and the 60 KB slices
    assert b.info(0) == len(vols) - 2      # every other volume is fused
    out = b.out_buffer()
    b.run(out)
    b.status()
    got = b.values(out)
    for (t, d), K, g in zip(tv, Ks, got):
        assert same(g, single(dpma, t, K, d)), (tuple(t.shape), K)


def test_batched_matches_oracle(dpma):
    vols, Ks = mixed_batch()
    pick = [0, 7, 39, 40, 41, 42, 45, 46, 47, 48, 50, 52, 55, 56]
    vs = [vols[i] for i in pick]
    ks = [Ks[i] for i in pick]
    tv = [dev(v) for v in vs]
    got = dpma.moments_batched([t for t, _ in tv], ks, [d for _, d in tv])
    for v, K, g in zip(vs, ks, got):
        assert g == oracle.moments(v, K), (v.shape, K)


def test_batch_run_twice_and_reuse(dpma):
    vols, Ks = mixed_batch()
    tv = [dev(v) for v in vols[:20]]
    b = dpma.Batch([t for t, _ in tv], Ks[:20], [d for _, d in tv])
    out1, out2 = b.out_buffer(), b.out_buffer()
    b.run(out1)
    b.run(out2)
    b.status()
    assert torch.equal(out1, out2)


def test_graph_capture_and_replay(dpma):
    vols, Ks = mixed_batch()
    sel = list(range(0, 40, 5)) + [40, 41, 42, 51]   # fused ROIs, u16 volumes, one float
    tv = [dev(vols[i]) for i in sel]
    ks = [Ks[i] for i in sel]
    b = dpma.Batch([t for t, _ in tv], ks, [d for _, d in tv])
    out = b.out_buffer()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(out)                     # warm: kernel attributes and plans set up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(out)
    # new contents in the same buffers, then replay
    for j, (t, d) in enumerate(tv):
        v = vols[sel[j]]
        fresh = synth.uniform_volume(v.shape, v.dtype, seed=900 + j)
        if d == dpma.U8 and v.max() <= 1:
            fresh = (fresh > 127).astype(np.uint8)
        t.copy_(dev(fresh)[0])
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    got = b.values(out)
    for (t, d), K, gv in zip(tv, ks, got):
        assert same(gv, single(dpma, t, K, d)), (tuple(t.shape), K)


def test_autotune_keeps_results(dpma):
    vols, Ks = mixed_batch()
    tv = [dev(v) for v in vols[:40]]
    b = dpma.Batch([t for t, _ in tv], Ks[:40], [d for _, d in tv], autotune=True)
    assert b.info(2) in (256, 512)
    out = b.out_buffer()
    b.run(out)
    b.status()
    for (t, d), K, g in zip(tv, Ks[:40], b.values(out)):
        assert g == single(dpma, t, K, d)


def test_config_4096_roi_masks_k4(dpma):
    """4096 binary ROI masks (sizes log-uniform 8..96), K = 4, one fused launch."""
    rb = synth.roi_batch(4096, seed=4)
    tv = [dev(v) for v in rb.volumes]
    b = dpma.Batch([t for t, _ in tv], [4] * len(tv), [d for _, d in tv])
    assert b.info(0) == 4096 and b.info(1) == 0
    out = b.out_buffer()
    b.run(out)
    b.status()
    got = b.values(out)
    want = oracle_all(rb.volumes, 4)
    for i in range(len(rb.volumes)):
        assert got[i] == want[i], i


def test_footprint_split_matches_single_volume(dpma):
    """ROI masks of mixed sizes: the small-footprint volumes run in a second
    fused launch with two 256-thread CTAs per SM; every result is unchanged."""
    rb = synth.roi_batch(1600, seed=5)
    tv = [dev(v) for v in rb.volumes]
    b = dpma.Batch([t for t, _ in tv], [4] * len(tv), [d for _, d in tv])
    assert b.info(0) == len(tv) and b.info(5) == 2
    assert 0 < b.info(6) < len(tv) and b.info(7) == 256
    out = b.out_buffer()
    b.run(out)
    b.status()
    got = b.values(out)
    want = oracle_all(rb.volumes, 4)
    for i in range(len(tv)):
        assert got[i] == want[i], i
    # all small: one launch of 256-thread CTAs
    sv = synth.roi_batch(64, seed=6, size_range=(8, 24)).volumes
    small = [dev(v) for v in sv]
    bs = dpma.Batch([t for t, _ in small], [3] * len(small), [d for _, d in small])
    assert bs.info(5) == 1 and bs.info(2) == 256
    out = bs.out_buffer()
    bs.run(out)
    bs.status()
    small_want = oracle_all(sv, 3)
    for g, w in zip(bs.values(out), small_want):
        assert g == w


def test_two_cta_launch_every_order(dpma):
    """Small volumes only: one fused launch of 256-thread CTAs, two per SM,
    through every order 0..8, 16- and 32-bit pixels, int64 and int128 row
    sums (the (4, 8, 40) u16 volume at K = 8 needs int128)."""
    cases = [((4, 8, 40), np.uint16, 8), ((6, 10, 12), np.uint16, 8), ((5, 7, 9), np.uint8, 7),
             ((3, 30, 20), np.uint16, 6), ((8, 8, 8), np.uint8, 5), ((2, 3, 50), np.uint16, 4),
             ((7, 5, 3), np.uint8, 3), ((1, 1, 1), np.uint16, 0), ((2, 2, 2), np.uint8, 1),
             ((3, 4, 5), np.uint16, 2), ((9, 13, 17), np.uint8, 8)]
    tv = [dev(synth.uniform_volume(sh, dt, seed=300 + i)) for i, (sh, dt, _) in enumerate(cases)]
    Ks = [K for _, _, K in cases]
    b = dpma.Batch([t for t, _ in tv], Ks, [d for _, d in tv])
    assert b.info(0) == len(tv) and b.info(5) == 1 and b.info(2) == 256
    out = b.out_buffer()
    b.run(out)
    b.status()
    for (t, d), K, g in zip(tv, Ks, b.values(out)):
        assert g == single(dpma, t, K, d), (tuple(t.shape), K)


def test_batch_rejects_bad_descriptors(dpma):
    t, d = dev(synth.uniform_volume((4, 4, 4), np.uint8, seed=1))
    with pytest.raises(dpma.DpmaError) as e:
        dpma.Batch([t], [9], [d])
    assert e.value.status == 1
    with pytest.raises(dpma.DpmaError) as e:
        dpma.Batch([t], [3], [7])
    assert e.value.status == 1
