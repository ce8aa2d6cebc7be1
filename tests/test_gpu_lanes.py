"""GPU parity of the integer-lane projection (volumes with 16-byte aligned rows;
images 0-8, with the in-slice diagonal images 7 and 8 at K = 7, 8).

Integer volumes: images and moments bit for bit against the oracle.  Float32
volumes are quantised onto two int32 limbs and projected exactly; their
moments must satisfy |M_gpu - M_oracle| <= 1e-6 * M_pqr(|V|), and for these
volumes the quantised pipeline itself must have produced them (no fallback).
Volumes with a dynamic range beyond the quantisation grid must take the
compensated fallback and still meet the tolerance.  A bounded device wait
that is made to run out must come back as DPMA_ERR_TIMEOUT.
"""
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


def dev(vol):
    import paper_2012_08099_gb300 as d
    if vol.dtype == np.uint16:
        return torch.from_numpy(vol.view(np.int16)).cuda(), d.U16
    if vol.dtype == np.uint8:
        return torch.from_numpy(vol).cuda(), d.U8
    return torch.from_numpy(vol).cuda(), d.F32


# (N, M, L) with L a multiple of 16: rows are 16-byte aligned for every
# element type.  They span several 64-column tiles and 48/64-row bands,
# ragged in x, y and z, odd and even N (z-pairs), and single slices.
SHAPES = [
    (1, 1, 16), (2, 5, 16), (1, 9, 32), (3, 1, 48), (9, 70, 80), (17, 97, 208),
    (33, 130, 192), (64, 64, 64), (65, 50, 144), (4, 200, 272),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_lane_images_bit_exact(dpma, shape, dtype):
    vol = synth.uniform_volume(shape, dtype, seed=sum(shape) + 17)
    t, dt = dev(vol)
    for K in (2, 3, 4, 5, 6, 7, 8):
        got = dpma.project(t, K, dt)
        want = oracle.project(vol, oracle.num_images(K))
        for k, (g, w) in enumerate(zip(got, want)):
            np.testing.assert_array_equal(g, w, err_msg=f"image {k} K={K} {shape}")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_lane_moments_bit_exact(dpma, shape, dtype):
    vol = synth.uniform_volume(shape, dtype, seed=3 * sum(shape) + 1)
    t, dt = dev(vol)
    for K in range(9):
        assert dpma.moments_values(t, K, dt) == oracle.moments(vol, K), f"K={K} {shape}"


def test_lane_u16_phantom_k6(dpma):
    vol = synth.ct_phantom_u16(96, 80, 50, seed=2, axis_scale=0.4)
    t, dt = dev(vol)
    assert dpma.moments_values(t, 6, dt) == oracle.moments(vol, 6)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["uniform", "signed", "mri"])
def test_lane_float_moments(dpma, shape, kind):
    N, M, L = shape
    if kind == "mri":
        vol = synth.mri_like_f32(L, M, N, seed=sum(shape), n_blobs=6)
    elif kind == "signed":
        vol = synth.uniform_volume(shape, np.float32, sum(shape), low=-1.0, high=1.0)
    else:
        vol = synth.uniform_volume(shape, np.float32, sum(shape))
    t, dt = dev(vol)
    for K in (0, 1, 3, 4, 6, 7, 8):
        got = dpma.moments_values(t, K, dt)
        assert dpma.last_float_path() == 0, f"K={K} {shape} took the fallback"
        want = oracle.moments(vol, K)
        mag = oracle.moments(vol, K, absolute=True)
        err = np.abs(got - want)
        assert np.all(err <= TOL * mag), (K, shape, float(np.max(err / np.maximum(mag, 1e-300))))


def test_lane_float_results_are_deterministic(dpma):
    """The quantised float pipeline sums integers only, so repeated calls on
    the same volume give bit-identical moments (no order-dependent float
    merges), through the synchronous and the asynchronous entry points."""
    vol = synth.mri_like_f32(96, 80, 70, seed=12, n_blobs=8)
    t, dt = dev(vol)
    first = dpma.moments_values(t, 6, dt)
    assert dpma.last_float_path() == 0
    for _ in range(3):
        np.testing.assert_array_equal(dpma.moments_values(t, 6, dt), first)
    out = torch.empty(dpma.num_moments(6), dtype=torch.float64, device="cuda")
    dpma.moments_async(t, 6, out, dt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), first)


def test_lane_float_full_range_goes_to_fallback(dpma):
    """One voxel 2^40 times the rest: the quantisation grid that holds it
    cannot resolve the others within the tolerance, so the compensated
    pipeline recomputes the volume."""
    vol = synth.uniform_volume((20, 40, 64), np.float32, 5, low=0.5, high=1.0)
    vol[7, 11, 13] = 2.0 ** 40
    t, dt = dev(vol)
    got = dpma.moments_values(t, 4, dt)
    assert dpma.last_float_path() != 0
    want = oracle.moments(vol, 4)
    mag = oracle.moments(vol, 4, absolute=True)
    assert np.all(np.abs(got - want) <= TOL * mag)


def test_lane_float_voxel_beyond_sampled_grid(dpma):
    """A hot voxel in a row the magnitude sample skips leaves the grid: the
    range flag sends the volume to the fallback."""
    N, M, L = 64, 128, 64          # 8192 rows: every other row is sampled
    vol = synth.uniform_volume((N, M, L), np.float32, 9, low=0.5, high=1.0)
    rows = M * N
    nsr = 4096
    step = rows // nsr
    sampled = {j * rows // nsr + ((j * 7919) % step if step > 1 else 0) for j in range(nsr)}
    row = next(r for r in range(rows // 2, rows) if r not in sampled)
    vol[row // M, row % M, 5] = 1.0e6
    t, dt = dev(vol)
    got = dpma.moments_values(t, 3, dt)
    assert dpma.last_float_path() & 1
    want = oracle.moments(vol, 3)
    mag = oracle.moments(vol, 3, absolute=True)
    assert np.all(np.abs(got - want) <= TOL * mag)


@pytest.mark.parametrize("dtype", [np.uint16, np.float32])
def test_lane_host_path_in_chunks(dpma, dtype):
    """dpma_moments_host copies the volume in even z-chunks and projects each
    as it lands (the float grid comes from rows sampled over the whole volume
    before the first chunk)."""
    shape = (301, 40, 48)
    if dtype == np.float32:
        vol = synth.mri_like_f32(48, 40, 301, seed=4, n_blobs=5)
    else:
        vol = synth.uniform_volume(shape, dtype, seed=4)
    got = dpma.moments_host(vol, 6)
    if dtype == np.float32:
        assert dpma.last_float_path() == 0
        want = oracle.moments(vol, 6)
        mag = oracle.moments(vol, 6, absolute=True)
        assert np.all(np.abs(np.asarray(got) - want) <= TOL * mag)
    else:
        assert dpma.int128_to_ints(got) == oracle.moments(vol, 6)


def test_lane_host_path_grid_covers_later_chunks(dpma):
    """The host path's quantisation grid is sampled from the whole volume, so
    a volume whose first chunks are faint and whose last ones are 100 times
    brighter stays on the quantised pipeline and meets the tolerance."""
    vol = synth.uniform_volume((301, 40, 48), np.float32, 8, low=0.5, high=1.0)
    vol[200:] *= 100.0
    got = np.asarray(dpma.moments_host(vol, 6))
    assert dpma.last_float_path() == 0
    want = oracle.moments(vol, 6)
    mag = oracle.moments(vol, 6, absolute=True)
    assert np.all(np.abs(got - want) <= TOL * mag)


def test_lane_async_fallback_gate(dpma):
    """dpma_moments_async on a float volume that needs the fallback: the
    gated compensated kernels on the same stream give the right result."""
    vol = synth.uniform_volume((12, 30, 32), np.float32, 21, low=0.5, high=1.0)
    vol[3, 4, 5] = 2.0 ** 40
    t, dt = dev(vol)
    nm = dpma.num_moments(4)
    out = torch.empty(nm, dtype=torch.float64, device="cuda")
    dpma.moments_async(t, 4, out, dt)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = oracle.moments(vol, 4)
    mag = oracle.moments(vol, 4, absolute=True)
    assert np.all(np.abs(got - want) <= TOL * mag)


def test_lane_fallback_graph_repeated_calls(dpma):
    """Repeated dpma_moments_async calls with the same buffers run the
    fallback as a cached graph (gate kernel + conditional body) from the
    second call on.  The buffer's contents alternate between a volume the
    quantised pipeline serves and one that needs the fallback: every result
    must meet the tolerance, so the condition is taken exactly when needed."""
    shape = (12, 30, 32)
    good = synth.uniform_volume(shape, np.float32, 31, low=0.5, high=1.0)
    bad = good.copy()
    bad[3, 4, 5] = 2.0 ** 40
    t = torch.empty(shape, dtype=torch.float32, device="cuda")
    nm = dpma.num_moments(4)
    out = torch.empty(nm, dtype=torch.float64, device="cuda")
    ws = torch.empty(dpma.workspace_size(32, 30, 12, dpma.F32, 4), dtype=torch.uint8,
                     device="cuda")
    want = {}
    for name, v in (("good", good), ("bad", bad)):
        want[name] = (oracle.moments(v, 4), oracle.moments(v, 4, absolute=True))
    for i, name in enumerate(["good", "good", "bad", "good", "bad", "bad", "good"]):
        t.copy_(torch.from_numpy(good if name == "good" else bad))
        dpma.moments_async(t, 4, out, dpma.F32, workspace=ws)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        w, mag = want[name]
        assert np.all(np.abs(got - w) <= TOL * mag), (i, name)


def test_fallback_inside_a_caller_captured_graph(dpma):
    """A float32 call captured by the caller (torch.cuda.graph) holds the
    fallback as a gate kernel and a conditional node.  Replays with contents
    the quantised pipeline serves and contents that need the fallback must
    both meet the tolerance."""
    shape = (12, 30, 32)
    good = synth.uniform_volume(shape, np.float32, 41, low=0.5, high=1.0)
    bad = good.copy()
    bad[5, 6, 7] = 2.0 ** 40
    want = {n: (oracle.moments(v, 4), oracle.moments(v, 4, absolute=True))
            for n, v in (("good", good), ("bad", bad))}
    t = torch.from_numpy(good).cuda()
    out = torch.empty(dpma.num_moments(4), dtype=torch.float64, device="cuda")
    ws = torch.empty(dpma.workspace_size(32, 30, 12, dpma.F32, 4), dtype=torch.uint8,
                     device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dpma.moments_async(t, 4, out, dpma.F32, workspace=ws)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        dpma.moments_async(t, 4, out, dpma.F32, workspace=ws)
    for i, name in enumerate(["bad", "good", "bad", "bad", "good"]):
        t.copy_(torch.from_numpy(good if name == "good" else bad))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        w, mag = want[name]
        assert np.all(np.abs(out.cpu().numpy() - w) <= TOL * mag), (i, name)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float32])
def test_repeated_calls_replay_one_graph(dpma, dtype):
    """From its second call with the same buffers a device-resident pipeline
    is replayed as one cached graph (stage timing off).  The buffer's
    contents change between calls; every result must match the oracle
    (integers bit for bit, float32 within the tolerance)."""
    shape = (21, 37, 48)
    N, M, L = shape
    K = 6
    torch_dt = {np.uint8: torch.uint8, np.uint16: torch.int16, np.float32: torch.float32}[dtype]
    t = torch.empty(shape, dtype=torch_dt, device="cuda")
    dt = {np.uint8: dpma.U8, np.uint16: dpma.U16, np.float32: dpma.F32}[dtype]
    nm = dpma.num_moments(K)
    out = torch.empty(nm * (1 if dtype == np.float32 else 2),
                      dtype=torch.float64 if dtype == np.float32 else torch.int64, device="cuda")
    ws = torch.empty(dpma.workspace_size(L, M, N, dt, K), dtype=torch.uint8, device="cuda")
    for i in range(5):
        vol = synth.uniform_volume(shape, dtype, seed=100 + i)
        t.copy_(torch.from_numpy(vol.view(np.int16) if dtype == np.uint16 else vol))
        dpma.moments_async(t, K, out, dt, workspace=ws)
        torch.cuda.synchronize()
        want = oracle.moments(vol, K)
        if dtype == np.float32:
            mag = oracle.moments(vol, K, absolute=True)
            assert np.all(np.abs(out.cpu().numpy() - want) <= TOL * mag), i
        else:
            assert dpma.int128_to_ints(out.cpu().numpy()) == want, i


@pytest.mark.parametrize("dtype", [np.uint16, np.float32])
def test_bounded_wait_runs_out(dpma, dtype):
    """With a one-cycle wait budget the first pending copy of every CTA is not
    waited for: the kernel lets its copies land, leaves, and the call returns
    DPMA_ERR_TIMEOUT; the default budget then gives exact results again."""
    vol = synth.uniform_volume((40, 96, 128), dtype, seed=6)
    t, dt = dev(vol)
    dpma.set_wait_budget(1)
    try:
        with pytest.raises(dpma.DpmaError) as e:
            dpma.moments(t, 4, dt)
        assert e.value.status == 5
    finally:
        dpma.set_wait_budget(0)
    got = dpma.moments_values(t, 4, dt)
    want = oracle.moments(vol, 4)
    if dtype == np.float32:
        mag = oracle.moments(vol, 4, absolute=True)
        assert np.all(np.abs(got - want) <= TOL * mag)
    else:
        assert got == want
