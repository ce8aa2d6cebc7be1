"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer volumes must match bit for bit (images, 2-D moments, 3-D moments).
Float32 volumes must satisfy, per moment,

    |M_gpu - M_oracle| <= 1e-6 * M_pqr(|V|)

(the oracle's moment of the absolute volume), and per image pixel

    |I_gpu - I_oracle| <= 2^-40 * I_oracle(|V|)

because every float addition of the projection is compensated (Kahan pairs
and error-free TwoSum merges), so an image pixel carries float-float
accuracy; a single plain float32 rounding per pixel (2^-24) would fail it.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FLOAT_MOMENT_TOL = 1e-6
FLOAT_PIXEL_TOL = 2.0 ** -40


@pytest.fixture(scope="module")
def dpma():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_08099_gb300 as d
    d.lib()  # raises if the extension is missing: there is no fallback
    return d


def dev(vol):
    """numpy volume -> (CUDA tensor, library dtype)."""
    import paper_2012_08099_gb300 as d
    if vol.dtype == np.uint16:
        return torch.from_numpy(vol.view(np.int16)).cuda(), d.U16
    if vol.dtype == np.uint8:
        return torch.from_numpy(vol).cuda(), d.U8
    return torch.from_numpy(vol).cuda(), d.F32


def make(shape, dtype, seed, kind="uniform"):
    if kind == "signed":
        return synth.uniform_volume(shape, dtype, seed, low=-1.0, high=1.0)
    return synth.uniform_volume(shape, dtype, seed)


SHAPES = [
    (1, 1, 1), (1, 1, 7), (3, 1, 1), (1, 5, 1), (2, 3, 5), (5, 7, 3), (9, 17, 33),
    (16, 16, 16), (7, 19, 130), (3, 40, 515), (31, 5, 1030), (20, 33, 64),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_images_bit_exact(dpma, shape, dtype):
    vol = make(shape, dtype, seed=sum(shape))
    t, dt = dev(vol)
    for K in (2, 3, 4, 6, 8):
        got = dpma.project(t, K, dt)
        want = oracle.project(vol, oracle.num_images(K))
        for k, (g, w) in enumerate(zip(got, want)):
            assert g.shape == w.shape
            np.testing.assert_array_equal(g, w, err_msg=f"image {k} K={K}")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["uniform", "signed"])
def test_images_float(dpma, shape, kind):
    vol = make(shape, np.float32, seed=3 + sum(shape), kind=kind)
    t, dt = dev(vol)
    K = 8
    got = dpma.project(t, K, dt)
    want = oracle.project(vol, 9)
    mag = oracle.project(np.abs(vol), 9)
    for k in range(9):
        err = np.abs(got[k] - want[k])
        assert np.all(err <= FLOAT_PIXEL_TOL * mag[k] + 1e-30), f"image {k}"


@pytest.mark.parametrize("shape", [(5, 7, 3), (9, 17, 33), (31, 5, 1030), (20, 33, 64)])
def test_image_moments_exact(dpma, shape):
    vol = make(shape, np.uint16, seed=11)
    N, M, L = shape
    t, dt = dev(vol)
    for K in (3, 6, 8):
        got = dpma.image_moments_of(t, K, dt)
        imgs = oracle.project(vol, oracle.num_images(K))
        for k, im in enumerate(imgs):
            S, F, os_, of = oracle.image_geometry(k, L, M, N)
            assert got[k] == oracle.image_moments(im, os_, of, K), f"image {k} K={K}"


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_moments_bit_exact(dpma, shape, dtype):
    vol = make(shape, dtype, seed=7 * sum(shape))
    t, dt = dev(vol)
    for K in range(9):
        assert dpma.moments_values(t, K, dt) == oracle.moments(vol, K), f"K={K}"


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["uniform", "signed"])
def test_moments_float(dpma, shape, kind):
    vol = make(shape, np.float32, seed=5 * sum(shape), kind=kind)
    t, dt = dev(vol)
    for K in (0, 3, 4, 6, 8):
        got = dpma.moments_values(t, K, dt)
        want = oracle.moments(vol, K)
        mag = oracle.moments(vol, K, absolute=True)
        assert np.all(np.abs(got - want) <= FLOAT_MOMENT_TOL * mag), f"K={K}"


def test_config_64cubed_u8_k3(dpma):
    vol = synth.uniform_volume((64, 64, 64), np.uint8, seed=1)
    t, dt = dev(vol)
    assert dpma.moments_values(t, 3, dt) == oracle.moments(vol, 3)


def test_config_256cubed_u16_phantom_k6(dpma):
    vol = synth.ct_phantom_u16(256, 256, 256, seed=2)
    t, dt = dev(vol)
    assert dpma.moments_values(t, 6, dt) == oracle.moments(vol, 6)


def test_config_512cubed_f32_mri_k6(dpma):
    vol = synth.mri_like_f32(512, 512, 512, seed=3)
    t, dt = dev(vol)
    got = dpma.moments_values(t, 6, dt)
    # the bench workload is served by the quantised integer-lane pipeline
    assert dpma.last_float_path() == 0
    want = oracle.moments(vol, 6)
    mag = oracle.moments(vol, 6, absolute=True)
    rel = np.abs(got - want) / mag
    assert rel.max() <= FLOAT_MOMENT_TOL, rel.max()


def test_async_stream_and_workspace(dpma):
    vol = make((33, 20, 70), np.uint16, seed=4)
    t, dt = dev(vol)
    K = 6
    N, M, L = vol.shape
    ws = torch.empty(dpma.workspace_size(L, M, N, dt, K), dtype=torch.uint8, device="cuda")
    out = torch.zeros((dpma.num_moments(K), 2), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dpma.moments_async(t, K, out, dt, stream=s, workspace=ws)
    s.synchronize()
    assert dpma.int128_to_ints(out.cpu().numpy()) == oracle.moments(vol, K)


def test_host_path_matches_device_path(dpma):
    for dtype in (np.uint8, np.uint16, np.float32):
        vol = make((12, 13, 14), dtype, seed=9)
        t, dt = dev(vol)
        K = 4
        host = dpma.moments_host(vol.view(np.int16) if dtype == np.uint16 else vol, K, dt)
        d = dpma.moments(t, K, dt).cpu().numpy()
        if dtype == np.float32:
            # the host path takes its quantisation grid from another sample
            # of rows, so the last bits may differ
            mag = oracle.moments(vol, K, absolute=True)
            assert np.all(np.abs(host - d) <= 1e-12 * mag)
        else:
            np.testing.assert_array_equal(host, d)


@pytest.mark.parametrize("shape,dtype,K", [
    ((256, 256, 256), np.uint16, 6),   # 32 MB: 8 chunks of 32 slices
    ((250, 256, 256), np.uint8, 4),    # 16 MB: 4 chunks of 63 slices (not a multiple of 4)
    ((96, 256, 256), np.float32, 6),   # 24 MB: 6 chunks of 16 slices
    ((37, 200, 300), np.uint16, 8),    # unaligned rows (no bulk copies): chunked too
])
def test_host_path_chunked_matches_device_path(dpma, shape, dtype, K):
    """The host entry point copies z-chunks while earlier chunks are projected;
    the sum over chunks must equal the device-resident result."""
    if dtype == np.float32:
        vol = synth.mri_like_f32(shape[2], shape[1], shape[0], seed=21)
    elif dtype == np.uint16:
        vol = synth.ct_phantom_u16(shape[2], shape[1], shape[0], seed=22)
    else:
        vol = synth.uniform_volume(shape, np.uint8, seed=23)
    t, dt = dev(vol)
    host = dpma.moments_host(vol.view(np.int16) if dtype == np.uint16 else vol, K, dt)
    if dtype == np.float32:
        d = dpma.moments(t, K, dt).cpu().numpy()
        mag = dpma.moments(t.abs(), K, dt).cpu().numpy()
        assert np.all(np.abs(host - d) <= 1e-12 * mag)
    else:
        np.testing.assert_array_equal(host, dpma.moments(t, K, dt).cpu().numpy())


def test_repeat_calls_identical_for_integers(dpma):
    vol = synth.ct_phantom_u16(96, 80, 70, seed=5)
    t, dt = dev(vol)
    a = dpma.moments_values(t, 8, dt)
    b = dpma.moments_values(t, 8, dt)
    assert a == b == oracle.moments(vol, 8)


def test_z_slab_additivity_at_full_size(dpma):
    """Property at any size: M(V) = M(top) + z-shifted M(bottom) (binomial)."""
    from math import comb
    vol = synth.ct_phantom_u16(256, 256, 256, seed=2)
    t, dt = dev(vol)
    K = 6
    whole = dpma.moments_values(t, K, dt)
    h = 100
    lo = dpma.moments_values(t[:h].contiguous(), K, dt)
    hi = dpma.moments_values(t[h:].contiguous(), K, dt)
    idx = {tr: i for i, tr in enumerate(oracle.graded_triples(K))}
    for (p, q, r), i in idx.items():
        shifted = sum(comb(r, k) * h ** (r - k) * hi[idx[(p, q, k)]] for k in range(r + 1))
        assert whole[i] == lo[i] + shifted


@pytest.mark.parametrize("shape,dtype,K,full", [
    ((2, 3, 65536), np.uint16, 4, True),   # x-lines of 65536 voxels at 65535: pixel sums
                                           # 65536 * 65535, the top of the uint32 range
    ((65536, 1, 16), np.uint8, 3, False),  # z-lines of 65536 slices, one row per slice
    ((3, 65536, 16), np.uint16, 4, False), # 65536 rows
    ((2, 2, 65536), np.float32, 4, False), # float32 at the largest dimension
])
def test_largest_dimensions(dpma, shape, dtype, K, full):
    """Maximum sizes: dimensions at the 65536 limit on each axis, and (first
    case) every voxel at the type's maximum, so the longest line sum is
    65536 * 65535 < 2^32: integers bit for bit, float32 within the
    tolerance."""
    if full:
        vol = np.full(shape, np.iinfo(dtype).max, dtype=dtype)
    else:
        vol = make(shape, dtype, seed=sum(shape) % 1000)
    t, dt = dev(vol)
    got = dpma.moments_values(t, K, dt)
    want = oracle.moments(vol, K)
    if dtype == np.float32:
        mag = oracle.moments(vol, K, absolute=True)
        assert np.all(np.abs(got - want) <= FLOAT_MOMENT_TOL * mag)
    else:
        assert got == want


def test_invalid_arguments(dpma):
    t = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(dpma.DpmaError) as e:
        dpma.moments(t, 11)
    assert e.value.status == 1
    big = torch.zeros((1, 1, 1), dtype=torch.int16, device="cuda")
    # 65536^3 voxels of uint16 at K=8 would overflow int128: refused before launch
    rc = dpma.lib().dpma_moments(big.data_ptr(), 65536, 65536, 65536, dpma.U16, 8,
                                 big.data_ptr())
    assert rc == 2


def test_combine_self_check_flags_corrupted_moments(dpma):
    import ctypes
    vol = make((10, 11, 12), np.uint8, seed=6)
    t, dt = dev(vol)
    K = 4
    N, M, L = vol.shape
    P = dpma.num_images(K)
    npairs = (K + 1) * (K + 2) // 2
    lib = dpma.lib()
    imgs = torch.empty(dpma.images_size(L, M, N, dt, K) // 4, dtype=torch.int32, device="cuda")
    m2d = torch.empty(P * npairs * 2, dtype=torch.int64, device="cuda")
    assert lib.dpma_project(t.data_ptr(), L, M, N, dt, K, imgs.data_ptr(), None) == 0
    assert lib.dpma_image_moments(imgs.data_ptr(), L, M, N, dt, K, m2d.data_ptr(), None,
                                  None, 0) == 0
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((dpma.num_moments(K), 2), dtype=torch.int64, device="cuda")
    assert lib.dpma_combine(m2d.data_ptr(), dt, K, out.data_ptr(), None, status.data_ptr()) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert dpma.int128_to_ints(out.cpu().numpy()) == oracle.moments(vol, K)
    # corrupt one selected degree-4 moment whose combine coefficient is not a
    # multiple of D_4: the exact division must then leave a remainder
    D, img, a, C = dpma.combine_plan(K, 4)
    j = next(j for j in range(C.shape[1]) if any(int(c) % D for c in C[:, j]))
    bad = m2d.view(P, npairs, 2).clone()
    bad[img[j], 4 * 5 // 2 + (4 - a[j]), 0] += 1
    assert lib.dpma_combine(bad.data_ptr(), dt, K, out.data_ptr(), None, status.data_ptr()) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 7
