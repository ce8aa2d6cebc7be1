"""Orders 9 and 10 on the GPU (integer volumes): the arctan(1/2) image about
y and the isometric image join the fused projection's images 0-8; images and
moments are compared with the oracle bit for bit.  Volumes whose moments
could leave int128 are refused, float32 volumes and batches stay at K <= 8.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(1, 1, 1), (2, 3, 5), (7, 9, 11), (16, 5, 33), (31, 18, 7), (40, 64, 48), (9, 70, 130)]


@pytest.fixture(scope="module")
def dpma():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_08099_gb300 as d
    d.lib()
    return d


def dev(vol, d):
    if vol.dtype == np.uint16:
        return torch.from_numpy(vol.view(np.int16)).cuda(), d.U16
    return torch.from_numpy(vol).cuda(), d.U8


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_high_order_images_bit_exact(dpma, shape, dtype):
    vol = synth.uniform_volume(shape, dtype, seed=sum(shape) + 90)
    t, dt = dev(vol, dpma)
    got = dpma.project(t, 10, dt)
    want = oracle.project(vol, 11)
    assert len(got) == 11
    for k, (g, w) in enumerate(zip(got, want)):
        np.testing.assert_array_equal(g, w, err_msg=f"image {k} {shape}")


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_high_order_moments_bit_exact(dpma, shape, dtype):
    vol = synth.uniform_volume(shape, dtype, seed=2 * sum(shape) + 3)
    t, dt = dev(vol, dpma)
    for K in (9, 10):
        assert dpma.moments_values(t, K, dt) == oracle.moments(vol, K), (K, shape)


def test_high_order_phantom_and_host_path(dpma):
    vol = synth.ct_phantom_u16(48, 40, 36, seed=5, axis_scale=0.3)
    t, dt = dev(vol, dpma)
    want = oracle.moments(vol, 10)
    assert dpma.moments_values(t, 10, dt) == want
    assert dpma.int128_to_ints(dpma.moments_host(vol, 10)) == want


def test_high_order_binary_mask(dpma):
    """Mostly-zero volumes (the extra images skip zero voxels)."""
    vol = synth.roi_mask_u8(37, 29, 23, 0.4)
    t, dt = dev(vol, dpma)
    assert dpma.moments_values(t, 9, dt) == oracle.moments(vol, 9)


def test_high_order_refusals(dpma):
    big = torch.zeros((512, 512, 512), dtype=torch.int16, device="cuda")
    with pytest.raises(dpma.DpmaError) as e:
        dpma.moments(big, 10, dpma.U16)
    assert e.value.status == 2  # DPMA_ERR_OVERFLOW: moments could leave int128
    f = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(dpma.DpmaError) as e:
        dpma.moments(f, 9, dpma.F32)
    assert e.value.status == 1
    small = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(dpma.DpmaError):
        dpma.moments_batched([small], [9], [dpma.U8])
