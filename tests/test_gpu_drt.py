"""GPU parity of the discrete Radon step 2 (dpma_image_moments_drt).

For integer volumes the 2-D moments it computes from the projection images
must equal, bit for bit, both the power-sum step 2 (dpma_image_moments) and
the oracle's 2-D moments (Eq. 1 summed directly over the oracle's images),
for every order K = 0..10, on ragged shapes (tiles of 16 rows x 1024
columns cut through rows and columns), a CT-like phantom and a binary mask.
"""
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
    return torch.from_numpy(vol).cuda(), d.U8


SHAPES = [(1, 1, 1), (3, 2, 5), (17, 9, 23), (40, 33, 61), (5, 70, 300), (2, 20, 1100)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_drt_equals_power_sums_and_oracle(dpma, shape, dtype):
    vol = synth.uniform_volume(shape, dtype, seed=sum(shape) + 3)
    t, dt = dev(vol)
    for K in range(11):
        try:
            power = dpma.image_moments_of(t, K, dt)
        except dpma.DpmaError as e:
            # orders whose int128 bound the library refuses are refused alike
            assert e.status == 2
            with pytest.raises(dpma.DpmaError):
                dpma.image_moments_drt_of(t, K, dt)
            continue
        drt = dpma.image_moments_drt_of(t, K, dt)
        assert drt == power, (K, shape)
        if K in (0, 4, 10) and vol.size <= 20000:
            imgs = oracle.project(vol, oracle.num_images(K))
            L, M, N = shape[2], shape[1], shape[0]
            for k, img in enumerate(imgs):
                S, F, off_s, off_f = oracle.image_geometry(k, L, M, N)
                want = oracle.image_moments(img, off_s, off_f, K)
                assert drt[k] == list(want), (K, k, shape)


def test_drt_phantom_and_mask(dpma):
    vol = synth.ct_phantom_u16(96, 80, 50, seed=2, axis_scale=0.4)
    t, dt = dev(vol)
    for K in (3, 6, 8):
        assert dpma.image_moments_drt_of(t, K, dt) == dpma.image_moments_of(t, K, dt)
    mask = synth.roi_mask_u8(57, 44, 31, 0.5)
    t, dt = dev(mask)
    assert dpma.image_moments_drt_of(t, 4, dt) == dpma.image_moments_of(t, 4, dt)


def test_drt_status_clear_on_valid_images(dpma):
    vol = synth.uniform_volume((20, 30, 40), np.uint16, seed=9)
    t, dt = dev(vol)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    dpma.image_moments_drt_of(t, 6, dt, status=st)
    assert int(st.item()) == 0


def test_drt_rejects_float(dpma):
    vol = synth.uniform_volume((4, 5, 16), np.float32, seed=1)
    t = torch.from_numpy(vol).cuda()
    with pytest.raises(dpma.DpmaError) as e:
        dpma.image_moments_drt_of(t, 3, dpma.F32)
    assert e.value.status == 1
