"""The multithreaded CPU DPMA baseline against the oracle.

Integer volumes: every moment bit for bit, K = 0..8, on shapes with single
voxels, single rows/slices and ragged sizes, for several thread counts.
Float32 volumes: within 1e-6 of M_pqr(|V|), including signed values.
"""
import numpy as np
import pytest

import cpu_dpma
import oracle
from paper_2012_08099_gb300 import synth

SHAPES = [(1, 1, 1), (1, 1, 17), (1, 13, 1), (9, 1, 1), (2, 3, 5), (7, 9, 11),
          (16, 5, 33), (31, 18, 7)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_cpu_dpma_integer_exact(shape, dtype):
    vol = synth.uniform_volume(shape, dtype, seed=sum(shape) + 5)
    for K in range(9):
        assert cpu_dpma.moments(vol, K, threads=4) == oracle.moments(vol, K), (K, shape)


def test_cpu_dpma_full_range_u16_k8():
    """All voxels at 65535 on a box with long edges: the largest sums."""
    vol = np.full((40, 3, 300), 65535, dtype=np.uint16)
    assert cpu_dpma.moments(vol, 8) == oracle.moments(vol, 8)


@pytest.mark.parametrize("threads", [1, 2, 3, 7, 64])
def test_cpu_dpma_thread_count_invariant(threads):
    vol = synth.ct_phantom_u16(40, 36, 28, seed=1, axis_scale=0.25)
    got, used = cpu_dpma.moments(vol, 6, threads=threads, return_threads=True)
    assert 1 <= used <= threads
    assert got == oracle.moments(vol, 6)


@pytest.mark.parametrize("kind", ["mri", "signed", "anisotropic"])
def test_cpu_dpma_float_tolerance(kind):
    if kind == "mri":
        vol = synth.mri_like_f32(48, 40, 32, seed=2, n_blobs=5)
    elif kind == "signed":
        vol = synth.uniform_volume((33, 30, 47), np.float32, 8, low=-1.0, high=1.0)
    else:
        vol = synth.uniform_volume((3, 70, 9), np.float32, 9, low=-5.0, high=100.0)
    for K in (0, 2, 4, 6, 8):
        got = cpu_dpma.moments(vol, K)
        want = np.array(oracle.moments(vol, K))
        mag = np.array(oracle.moments(vol, K, absolute=True))
        assert np.all(np.abs(got - want) <= 1e-6 * mag), (kind, K)


def test_cpu_dpma_rejects():
    vol = np.ones((2, 2, 2), np.float32)
    vol[1, 1, 1] = np.nan
    with pytest.raises(cpu_dpma.CpuDpmaError) as e:
        cpu_dpma.moments(vol, 2)
    assert e.value.code == 2
    with pytest.raises(cpu_dpma.CpuDpmaError) as e:
        cpu_dpma.moments(np.ones((2, 2, 2), np.uint8), cpu_dpma.max_order() + 1)
    assert e.value.code == 1


def test_cpu_dpma_image_count():
    """K + 1 images (one for K = 0) reach full rank at every degree up to K."""
    for K in range(cpu_dpma.max_order() + 1):
        assert cpu_dpma.num_images(K) == max(1, K + 1)
