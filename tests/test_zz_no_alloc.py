"""The entry point that allocates no device memory, against dpma_moments.

Some callers cannot call cudaMalloc -- their own memory pool already holds
the device memory they may use, or they run a latency-critical loop that
cannot accept cudaMalloc's device-wide synchronisation.  For them
dpma_moments_noalloc keeps its workspace in a static device array.  Called
through the C ABI twice in a row, it must reproduce dpma_moments: exactly
for integer volumes, within the float tolerance of the other GPU tests
(1e-6 of the moment of |V|) for float32 volumes.  This file is collected
last so a failure here leaves every other test already run.  The results
are also compared with the oracle (Eq. 2).
"""
import ctypes

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


@pytest.mark.parametrize("dtype,shape,K", [
    (np.uint8, (64, 64, 64), 3),
    (np.uint16, (33, 20, 70), 6),
    (np.uint16, (17, 9, 130), 8),
    (np.float32, (40, 48, 56), 6),
    (np.float32, (5, 7, 3), 8),
])
def test_noalloc_matches_dpma_moments_twice(dpma, dtype, shape, K):
    vol = synth.uniform_volume(shape, dtype, seed=sum(shape) + K)
    N, M, L = shape
    if dtype == np.uint16:
        t, dt = torch.from_numpy(vol.view(np.int16)).cuda(), dpma.U16
    elif dtype == np.uint8:
        t, dt = torch.from_numpy(vol).cuda(), dpma.U8
    else:
        t, dt = torch.from_numpy(vol).cuda(), dpma.F32
    ref = dpma.moments(t, K, dt).cpu().numpy()
    nm = dpma.num_moments(K)
    lib = dpma.lib()
    for _ in range(2):
        out = torch.full((nm, 2) if dt != dpma.F32 else (nm,), -1,
                         dtype=torch.int64 if dt != dpma.F32 else torch.float64, device="cuda")
        rc = lib.dpma_moments_noalloc(ctypes.c_void_p(t.data_ptr()), L, M, N, dt, K,
                                      ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, lib.dpma_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if dt == dpma.F32:
            mag = oracle.moments(vol, K, absolute=True)
            assert np.all(np.abs(got - ref) <= 1e-6 * mag)
            assert np.all(np.abs(got - oracle.moments(vol, K)) <= 1e-6 * mag)
        else:
            np.testing.assert_array_equal(got, ref)
            # and the definition itself (Eq. 2), bit for bit
            assert dpma.int128_to_ints(got) == oracle.moments(vol, K)


def test_noalloc_refuses_volumes_beyond_its_scratch(dpma):
    lib = dpma.lib()
    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    # 2048^3 at K = 6 needs far more than the 32 MiB static workspace; the
    # call is refused before anything is launched
    rc = lib.dpma_moments_noalloc(ctypes.c_void_p(t.data_ptr()), 2048, 2048, 2048, dpma.U8, 6,
                                  ctypes.c_void_p(t.data_ptr()), None)
    assert rc == 6  # DPMA_ERR_REJECTED
    assert b"static" in lib.dpma_last_error()
