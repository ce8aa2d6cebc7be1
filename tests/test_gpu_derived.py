"""GPU tests of the derived features (Sec. 4) and of the moments from given
projections (the tomographic use, Sec. 3.2).

Derived features against the oracle's definitions over the voxels:
|mu_gpu - mu_oracle| <= 1e-9 * muabs (the sum of |V| |x-xbar|^p ...), the
same for eta against muabs / M000^((p+q+r)/3+1), the centroid to 1e-13
relative, and mu' against the spacing powers of Sec. 4.
Moments from projections: images from the CUDA projection and, independently,
from the oracle's projection give the oracle's moments exactly.
"""
import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-9


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


def triples(K):
    return [(p, q, n - p - q) for n in range(K + 1) for p in range(n, -1, -1)
            for q in range(n - p, -1, -1)]


CASES = [
    ((16, 20, 24), np.uint8, 4, "uniform"), ((30, 25, 40), np.uint16, 6, "uniform"),
    ((64, 48, 80), np.uint16, 8, "phantom"), ((20, 22, 24), np.float32, 6, "signed"),
    ((9, 40, 33), np.float32, 8, "uniform"), ((1, 1, 5), np.uint8, 3, "uniform"),
]


def make(shape, dt, kind, seed):
    if kind == "phantom":
        N, M, L = shape
        return synth.ct_phantom_u16(L, M, N, seed=seed, axis_scale=min(shape) / 256)
    if kind == "signed":
        return synth.uniform_volume(shape, dt, seed, low=-1.0, high=1.0)
    return synth.uniform_volume(shape, dt, seed)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_derived_against_oracle(dpma, case):
    shape, dt, K, kind = CASES[case]
    vol = make(shape, dt, kind, 10 + case)
    t, code = dev(vol)
    m = dpma.moments(t, K, code)
    spacing = (1.0, 0.75, 0.4)
    d = dpma.derived_moments(m, K, code, spacing)
    cen, mu, ma = oracle.central_moments(vol, K)
    assert np.allclose(d["centroid"], cen, rtol=1e-13, atol=1e-12)
    assert np.all(np.abs(d["mu"] - mu) <= TOL * ma + 1e-300)
    m0 = mu[0]
    if m0 > 0:
        for j, (p, q, r) in enumerate(triples(K)):
            scale = ma[j] / m0 ** ((p + q + r) / 3 + 1)
            assert abs(d["eta"][j] - mu[j] / m0 ** ((p + q + r) / 3 + 1)) <= TOL * scale + 1e-300
            want = spacing[0] ** (1 + p) * spacing[1] ** (1 + q) * spacing[2] ** (1 + r) * d["mu"][j]
            assert abs(d["mu_phys"][j] - want) <= 1e-14 * abs(want) + 1e-300


def test_derived_of_empty_volume_is_nan(dpma):
    vol = np.zeros((4, 4, 4), dtype=np.uint8)
    t, code = dev(vol)
    m = dpma.moments(t, 3, code)
    d = dpma.derived_moments(m, 3, code)
    assert np.all(np.isnan(d["centroid"])) and np.all(np.isnan(d["mu"]))


def test_derived_rejects_bad_spacing(dpma):
    t, code = dev(synth.uniform_volume((3, 3, 3), np.uint8, seed=1))
    m = dpma.moments(t, 2, code)
    with pytest.raises(dpma.DpmaError):
        dpma.derived_moments(m, 2, code, (1.0, 0.0, 1.0))


@pytest.mark.parametrize("shape,dt,K", [((7, 9, 11), np.uint16, 4), ((20, 3, 33), np.uint8, 8),
                                        ((12, 13, 14), np.uint16, 6), ((5, 6, 7), np.float32, 5)])
def test_moments_from_projections(dpma, shape, dt, K):
    vol = synth.uniform_volume(shape, dt, seed=sum(shape))
    N, M, L = shape
    t, code = dev(vol)
    P = dpma.num_images(K)
    # images from the oracle's own projection, uploaded in the library layout
    imgs = oracle.project(vol, P)
    if dt == np.float32:
        flat = np.concatenate([im.astype(np.float64).ravel() for im in imgs])
        timg = torch.from_numpy(flat).cuda()
    else:
        flat = np.concatenate([im.astype(np.uint32).ravel() for im in imgs])
        timg = torch.from_numpy(flat.view(np.int32)).cuda()
    got = dpma.moments_from_projections(timg, L, M, N, K, code)
    want = oracle.moments(vol, K)
    if dt == np.float32:
        ref = np.asarray(oracle.moments(vol, K, absolute=True))
        assert np.all(np.abs(got - np.asarray(want)) <= 1e-6 * ref)
    else:
        assert got == want
        # and through the CUDA projection
        assert dpma.moments_values(t, K, code) == got
