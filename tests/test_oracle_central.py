"""Pins of the oracle's centroid and central moments (Sec. 4).

* a constant box: mu_pqr = c * S_p(L) S_q(M) S_r(N) with S_p(n) the 1-D
  power sums about the box centre (separability, exact rationals);
* exact rational brute force on small random volumes (integer and signed
  float32), including the rational centroid;
* a volume mirrored in x has vanishing central moments of odd p;
* translation invariance: embedding the volume in a larger zero box at an
  offset leaves every mu_pqr unchanged and moves the centroid by the offset;
* mu_000 = M_000 and |mu_pqr| <= muabs_pqr.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth

TOL = 1e-12


def triples(K):
    return [(p, q, n - p - q) for n in range(K + 1) for p in range(n, -1, -1)
            for q in range(n - p, -1, -1)]


def exact_central(vol, K):
    N, M, L = vol.shape
    pts = [(Fraction(float(vol[z, y, x])), x, y, z) for z in range(N) for y in range(M)
           for x in range(L) if vol[z, y, x] != 0]
    m0 = sum(v for v, *_ in pts)
    cx = sum(v * x for v, x, y, z in pts) / m0
    cy = sum(v * y for v, x, y, z in pts) / m0
    cz = sum(v * z for v, x, y, z in pts) / m0
    mu = [sum(v * (x - cx) ** p * (y - cy) ** q * (z - cz) ** r for v, x, y, z in pts)
          for p, q, r in triples(K)]
    return (cx, cy, cz), mu


@pytest.mark.parametrize("dims,c", [((5, 4, 3), 7), ((6, 6, 2), 255), ((1, 9, 4), 1000)])
def test_constant_box(dims, c):
    L, M, N = dims
    vol = np.full((N, M, L), c, dtype=np.uint16)
    K = 6

    def S(p, n):
        ctr = Fraction(n - 1, 2)
        return sum((t - ctr) ** p for t in range(n))

    cen, mu, ma = oracle.central_moments(vol, K)
    assert np.allclose(cen, [(L - 1) / 2, (M - 1) / 2, (N - 1) / 2], rtol=0, atol=1e-13)
    for m, (p, q, r) in enumerate(triples(K)):
        want = c * S(p, L) * S(q, M) * S(r, N)
        assert abs(Fraction(mu[m]) - want) <= Fraction(TOL) * Fraction(ma[m]) + Fraction(1, 10**30)


@pytest.mark.parametrize("dtype,seed", [(np.uint8, 1), (np.uint16, 2), (np.float32, 3)])
def test_exact_rational_brute_force(dtype, seed):
    if dtype == np.float32:
        vol = synth.uniform_volume((3, 4, 5), dtype, seed, low=-1.0, high=1.0)
    else:
        vol = synth.uniform_volume((3, 4, 5), dtype, seed)
    K = 5
    (cx, cy, cz), mu_exact = exact_central(vol, K)
    cen, mu, ma = oracle.central_moments(vol, K)
    for got, want in zip(cen, (cx, cy, cz)):
        assert abs(Fraction(got) - want) <= Fraction(1e-14) * max(1, abs(want))
    for m in range(len(mu)):
        assert abs(Fraction(mu[m]) - mu_exact[m]) <= Fraction(TOL) * Fraction(ma[m])


def test_mirror_kills_odd_p():
    half = synth.uniform_volume((6, 7, 5), np.uint16, seed=4)
    vol = np.concatenate([half, half[:, :, ::-1]], axis=2)  # symmetric in x
    K = 6
    cen, mu, ma = oracle.central_moments(vol, K)
    assert abs(cen[0] - (vol.shape[2] - 1) / 2) < 1e-12
    for m, (p, q, r) in enumerate(triples(K)):
        if p % 2 == 1:
            assert abs(mu[m]) <= TOL * ma[m]


def test_translation_invariance():
    vol = synth.uniform_volume((5, 6, 7), np.uint8, seed=5)
    big = np.zeros((11, 9, 20), dtype=np.uint8)
    big[3:8, 2:8, 10:17] = vol
    K = 6
    c1, mu1, ma1 = oracle.central_moments(vol, K)
    c2, mu2, ma2 = oracle.central_moments(big, K)
    assert np.allclose(c2 - c1, [10, 2, 3], rtol=0, atol=1e-12)
    assert np.all(np.abs(mu1 - mu2) <= TOL * ma1 + 1e-300)
    assert np.allclose(ma1, ma2, rtol=1e-12, atol=0)


def test_zeroth_moment_and_bound():
    vol = synth.uniform_volume((4, 4, 4), np.uint16, seed=6)
    cen, mu, ma = oracle.central_moments(vol, 4)
    assert mu[0] == float(vol.astype(np.int64).sum())
    assert np.all(np.abs(mu) <= ma * (1 + 1e-15))
