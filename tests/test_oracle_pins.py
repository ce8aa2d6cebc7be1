"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test fixes the oracle to something other than itself: a closed form
(Faulhaber power sums for a constant box), a single voxel, a separable
volume (products of 1-D moments), pure-Python brute force on tiny volumes,
exact rational arithmetic for float32 inputs, and invariants of Eq. 2
(linearity, axis permutation, mirror and translation as binomial shifts,
additivity over z-slabs).
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth


# ----------------------------------------------------------------------
# independent reference quantities


def bernoulli(m: int) -> list[Fraction]:
    """B_0..B_m with B_1 = -1/2 (from sum_{j<=k} C(k+1, j) B_j = 0)."""
    B = [Fraction(1)]
    for k in range(1, m + 1):
        B.append(-sum(comb(k + 1, j) * B[j] for j in range(k)) / (k + 1))
    return B


def faulhaber(p: int, n: int) -> int:
    """sum_{t=0}^{n-1} t^p in closed form (with 0^0 = 1)."""
    B = bernoulli(p)
    s = sum(comb(p + 1, j) * B[j] * Fraction(n) ** (p + 1 - j) for j in range(p + 1))
    s /= p + 1
    assert s.denominator == 1
    return int(s)


def brute_moments(vol, K):
    """Pure-Python sum of Eq. 2 over a tiny volume (Python ints / Fractions)."""
    N, M, L = vol.shape
    out = []
    for p, q, r in oracle.graded_triples(K):
        s = 0
        for z in range(N):
            for y in range(M):
                for x in range(L):
                    v = vol[z, y, x]
                    v = Fraction(float(v)) if vol.dtype == np.float32 else int(v)
                    s += v * x ** p * y ** q * z ** r
        out.append(s)
    return out


def idx(K):
    return {t: i for i, t in enumerate(oracle.graded_triples(K))}


# ----------------------------------------------------------------------


def test_faulhaber_reference_itself():
    # the closed form against direct sums (pins the pin)
    for p in range(11):
        for n in (1, 2, 7, 30):
            assert faulhaber(p, n) == sum(t ** p for t in range(n))


def test_graded_order():
    assert oracle.graded_triples(2) == [
        (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1),
        (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for K, n in ((3, 20), (4, 35), (6, 84), (8, 165)):
        assert oracle.num_moments(K) == n == len(oracle.graded_triples(K))


@pytest.mark.parametrize("dtype,c", [(np.uint8, 255), (np.uint16, 4095), (np.uint16, 65535)])
@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 7, 3), (16, 9, 33)])
def test_constant_box_closed_form(dtype, c, shape):
    N, M, L = shape
    vol = np.full(shape, c, dtype=dtype)
    K = 8
    got = oracle.moments(vol, K, nthreads=3)
    for (p, q, r), g in zip(oracle.graded_triples(K), got):
        assert g == c * faulhaber(p, L) * faulhaber(q, M) * faulhaber(r, N), (p, q, r)


def test_constant_box_float_closed_form():
    N, M, L = 6, 5, 9
    c = 0.375
    vol = np.full((N, M, L), c, dtype=np.float32)
    got = oracle.moments(vol, 6, nthreads=2)
    for (p, q, r), g in zip(oracle.graded_triples(6), got):
        want = c * faulhaber(p, L) * faulhaber(q, M) * faulhaber(r, N)
        assert g == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("pos", [(0, 0, 0), (12, 0, 0), (0, 9, 0), (0, 0, 7), (12, 9, 7), (5, 3, 2)])
def test_single_voxel(pos):
    x0, y0, z0 = pos
    vol = np.zeros((8, 10, 13), dtype=np.uint16)
    vol[z0, y0, x0] = 4093
    got = oracle.moments(vol, 8, nthreads=2)
    for (p, q, r), g in zip(oracle.graded_triples(8), got):
        assert g == 4093 * x0 ** p * y0 ** q * z0 ** r


def test_separable_volume():
    g = np.random.Generator(np.random.PCG64(11))
    fx = g.integers(0, 16, size=11)
    fy = g.integers(0, 16, size=6)
    fz = g.integers(0, 16, size=9)
    vol = (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]).astype(np.uint16)
    K = 6
    got = oracle.moments(vol, K, nthreads=4)

    def m1(f, p):
        return sum(int(f[t]) * t ** p for t in range(len(f)))

    for (p, q, r), v in zip(oracle.graded_triples(K), got):
        assert v == m1(fx, p) * m1(fy, q) * m1(fz, r)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_4cubed(seed):
    vol = synth.uniform_volume((4, 4, 4), np.uint8, seed=100 + seed)
    assert oracle.moments(vol, 5, nthreads=1) == brute_moments(vol, 5)
    vol16 = synth.uniform_volume((4, 3, 5), np.uint16, seed=200 + seed)
    assert oracle.moments(vol16, 4, nthreads=2) == brute_moments(vol16, 4)


def test_exhaustive_binary_2cubed():
    K = 4
    for bits in range(256):
        vol = np.array([(bits >> i) & 1 for i in range(8)], dtype=np.uint8).reshape(2, 2, 2)
        assert oracle.moments(vol, K, nthreads=1) == brute_moments(vol, K), bits


@pytest.mark.parametrize("signed", [False, True])
def test_float_against_exact_rationals(signed):
    vol = synth.uniform_volume((4, 5, 6), np.float32, seed=7,
                               low=-1.0 if signed else 0.0, high=1.0 if signed else 1000.0)
    K = 6
    got = oracle.moments(vol, K, nthreads=2)
    ref_abs = oracle.moments(vol, K, nthreads=2, absolute=True)
    exact = brute_moments(vol, K)
    for g, e, a in zip(got, exact, ref_abs):
        # FP64 with compensation: a few ulps of the magnitude
        assert abs(Fraction(g) - e) <= Fraction(1e-14) * Fraction(a) + Fraction(1e-300)


def test_float_abs_moments_are_moments_of_abs():
    vol = synth.uniform_volume((3, 4, 5), np.float32, seed=8, low=-1.0, high=1.0)
    a = oracle.moments(vol, 4, absolute=True)
    b = oracle.moments(np.abs(vol), 4)
    np.testing.assert_array_equal(a, b)


def test_linearity():
    v = synth.uniform_volume((7, 6, 9), np.uint16, seed=3, high=1000)
    w = synth.uniform_volume((7, 6, 9), np.uint16, seed=4, high=1000)
    K = 6
    mv, mw = oracle.moments(v, K), oracle.moments(w, K)
    mc = oracle.moments((3 * v + 5 * w).astype(np.uint16), K)
    assert mc == [3 * a + 5 * b for a, b in zip(mv, mw)]


def test_axis_permutation():
    vol = synth.uniform_volume((5, 6, 7), np.uint8, seed=5)
    K = 5
    m = oracle.moments(vol, K)
    I = idx(K)
    # swap x and y: V'[z, x, y] = V[z, y, x]
    mt = oracle.moments(np.ascontiguousarray(vol.transpose(0, 2, 1)), K)
    # cycle: V''[x, z, y] holds (x', y', z') = (y, z, x)
    mc = oracle.moments(np.ascontiguousarray(vol.transpose(2, 0, 1)), K)
    for (p, q, r), i in I.items():
        assert mt[i] == m[I[(q, p, r)]]
        assert mc[i] == m[I[(r, p, q)]]


def test_mirror_is_binomial():
    vol = synth.uniform_volume((4, 5, 6), np.uint16, seed=6)
    N, M, L = vol.shape
    K = 6
    m = oracle.moments(vol, K)
    mm = oracle.moments(np.ascontiguousarray(vol[:, :, ::-1]), K)
    I = idx(K)
    for (p, q, r), i in I.items():
        # x -> (L-1) - x
        want = sum(comb(p, k) * (L - 1) ** (p - k) * (-1) ** k * m[I[(k, q, r)]] for k in range(p + 1))
        assert mm[i] == want


def test_translation_is_binomial():
    vol = synth.uniform_volume((4, 5, 6), np.uint8, seed=9)
    K = 6
    t = 3
    padded = np.zeros((4 + t, 5, 6), dtype=np.uint8)
    padded[t:] = vol  # z -> z + t
    m = oracle.moments(vol, K)
    mp = oracle.moments(padded, K)
    I = idx(K)
    for (p, q, r), i in I.items():
        want = sum(comb(r, k) * t ** (r - k) * m[I[(p, q, k)]] for k in range(r + 1))
        assert mp[i] == want


def test_slab_additivity():
    vol = synth.uniform_volume((11, 5, 6), np.uint16, seed=10)
    K = 4
    whole = oracle.moments(vol, K, nthreads=1)
    a = np.zeros_like(vol)
    b = np.zeros_like(vol)
    a[:6] = vol[:6]
    b[6:] = vol[6:]
    assert whole == [x + y for x, y in zip(oracle.moments(a, K), oracle.moments(b, K))]
    # thread count does not change exact results
    assert whole == oracle.moments(vol, K, nthreads=5)


def test_int128_overflow_is_detected():
    vol = np.zeros((1, 1, 32768), dtype=np.uint16)
    vol[0, 0, 32767] = 65535  # 65535 * 32767^8 > 2^127
    with pytest.raises(OverflowError):
        oracle.moments(vol, 8)
    assert oracle.moments(vol, 7)[oracle.graded_triples(7).index((7, 0, 0))] == 65535 * 32767 ** 7


def test_bad_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.moments(np.zeros((2, 2, 2), np.uint8), 11)
    with pytest.raises(TypeError):
        oracle.moments(np.zeros((2, 2, 2), np.int32), 3)


def test_golden_small_volumes():
    """Fixture written by tests/golden/make_golden.py (oracle only)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "small_volumes.json")
    with open(path) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        dt = np.uint8 if c["dtype"] == "u8" else np.uint16
        vol = synth.uniform_volume(tuple(c["shape_zyx"]), dt, seed=c["seed"])
        assert oracle.moments(vol, c["K"]) == [int(v) for v in c["moments"]]
        assert brute_moments(vol, min(c["K"], 3)) == [int(v) for v in c["moments"]][:oracle.num_moments(min(c["K"], 3))]


# ----------------------------------------------------------------------
# orders 9 and 10


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 7, 3), (16, 9, 33)])
def test_constant_box_closed_form_k10(shape):
    N, M, L = shape
    vol = np.full(shape, 65535, dtype=np.uint16)
    got = oracle.moments(vol, 10, nthreads=3)
    for (p, q, r), g in zip(oracle.graded_triples(10), got):
        assert g == 65535 * faulhaber(p, L) * faulhaber(q, M) * faulhaber(r, N), (p, q, r)


@pytest.mark.parametrize("pos", [(0, 0, 0), (12, 9, 7), (5, 3, 2)])
def test_single_voxel_k10(pos):
    x0, y0, z0 = pos
    vol = np.zeros((8, 10, 13), dtype=np.uint8)
    vol[z0, y0, x0] = 251
    got = oracle.moments(vol, 10, nthreads=2)
    for (p, q, r), g in zip(oracle.graded_triples(10), got):
        assert g == 251 * x0 ** p * y0 ** q * z0 ** r


@pytest.mark.parametrize("seed", range(2))
def test_brute_force_k10(seed):
    vol = synth.uniform_volume((3, 4, 5), np.uint16, seed=300 + seed)
    assert oracle.moments(vol, 10, nthreads=2) == brute_moments(vol, 10)


def test_float_k10_against_exact_rationals():
    vol = synth.uniform_volume((3, 4, 5), np.float32, 41, low=-2.0, high=3.0)
    got = oracle.moments(vol, 10)
    for g, w in zip(got, brute_moments(vol, 10)):
        assert g == pytest.approx(float(w), rel=1e-12, abs=1e-9)


def test_int128_overflow_is_detected_k10():
    vol = np.zeros((1, 1, 8192), dtype=np.uint16)
    vol[0, 0, 8191] = 65535  # 65535 * 8191^9 > 2^127 > 65535 * 8191^8
    with pytest.raises(OverflowError):
        oracle.moments(vol, 9)
    assert oracle.moments(vol, 8)[oracle.graded_triples(8).index((8, 0, 0))] == 65535 * 8191 ** 8


def test_coordinate_power_overflow_is_detected():
    """x^10 for x = 65535 leaves the int128 range on its own (x^7 does not);
    the moment (10, 0, 0) of that voxel then overflows too."""
    vol = np.zeros((1, 1, 65536), dtype=np.uint8)
    vol[0, 0, 65535] = 1
    with pytest.raises(OverflowError):
        oracle.moments(vol, 10)
    assert oracle.moments(vol, 7)[oracle.graded_triples(7).index((7, 0, 0))] == 65535 ** 7


@pytest.mark.parametrize("shape", [(1, 2, 65536), (2, 65536, 1), (65536, 1, 2)])
def test_constant_box_closed_form_at_largest_dimension(shape):
    N, M, L = shape
    vol = np.full(shape, 65535, dtype=np.uint16)
    got = oracle.moments(vol, 4, nthreads=4)
    for (p, q, r), g in zip(oracle.graded_triples(4), got):
        assert g == 65535 * faulhaber(p, L) * faulhaber(q, M) * faulhaber(r, N), (p, q, r)
    with pytest.raises(ValueError):
        oracle.moments(np.zeros((1, 1, 65537), np.uint8), 2)
