"""Pins of the oracle's projection images and image moments.

* image sizes of Eqs. 5-9 (with the x-y image read as L x M),
* a single voxel lands on exactly one pixel per image, where the image's
  two linear forms put it,
* mass conservation,
* the paper's identities Eqs. 10-16 between 2-D and 3-D moments, with the
  labels of Eqs. 15-16 corrected (the printed M112 and M211 formulas are
  swapped), checked between two independent oracle functions,
* the origin shift of the x-z image given in Sec. 5,
* Eq. 1 on single-pixel images and against exact rationals.
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle
from paper_2012_08099_gb300 import synth

# slow / fast linear forms of each image (coefficients of x, y, z)
FORMS = {
    0: ((0, 1, 0), (1, 0, 0)),
    1: ((0, 0, 1), (0, 1, 0)),
    2: ((0, 0, 1), (1, 0, 0)),
    3: ((0, 1, 0), (1, 0, 1)),
    4: ((0, 1, 0), (1, 0, -1)),
    5: ((0, 1, 1), (1, 0, 0)),
    6: ((0, 1, -1), (1, 0, 0)),
    7: ((0, 0, 1), (1, 1, 0)),
    8: ((0, 0, 1), (1, -1, 0)),
    9: ((0, 1, 0), (1, 0, 2)),     # arctan(1/2) about y
    10: ((1, 0, 1), (1, 2, -1)),   # isometric: (x+z, 2y+x-z)
}


def img_moment(imgs, geo, k, a, b, K):
    """T_ab of image k with signed coordinates (a: slow exponent)."""
    S, F, os_, of = geo[k]
    T = oracle.image_moments(imgs[k], os_, of, K)
    order = [(aa, n - aa) for n in range(K + 1) for aa in range(n, -1, -1)]
    return T[order.index((a, b))]


def test_image_sizes():
    L, M, N = 7, 5, 3
    want = {
        0: (M, L), 1: (N, M), 2: (N, L),          # Eqs. 5-7 (x-y image is L x M)
        3: (M, L + N - 1), 4: (M, L + N - 1),     # Eqs. 8-9: (L+N-1) x M
        5: (M + N - 1, L), 6: (M + N - 1, L),
        7: (N, L + M - 1), 8: (N, L + M - 1),
        9: (M, L + 2 * N - 2),
        10: (L + N - 1, L + 2 * M + N - 3),       # the paper's zero-padded isometric size
    }
    for k, (S, F) in want.items():
        assert oracle.image_geometry(k, L, M, N)[:2] == (S, F)
    assert [oracle.num_images(K) for K in (0, 1, 2, 3, 4, 6, 8, 9, 10)] == [
        3, 3, 3, 4, 5, 7, 9, 10, 11]


@pytest.mark.parametrize("pos", [(0, 0, 0), (6, 4, 2), (6, 0, 2), (0, 4, 0), (3, 2, 1)])
def test_single_voxel_lands_on_predicted_pixel(pos):
    L, M, N = 7, 5, 3
    x, y, z = pos
    vol = np.zeros((N, M, L), dtype=np.uint8)
    vol[z, y, x] = 9
    imgs = oracle.project(vol, 11)
    for k in range(11):
        S, F, os_, of = oracle.image_geometry(k, L, M, N)
        (sa, sb, sc), (fa, fb, fc) = FORMS[k]
        s = sa * x + sb * y + sc * z + os_
        f = fa * x + fb * y + fc * z + of
        assert 0 <= s < S and 0 <= f < F
        assert imgs[k][s, f] == 9
        assert int(imgs[k].sum()) == 9


def test_mass_conservation():
    vol = synth.uniform_volume((6, 5, 8), np.uint16, seed=1)
    tot = int(vol.astype(np.uint64).sum())
    for im in oracle.project(vol, 11):
        assert int(im.sum()) == tot
    fvol = synth.uniform_volume((6, 5, 8), np.float32, seed=1)
    for im in oracle.project(fvol, 11):
        assert im.sum() == pytest.approx(float(fvol.astype(np.float64).sum()), rel=1e-13)


def expand(form_s, form_f, a, b):
    """Coefficients of (form_s . x)^a (form_f . x)^b over monomials x^p y^q z^r."""
    poly = {(0, 0, 0): 1}

    def mul(poly, form):
        out = {}
        for (p, q, r), c in poly.items():
            for d, w in enumerate(form):
                if w == 0:
                    continue
                e = [p, q, r]
                e[d] += 1
                out[tuple(e)] = out.get(tuple(e), 0) + c * w
        return out

    for _ in range(a):
        poly = mul(poly, form_s)
    for _ in range(b):
        poly = mul(poly, form_f)
    return poly


def test_image_moments_expand_to_3d_moments():
    """sum I (s.x)^a (f.x)^b equals the multinomial expansion of 3-D moments."""
    vol = synth.uniform_volume((5, 6, 7), np.uint16, seed=2)
    N, M, L = vol.shape
    K = 6
    m3 = oracle.moments(vol, K)
    I = {t: i for i, t in enumerate(oracle.graded_triples(K))}
    imgs = oracle.project(vol, 9)
    geo = [oracle.image_geometry(k, L, M, N) for k in range(9)]
    for k in range(9):
        for n in range(K + 1):
            for a in range(n, -1, -1):
                want = sum(c * m3[I[e]] for e, c in expand(*FORMS[k], a, n - a).items())
                assert img_moment(imgs, geo, k, a, n - a, K) == want, (k, a, n - a)


def test_paper_identities_eq10_to_eq16():
    vol = synth.uniform_volume((6, 5, 7), np.uint8, seed=3)
    N, M, L = vol.shape
    K = 4
    m = oracle.moments(vol, K)
    I = {t: i for i, t in enumerate(oracle.graded_triples(K))}
    M3 = lambda p, q, r: m[I[(p, q, r)]]
    imgs = oracle.project(vol, 5)
    geo = [oracle.image_geometry(k, L, M, N) for k in range(5)]

    # paper convention M_pq = sum I(i,j) i^p j^q with (i, j) as printed in
    # Eqs. 5-9; map to the stored (slow, fast) exponents of each image.
    def xy(p, q):   # i = x (fast), j = y (slow)
        return img_moment(imgs, geo, 0, q, p, K)

    def yz(p, q):   # i = y (fast), j = z (slow)
        return img_moment(imgs, geo, 1, q, p, K)

    def zx(p, q):   # i = z (slow), j = x (fast)
        return img_moment(imgs, geo, 2, p, q, K)

    def plus(p, q):  # i = x+z (fast), j = y (slow)
        return img_moment(imgs, geo, 3, q, p, K)

    def minus(p, q):  # i = x-z (fast, signed), j = y (slow)
        return img_moment(imgs, geo, 4, q, p, K)

    for n in range(K + 1):
        for p in range(n + 1):
            q = n - p
            assert M3(p, q, 0) == xy(p, q)            # Eq. 10
            assert M3(0, p, q) == yz(p, q)            # Eq. 11
            assert M3(q, 0, p) == zx(p, q)            # Eq. 12
    assert 2 * M3(1, 1, 1) == plus(2, 1) - M3(2, 1, 0) - M3(0, 1, 2)        # Eq. 13
    assert 2 * M3(1, 2, 1) == plus(2, 2) - M3(2, 2, 0) - M3(0, 2, 2)        # Eq. 14
    # Eqs. 15-16 with the labels corrected:
    assert 6 * M3(1, 1, 2) == plus(3, 1) + minus(3, 1) - 2 * M3(3, 1, 0)
    assert 6 * M3(2, 1, 1) == plus(3, 1) - minus(3, 1) - 2 * M3(0, 1, 3)
    # ... and the formulas exactly as printed give the other moment:
    printed_112 = Fraction(plus(3, 1) - minus(3, 1) - 2 * M3(0, 1, 3), 6)
    printed_211 = Fraction(plus(3, 1) + minus(3, 1) - 2 * M3(3, 1, 0), 6)
    assert printed_112 == M3(2, 1, 1) != M3(1, 1, 2)
    assert printed_211 == M3(1, 1, 2)


def test_origin_shift_of_the_x_minus_z_image():
    """Sec. 5: moments about the stored origin, shifted by x_hat = N - 1."""
    vol = synth.uniform_volume((5, 4, 6), np.uint16, seed=4)
    N, M, L = vol.shape
    K = 4
    img = oracle.project(vol, 5)[4]
    order = [(a, n - a) for n in range(K + 1) for a in range(n, -1, -1)]
    stored = oracle.image_moments(img, 0, 0, K)          # i measured from the array edge
    signed = oracle.image_moments(img, 0, N - 1, K)      # i = x - z
    # paper's M_pq: i^p j^q with i the fast (x-z) coordinate, j = y the slow one
    Ms = lambda p, q: stored[order.index((q, p))]
    Mt = lambda p, q: signed[order.index((q, p))]
    xh = N - 1
    assert Mt(3, 1) == Ms(3, 1) - 3 * Ms(2, 1) * xh + 3 * Ms(1, 1) * xh ** 2 - Ms(0, 1) * xh ** 3
    assert Mt(1, 3) == Ms(1, 3) - Ms(0, 3) * xh
    # and the general binomial shift for every order
    for p in range(K + 1):
        for q in range(K + 1 - p):
            assert Mt(p, q) == sum(comb(p, k) * (-xh) ** (p - k) * Ms(k, q) for k in range(p + 1))


@pytest.mark.parametrize("at", [(0, 0), (3, 7), (2, 0), (0, 5)])
def test_image_moments_single_pixel(at):
    s, f = at
    img = np.zeros((4, 8), dtype=np.uint64)
    img[s, f] = 12345
    K = 8
    off_s, off_f = 1, 5
    T = oracle.image_moments(img, off_s, off_f, K)
    order = [(a, n - a) for n in range(K + 1) for a in range(n, -1, -1)]
    for (a, b), t in zip(order, T):
        assert t == 12345 * (s - off_s) ** a * (f - off_f) ** b


def test_float_image_moments_exact():
    g = np.random.Generator(np.random.PCG64(5))
    img = g.random((5, 6)) * 100.0
    K = 6
    T = oracle.image_moments(img, 2, 3, K)
    order = [(a, n - a) for n in range(K + 1) for a in range(n, -1, -1)]
    for (a, b), t in zip(order, T):
        exact = sum(Fraction(float(img[s, f])) * (s - 2) ** a * (f - 3) ** b
                    for s in range(5) for f in range(6))
        mag = sum(Fraction(float(img[s, f])) * abs(s - 2) ** a * abs(f - 3) ** b
                  for s in range(5) for f in range(6))
        assert abs(Fraction(t) - exact) <= Fraction(1e-14) * mag


def test_brute_force_images_9_and_10():
    """Images 9 and 10 pixel by pixel from a pure-Python loop over the voxels."""
    vol = synth.uniform_volume((4, 3, 5), np.uint16, seed=7)
    N, M, L = vol.shape
    imgs = oracle.project(vol, 11)
    for k in (9, 10):
        S, F, os_, of = oracle.image_geometry(k, L, M, N)
        want = np.zeros((S, F), dtype=np.uint64)
        (sa, sb, sc), (fa, fb, fc) = FORMS[k]
        for z in range(N):
            for y in range(M):
                for x in range(L):
                    want[sa * x + sb * y + sc * z + os_, fa * x + fb * y + fc * z + of] += int(vol[z, y, x])
        np.testing.assert_array_equal(imgs[k], want)


def test_image_moments_expand_to_3d_moments_k10():
    """Images 9 and 10 at order 10: every 2-D moment is the multinomial
    expansion of the 3-D moments."""
    vol = synth.uniform_volume((3, 4, 5), np.uint8, seed=5)
    N, M, L = vol.shape
    K = 10
    m3 = oracle.moments(vol, K)
    I = {t: i for i, t in enumerate(oracle.graded_triples(K))}
    imgs = oracle.project(vol, 11)
    geo = [oracle.image_geometry(k, L, M, N) for k in range(11)]
    for k in (0, 4, 9, 10):
        for n in range(K + 1):
            for a in range(n, -1, -1):
                want = sum(c * m3[I[e]] for e, c in expand(*FORMS[k], a, n - a).items())
                assert img_moment(imgs, geo, k, a, n - a, K) == want, (k, a, n - a)


def exact_rank(rows):
    """Rank over the rationals (fraction-exact Gaussian elimination)."""
    A = [[Fraction(v) for v in r] for r in rows]
    rank, col = 0, 0
    ncol = len(A[0]) if A else 0
    while rank < len(A) and col < ncol:
        piv = next((i for i in range(rank, len(A)) if A[i][col] != 0), None)
        if piv is None:
            col += 1
            continue
        A[rank], A[piv] = A[piv], A[rank]
        for i in range(rank + 1, len(A)):
            f = A[i][col] / A[rank][col]
            if f:
                A[i] = [a - f * b for a, b in zip(A[i], A[rank])]
        rank += 1
        col += 1
    return rank


@pytest.mark.parametrize("K", [8, 9, 10])
def test_images_reach_full_rank(K):
    """The rank argument: the 2-D moments of degree n of images 0..K span all
    (n+1)(n+2)/2 monomials of degree n, for every n <= K, so the 3-D moments
    follow from the images (and K images would not be enough at n = K)."""
    P = oracle.num_images(K)
    for n in range(K + 1):
        monos = [(p, q, n - p - q) for p in range(n, -1, -1) for q in range(n - p, -1, -1)]
        rows = []
        for k in range(P):
            for a in range(n, -1, -1):
                e = expand(*FORMS[k], a, n - a)
                rows.append([e.get(m, 0) for m in monos])
        assert exact_rank(rows) == len(monos), (K, n)
    n = K
    monos = [(p, q, n - p - q) for p in range(n, -1, -1) for q in range(n - p, -1, -1)]
    rows = [[expand(*FORMS[k], a, n - a).get(m, 0) for m in monos]
            for k in range(P - 1) for a in range(n, -1, -1)]
    assert exact_rank(rows) < len(monos)
