"""Host checks of the discrete Radon step 2 (Sec. 3.2 and its DRT integral
listing), no GPU needed.

* The library's solve of every degree n <= 10 is an exact inverse: with
  A[j][b] = C(n,b) alpha_j^b beta_j^(n-b) built here from the directions,
  E A = diag(D).
* The first five directions are the paper's five integrals (columns, rows,
  diagonal, anti-diagonal, x + 2y) and all are pairwise non-proportional.
* The whole route, written out here in Python integers (1-D integrals of a
  small image, their 1-D moments, the library's E and D), reproduces the
  2-D moments of Eq. 1 summed directly, for every a + b <= 10.
"""
from math import comb

import numpy as np
import pytest

import paper_2012_08099_gb300 as dpma

PAPER_FIVE = [(1, 0), (0, 1), (1, 1), (1, -1), (1, 2)]


@pytest.fixture(scope="module")
def plans():
    return [dpma.drt_plan(n) for n in range(11)]


def test_paper_directions_first_and_distinct(plans):
    dirs = plans[10][0]
    assert dirs[:5] == PAPER_FIVE
    for i in range(len(dirs)):
        for j in range(i):
            (a, b), (c, d) = dirs[i], dirs[j]
            assert a * d - b * c != 0, (dirs[i], dirs[j])


@pytest.mark.parametrize("n", range(11))
def test_solve_is_exact_inverse(plans, n):
    dirs, E, D = plans[n]
    A = [[comb(n, b) * a ** b * be ** (n - b) for b in range(n + 1)] for (a, be) in dirs]
    for r in range(n + 1):
        assert D[r] > 0
        for c in range(n + 1):
            s = sum(E[r][j] * A[j][c] for j in range(n + 1))
            assert s == (D[r] if r == c else 0), (n, r, c)


def test_route_reproduces_eq1_on_a_small_image(plans):
    rng = np.random.default_rng(7)
    S, F, off_s, off_f = 9, 13, 4, 0   # an offset slow coordinate, like a "-" image
    img = rng.integers(0, 1000, size=(S, F))
    K = 10
    direct = {}
    for a in range(K + 1):
        for b in range(K + 1 - a):
            direct[(a, b)] = sum(int(img[s, f]) * (s - off_s) ** a * (f - off_f) ** b
                                 for s in range(S) for f in range(F))
    dirs = plans[K][0]
    # 1-D integrals keyed by the signed coordinate t = alpha f' + beta s'
    prof = []
    for (al, be) in dirs:
        P = {}
        for s in range(S):
            for f in range(F):
                t = al * (f - off_f) + be * (s - off_s)
                P[t] = P.get(t, 0) + int(img[s, f])
        prof.append(P)
    for n in range(K + 1):
        _, E, D = plans[n]
        mu = [sum(t ** n * v for t, v in prof[j].items()) for j in range(n + 1)]
        for b in range(n + 1):
            num = sum(E[b][j] * mu[j] for j in range(n + 1))
            assert num % D[b] == 0
            assert num // D[b] == direct[(n - b, b)], (n, b)
