"""C-ABI checks that need no GPU.

* the library loads and exports every function ``include/dpma.h`` declares;
* host-only helpers (moment order, image geometry, buffer sizes) agree with
  the oracle's independent definitions;
* the exact combine plan: C A_sel = D I recomputed here in Python integers
  from the image forms, full rank with K+1 directions, the denominators of
  every degree, and -- applied in Python to the oracle's 2-D moments -- it
  reproduces the oracle's 3-D moments exactly (the paper's Eqs. 10-16 are
  the K <= 4 special case);
* argument validation of host-only calls.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2012_08099_gb300 as dpma
from paper_2012_08099_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FORMS = {
    0: ((0, 1, 0), (1, 0, 0)), 1: ((0, 0, 1), (0, 1, 0)), 2: ((0, 0, 1), (1, 0, 0)),
    3: ((0, 1, 0), (1, 0, 1)), 4: ((0, 1, 0), (1, 0, -1)), 5: ((0, 1, 1), (1, 0, 0)),
    6: ((0, 1, -1), (1, 0, 0)), 7: ((0, 0, 1), (1, 1, 0)), 8: ((0, 0, 1), (1, -1, 0)),
    9: ((0, 1, 0), (1, 0, 2)), 10: ((1, 0, 1), (1, 2, -1)),
}


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(dpma.LIB_PATH):
        from paper_2012_08099_gb300 import build
        build.build()
    return dpma.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dpma.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dpma_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_moment_order_matches_oracle(lib):
    for K in range(11):
        assert dpma.num_moments(K) == oracle.num_moments(K)
        assert dpma.num_images(K) == oracle.num_images(K)
        for i, (p, q, r) in enumerate(oracle.graded_triples(K)):
            assert dpma.moment_index(p, q, r) == i
    assert dpma.num_moments(11) == 0 and dpma.num_moments(-1) == 0
    assert dpma.moment_index(6, 5, 0) == -1 and dpma.moment_index(-1, 0, 0) == -1


@pytest.mark.parametrize("dims", [(1, 1, 1), (7, 5, 3), (64, 64, 64), (512, 300, 17)])
def test_image_geometry_matches_oracle(lib, dims):
    L, M, N = dims
    for k in range(11):
        assert dpma.image_geometry(k, L, M, N) == oracle.image_geometry(k, L, M, N)


def test_buffer_sizes(lib):
    L, M, N = 37, 21, 13
    for dt, per in ((dpma.U8, 4), (dpma.U16, 4), (dpma.F32, 8)):
        for K in (0, 3, 6, 8) + ((9, 10) if dt != dpma.F32 else ()):
            want = sum(oracle.image_geometry(k, L, M, N)[0] * oracle.image_geometry(k, L, M, N)[1]
                       for k in range(oracle.num_images(K))) * per
            assert dpma.images_size(L, M, N, dt, K) == want
            assert dpma.workspace_size(L, M, N, dt, K) > want
    assert dpma.images_size(0, 5, 5, dpma.U8, 3) == 0
    assert dpma.workspace_size(5, 5, 5, dpma.U8, 11) == 0
    assert dpma.workspace_size(5, 5, 5, dpma.F32, 9) == 0  # float32 volumes: K <= 8


def expand(fs, ff, a, b, n):
    """Row of (fs.x)^a (ff.x)^b over the degree-n monomials in graded order."""
    poly = {(0, 0, 0): 1}
    for form in [fs] * a + [ff] * b:
        nxt = {}
        for e, c in poly.items():
            for d, w in enumerate(form):
                if w:
                    e2 = list(e)
                    e2[d] += 1
                    nxt[tuple(e2)] = nxt.get(tuple(e2), 0) + c * w
        poly = nxt
    monos = [(p, q, n - p - q) for p in range(n, -1, -1) for q in range(n - p, -1, -1)]
    return [poly.get(m, 0) for m in monos]


@pytest.mark.parametrize("K", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_combine_plan_is_an_exact_inverse(lib, K):
    for n in range(K + 1):
        D, img, a, C = dpma.combine_plan(K, n)
        nm = (n + 1) * (n + 2) // 2
        assert C.shape == (nm, nm)
        assert all(0 <= i < dpma.num_images(K) for i in img)
        A = np.array([expand(*FORMS[i], aa, n - aa, n) for i, aa in zip(img, a)], dtype=object)
        prod = np.array(C, dtype=object).dot(A)
        assert (prod == D * np.eye(nm, dtype=object)).all()


def test_combine_denominators():
    # D_n per degree (the lcm of the exact inverse's denominators); they do
    # not depend on K once the degree has enough images
    want = [1, 1, 1, 2, 6, 24, 120, 120, 1680]
    for n in range(9):
        assert dpma.combine_plan(8, n)[0] == want[n]
        if n <= 6:
            assert dpma.combine_plan(6, n)[0] == want[n]
    # small integer matrices: |C| <= 2100 at K = 8, 120 at K = 6
    assert max(abs(int(v)) for n in range(9) for v in dpma.combine_plan(8, n)[3].ravel()) == 2100
    assert max(abs(int(v)) for n in range(7) for v in dpma.combine_plan(6, n)[3].ravel()) == 120
    # orders 9 and 10 (with the arctan(1/2) and isometric images)
    assert [dpma.combine_plan(10, n)[0] for n in range(11)][:9] == want
    assert dpma.combine_plan(9, 9)[0] == dpma.combine_plan(10, 9)[0]


def test_k_plus_one_directions_are_needed():
    """With K directions the degree-K system is rank deficient (so P = K+1)."""
    from fractions import Fraction

    def rank(rows):
        m = [[Fraction(v) for v in r] for r in rows]
        rk, col = 0, 0
        ncol = len(m[0])
        while rk < len(m) and col < ncol:
            piv = next((i for i in range(rk, len(m)) if m[i][col] != 0), None)
            if piv is None:
                col += 1
                continue
            m[rk], m[piv] = m[piv], m[rk]
            for i in range(len(m)):
                if i != rk and m[i][col] != 0:
                    f = m[i][col] / m[rk][col]
                    m[i] = [x - f * y for x, y in zip(m[i], m[rk])]
            rk += 1
            col += 1
        return rk

    for n in (3, 4, 6, 9, 10):
        nm = (n + 1) * (n + 2) // 2
        full = [expand(*FORMS[k], a, n - a, n) for k in range(n + 1) for a in range(n, -1, -1)]
        short = [expand(*FORMS[k], a, n - a, n) for k in range(n) for a in range(n, -1, -1)]
        assert rank(full) == nm
        assert rank(short) < nm


@pytest.mark.parametrize("K,dtype", [(3, np.uint8), (4, np.uint16), (6, np.uint16), (8, np.uint8),
                                     (9, np.uint16), (10, np.uint8)])
def test_plan_applied_to_oracle_image_moments_gives_oracle_moments(K, dtype):
    vol = synth.uniform_volume((5, 6, 7), dtype, seed=K)
    N, M, L = vol.shape
    imgs = oracle.project(vol, oracle.num_images(K))
    T = []
    for k, im in enumerate(imgs):
        S, F, os_, of = oracle.image_geometry(k, L, M, N)
        T.append(oracle.image_moments(im, os_, of, K))
    m3 = oracle.moments(vol, K)
    for n in range(K + 1):
        D, img, a, C = dpma.combine_plan(K, n)
        t = [T[i][n * (n + 1) // 2 + (n - aa)] for i, aa in zip(img, a)]
        for row in range(C.shape[0]):
            acc = sum(int(c) * v for c, v in zip(C[row], t))
            assert acc % D == 0
            m = n * (n + 1) * (n + 2) // 6 + row
            assert acc // D == m3[m]


def test_status_strings(lib):
    for s in range(8):
        assert lib.dpma_status_string(s)
    assert lib.dpma_combine_plan(3, 4, None, None, None, None, None) == 1
    assert b"0 <= n <= K" in lib.dpma_last_error()


def test_batch_arguments_checked_on_the_host(lib):
    """dpma_batch_create validates every descriptor before touching a device."""
    import paper_2012_08099_gb300 as d
    h = ctypes.c_void_p()
    assert lib.dpma_batch_create(None, 1, 0, ctypes.byref(h)) == 1
    assert lib.dpma_batch_create(None, -1, 0, ctypes.byref(h)) == 1

    def one(**kw):
        f = dict(volume=0x1000, L=8, M=8, N=8, dtype=d.U8, K=3, out_offset=0)
        f.update(kw)
        arr = (d.VolumeDesc * 1)(d.VolumeDesc(**f))
        return lib.dpma_batch_create(arr, 1, 0, ctypes.byref(h))

    assert one(volume=None) == 1
    assert one(out_offset=8) == 1
    assert one(out_offset=-16) == 1
    assert one(L=0) == 1
    assert one(K=9) == 1
    assert one(dtype=5) == 1
    assert one(L=65536, M=65536, N=65536, dtype=d.U16, K=8) == 2
    arr = (d.VolumeDesc * 1)(d.VolumeDesc(0x1000, 8, 8, 8, d.U8, 3, 0))
    assert lib.dpma_batch_create(arr, 1, 4, ctypes.byref(h)) == 1  # unknown flag
    assert lib.dpma_batch_info(None, 0) == -1
    assert lib.dpma_batch_destroy(None) == 0


def test_server_arguments_checked(lib):
    import paper_2012_08099_gb300 as d
    h = ctypes.c_void_p()
    assert lib.dpma_server_create(None, None) == 1
    bad = d.ServerConfig(-1, 0, 0, 0, 0)
    assert lib.dpma_server_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    t = ctypes.c_uint64()
    assert lib.dpma_server_submit(None, None, ctypes.byref(t)) == 1
    assert lib.dpma_server_poll(None, 1) == -1
    assert lib.dpma_server_destroy(None) == 0
