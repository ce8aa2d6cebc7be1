"""CPU oracle for the Discrete Projection Moment method (test infrastructure).

TEST INFRASTRUCTURE ONLY: the product library never imports, links or calls
this package.  The test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are its only users.

The arithmetic lives in ``oracle.c`` (plain C, compiled on first use into
``liboracle.so`` beside it); this module only marshals numpy arrays.

* :func:`moments` -- Sec. 1, Eq. 2, the definition of the raw 3D moments,
  exact in ``__int128`` for uint8/uint16 volumes, FP64 (compensated) for
  float32 volumes.
* :func:`project` -- Sec. 3.1, Eq. 4 with Eqs. 5-9 and the +-pi/4 families:
  the projection images, pixel by pixel; orders 9 and 10 add the
  arctan(1/2) image about y and the isometric image (x+z, 2y+x-z) of the
  further families named after Eq. 9.  Orders up to K = 10.
* :func:`image_moments` -- Sec. 1, Eq. 1 on one stored image.
* :func:`central_moments` -- Sec. 4: centroid and central moments from
  their definitions over the voxels (with the matching sums of |.| as the
  error scale).

Volumes are numpy arrays of shape ``(N, M, L)`` (z, y, x) with x fastest,
i.e. ``V[z, y, x]``.  Moments come in graded order: degree ascending, then
p descending, then q descending.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (plain gcc, no GPU)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, vp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            lib.oracle_moments_int.argtypes = [vp, ip, i64, i64, i64, ip, ip, vp]
            lib.oracle_moments_f32.argtypes = [vp, i64, i64, i64, ip, ip, vp]
            lib.oracle_moments_f32_abs.argtypes = [vp, i64, i64, i64, ip, ip, vp]
            lib.oracle_project_int.argtypes = [vp, ip, i64, i64, i64, ip, vp]
            lib.oracle_project_f32.argtypes = [vp, i64, i64, i64, ip, vp]
            lib.oracle_image_moments_int.argtypes = [vp, i64, i64, i64, i64, ip, vp]
            lib.oracle_image_moments_f64.argtypes = [vp, i64, i64, i64, i64, ip, vp]
            lib.oracle_image_geometry.argtypes = [ip, i64, i64, i64] + [ctypes.POINTER(i64)] * 4
            lib.oracle_central_moments.argtypes = [vp, ip, i64, i64, i64, ip, vp, vp, vp]
            lib.oracle_central_moments.restype = ctypes.c_int
            for f in (
                lib.oracle_moments_int, lib.oracle_moments_f32, lib.oracle_moments_f32_abs,
                lib.oracle_project_int, lib.oracle_project_f32, lib.oracle_image_moments_int,
                lib.oracle_image_moments_f64, lib.oracle_image_geometry,
                lib.oracle_num_moments, lib.oracle_num_images,
            ):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_moments(K: int) -> int:
    return (K + 1) * (K + 2) * (K + 3) // 6


def num_images(K: int) -> int:
    return max(3, K + 1)


def graded_triples(K: int) -> list[tuple[int, int, int]]:
    """Exponent triples (p, q, r) with p+q+r <= K in graded order."""
    out = []
    for n in range(K + 1):
        for p in range(n, -1, -1):
            for q in range(n - p, -1, -1):
                out.append((p, q, n - p - q))
    return out


def _i128_pairs_to_ints(buf: np.ndarray) -> list[int]:
    out = []
    for k in range(len(buf) // 2):
        lo = int(buf[2 * k]) & ((1 << 64) - 1)
        hi = int(buf[2 * k + 1])
        out.append((hi << 64) | lo)
    return out


def moments(vol: np.ndarray, K: int, nthreads: int | None = None, absolute: bool = False):
    """Raw moments M_pqr, p+q+r <= K, of ``vol[z, y, x]`` (Eq. 2).

    Integer volumes return a list of Python ints (exact); float32 volumes a
    float64 numpy array.  ``absolute=True`` (float only) returns the moments
    of |V|, the magnitude the float tolerance is measured against.
    """
    lib = _load()
    vol = np.ascontiguousarray(vol)
    if vol.ndim != 3:
        raise ValueError("volume must be 3-D (N, M, L)")
    N, M, L = vol.shape
    nt = nthreads or min(os.cpu_count() or 1, 32)
    nm = num_moments(K)
    if vol.dtype in (np.uint8, np.uint16):
        if absolute:
            raise ValueError("absolute moments are only defined for float volumes")
        out = np.zeros(2 * nm, dtype=np.int64)
        rc = lib.oracle_moments_int(vol.ctypes.data, vol.dtype.itemsize, L, M, N, K, nt,
                                    out.ctypes.data)
        if rc == 2:
            raise OverflowError("moment exceeds the int128 range")
        if rc:
            raise ValueError(f"oracle_moments_int rejected the arguments (rc={rc})")
        return _i128_pairs_to_ints(out)
    if vol.dtype == np.float32:
        out = np.zeros(nm, dtype=np.float64)
        fn = lib.oracle_moments_f32_abs if absolute else lib.oracle_moments_f32
        rc = fn(vol.ctypes.data, L, M, N, K, nt, out.ctypes.data)
        if rc:
            raise ValueError(f"oracle_moments_f32 rejected the arguments (rc={rc})")
        return out
    raise TypeError(f"unsupported dtype {vol.dtype}")


def image_geometry(k: int, L: int, M: int, N: int) -> tuple[int, int, int, int]:
    """(S, F, off_s, off_f) of image k for an L x M x N volume."""
    lib = _load()
    vals = [ctypes.c_int64() for _ in range(4)]
    if lib.oracle_image_geometry(k, L, M, N, *[ctypes.byref(v) for v in vals]):
        raise ValueError(f"no image {k}")
    return tuple(int(v.value) for v in vals)


def project(vol: np.ndarray, P: int) -> list[np.ndarray]:
    """Images 0..P-1 of ``vol`` as 2-D arrays [S_k, F_k] (uint64 or float64)."""
    lib = _load()
    vol = np.ascontiguousarray(vol)
    N, M, L = vol.shape
    geo = [image_geometry(k, L, M, N) for k in range(P)]
    total = sum(S * F for S, F, _, _ in geo)
    if vol.dtype in (np.uint8, np.uint16):
        out = np.zeros(total, dtype=np.uint64)
        rc = lib.oracle_project_int(vol.ctypes.data, vol.dtype.itemsize, L, M, N, P,
                                    out.ctypes.data)
    elif vol.dtype == np.float32:
        out = np.zeros(total, dtype=np.float64)
        rc = lib.oracle_project_f32(vol.ctypes.data, L, M, N, P, out.ctypes.data)
    else:
        raise TypeError(f"unsupported dtype {vol.dtype}")
    if rc:
        raise ValueError(f"oracle_project rejected the arguments (rc={rc})")
    imgs, at = [], 0
    for S, F, _, _ in geo:
        imgs.append(out[at:at + S * F].reshape(S, F))
        at += S * F
    return imgs


def image_moments(img: np.ndarray, off_s: int, off_f: int, K: int):
    """T_ab = sum I[s,f] (s-off_s)^a (f-off_f)^b, a+b <= K (Eq. 1).

    Order: degree ascending, slow exponent a descending.  uint64 images give
    exact Python ints; float64 images give a float64 array.
    """
    lib = _load()
    img = np.ascontiguousarray(img)
    S, F = img.shape
    nm = (K + 1) * (K + 2) // 2
    if img.dtype == np.uint64:
        out = np.zeros(2 * nm, dtype=np.int64)
        rc = lib.oracle_image_moments_int(img.ctypes.data, S, F, off_s, off_f, K,
                                          out.ctypes.data)
        if rc == 2:
            raise OverflowError("image moment exceeds the int128 range")
        if rc:
            raise ValueError("bad arguments")
        return _i128_pairs_to_ints(out)
    if img.dtype == np.float64:
        out = np.zeros(nm, dtype=np.float64)
        rc = lib.oracle_image_moments_f64(img.ctypes.data, S, F, off_s, off_f, K,
                                          out.ctypes.data)
        if rc:
            raise ValueError("bad arguments")
        return out
    raise TypeError(f"unsupported image dtype {img.dtype}")


def central_moments(vol: np.ndarray, K: int):
    """(centroid[3], mu, muabs) of Sec. 4 from the definitions (FP64 numpy arrays).

    ``mu[m] = sum V (x-xbar)^p (y-ybar)^q (z-zbar)^r`` and ``muabs`` the same
    sum of absolute values, in graded order.
    """
    lib = _load()
    v = np.ascontiguousarray(vol)
    N, M, L = v.shape
    eb = {np.dtype(np.uint8): 1, np.dtype(np.uint16): 2, np.dtype(np.float32): 4}[v.dtype]
    nm = num_moments(K)
    c = np.empty(3, dtype=np.float64)
    mu = np.empty(nm, dtype=np.float64)
    ma = np.empty(nm, dtype=np.float64)
    rc = lib.oracle_central_moments(v.ctypes.data, eb, L, M, N, K, c.ctypes.data,
                                    mu.ctypes.data, ma.ctypes.data)
    if rc:
        raise ValueError("oracle_central_moments: bad arguments")
    return c, mu, ma
