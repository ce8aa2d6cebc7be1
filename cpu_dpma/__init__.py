"""Multithreaded CPU implementation of the Discrete Projection Moment method.

The timed CPU baseline: projection images of the volume (Sec. 3.1), their
2-D moments through 1-D integrals along K + 1 directions (the discrete Radon
transform route of Sec. 3.2 / Sec. 4), and the 3-D moments from those
(Eqs. 10-16, generalised), on all host cores.  The C++ lives in
``cpu_dpma.cpp`` (compiled into ``libcpu_dpma.so`` beside it); this module
only marshals numpy arrays.  It shares no code with the CUDA library or with
the oracle.

Volumes are numpy arrays of shape ``(N, M, L)`` (z, y, x), x fastest.
Moments come in graded order (degree ascending, then p descending, then q
descending): exact Python ints for uint8/uint16, float64 for float32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_dpma.cpp")
_HDR = os.path.join(_HERE, "cpu_dpma.h")
_LIB_PATH = os.path.join(_HERE, "libcpu_dpma.so")
_lock = threading.Lock()
_lib = None

ERRORS = {1: "invalid argument", 2: "non-finite float voxel", 3: "result outside int128",
          4: "no image set of full rank", 5: "out of memory"}


class CpuDpmaError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"cpu_dpma error {code}: {ERRORS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile ``cpu_dpma.cpp`` into ``libcpu_dpma.so`` (g++, no GPU)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, vp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            lib.cpu_dpma_moments.argtypes = [vp, i64, i64, i64, ip, ip, ip, vp,
                                             ctypes.POINTER(ip)]
            lib.cpu_dpma_moments.restype = ip
            lib.cpu_dpma_num_images.argtypes = [ip]
            lib.cpu_dpma_num_images.restype = ip
            lib.cpu_dpma_max_order.restype = ip
            lib.cpu_dpma_last_float_exponent.restype = ip
            _lib = lib
    return _lib


def max_order() -> int:
    return _load().cpu_dpma_max_order()


def num_images(K: int) -> int:
    return _load().cpu_dpma_num_images(K)


def num_moments(K: int) -> int:
    return (K + 1) * (K + 2) * (K + 3) // 6


def moments(vol: np.ndarray, K: int, threads: int = 0, return_threads: bool = False):
    """All M_pqr, p+q+r <= K, of a host volume (N, M, L)."""
    lib = _load()
    codes = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2}
    if vol.dtype not in codes or vol.ndim != 3:
        raise CpuDpmaError(1)
    v = np.ascontiguousarray(vol)
    N, M, L = v.shape
    dt = codes[v.dtype]
    nm = num_moments(K) if K >= 0 else 0
    out = np.zeros(max(nm, 1) * (1 if dt == 2 else 2),
                   dtype=np.float64 if dt == 2 else np.int64)
    used = ctypes.c_int(0)
    rc = lib.cpu_dpma_moments(v.ctypes.data, L, M, N, dt, K, threads, out.ctypes.data,
                              ctypes.byref(used))
    if rc:
        raise CpuDpmaError(rc)
    if dt == 2:
        res = out[:nm]
    else:
        w = out[:2 * nm].reshape(-1, 2)
        res = [(int(hi) << 64) | (int(lo) & ((1 << 64) - 1)) for lo, hi in w]
    return (res, used.value) if return_threads else res
