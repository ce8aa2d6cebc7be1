"""GB300-native Discrete Projection Moment library (Diggin & Diggin 2020).

Thin ctypes binding over ``libdpma.so`` (C ABI declared in
``include/dpma.h``).  Every step of the computation runs in the library's
CUDA kernels; this module only marshals arguments.  PyTorch supplies device
memory and streams.  If the compiled library is missing, every call raises
``RuntimeError``; there is no fallback.

Volumes are tensors of shape ``(N, M, L)`` (z, y, x) with x contiguous.
Moments come back in graded order (degree ascending, then p descending,
then q descending): exact Python ints for integer volumes, float64 for
float32 volumes.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdpma.so")

U8, U16, F32 = 0, 1, 2
STATUS = {
    0: "ok", 1: "invalid argument", 2: "exact range exceeded", 3: "out of device memory",
    4: "CUDA error", 5: "device wait timed out", 6: "request rejected",
    7: "internal self-check failed",
}

_lock = threading.Lock()
_lib = None


class DpmaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class VolumeDesc(ctypes.Structure):
    """``dpma_volume_desc`` of include/dpma.h."""
    _fields_ = [("volume", ctypes.c_void_p), ("L", ctypes.c_int64), ("M", ctypes.c_int64),
                ("N", ctypes.c_int64), ("dtype", ctypes.c_int32), ("K", ctypes.c_int32),
                ("out_offset", ctypes.c_int64)]


BATCH_AUTOTUNE = 1


class ServerConfig(ctypes.Structure):
    """``dpma_server_config`` of include/dpma.h (zero fields take the defaults)."""
    _fields_ = [("device_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("max_group", ctypes.c_int32),
                ("max_pending", ctypes.c_int32)]


class ServerCounters(ctypes.Structure):
    """``dpma_server_counters`` of include/dpma.h."""
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "rejected",
                                              "pending", "inflight", "launches",
                                              "device_bytes_peak")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "max_ms",
                                               "volumes_per_s", "voxels_per_s")] + \
               [(n, ctypes.c_int64) for n in ("cache_hits", "resident_volumes")]


def lib():
    """The loaded ``libdpma.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_2012_08099_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            i64, vp, ip, sz = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            P64 = ctypes.POINTER(ctypes.c_int64)
            sigs = {
                "dpma_num_moments": (ip, [ip]),
                "dpma_num_images": (ip, [ip]),
                "dpma_moment_index": (ip, [ip, ip, ip]),
                "dpma_status_string": (ctypes.c_char_p, [ip]),
                "dpma_last_error": (ctypes.c_char_p, []),
                "dpma_last_float_path": (ip, []),
                "dpma_set_wait_budget": (ip, [i64]),
                "dpma_image_geometry": (ip, [ip, i64, i64, i64, P64, P64, P64, P64]),
                "dpma_images_size": (sz, [i64, i64, i64, ip, ip]),
                "dpma_workspace_size": (sz, [i64, i64, i64, ip, ip]),
                "dpma_combine_plan": (ip, [ip, ip, ctypes.POINTER(ctypes.c_int), P64,
                                           ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), P64]),
                "dpma_moments": (ip, [vp, i64, i64, i64, ip, ip, vp]),
                "dpma_moments_async": (ip, [vp, i64, i64, i64, ip, ip, vp, vp, vp, sz]),
                "dpma_moments_host": (ip, [vp, i64, i64, i64, ip, ip, vp]),
                "dpma_project": (ip, [vp, i64, i64, i64, ip, ip, vp, vp]),
                "dpma_image_moments": (ip, [vp, i64, i64, i64, ip, ip, vp, vp, vp, sz]),
                "dpma_image_moments_drt": (ip, [vp, i64, i64, i64, ip, ip, vp, vp, vp, sz, vp]),
                "dpma_drt_workspace_size": (sz, [i64, i64, i64, ip, ip]),
                "dpma_drt_plan": (ip, [ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       P64, P64]),
                "dpma_combine": (ip, [vp, ip, ip, vp, vp, vp]),
                "dpma_moments_noalloc": (ip, [vp, i64, i64, i64, ip, ip, vp, vp]),
                "dpma_stage_timing": (ip, [ip]),
                "dpma_stage_times": (ip, [ctypes.POINTER(ctypes.c_double), P64, ip]),
                "dpma_batch_create": (ip, [ctypes.POINTER(VolumeDesc), ip, ip,
                                           ctypes.POINTER(vp)]),
                "dpma_batch_run": (ip, [vp, vp, vp]),
                "dpma_batch_status": (ip, [vp, vp]),
                "dpma_batch_info": (ip, [vp, ip]),
                "dpma_batch_destroy": (ip, [vp]),
                "dpma_moments_batched": (ip, [ctypes.POINTER(VolumeDesc), ip, vp, vp]),
                "dpma_moments_from_projections": (ip, [vp, i64, i64, i64, ip, ip, vp, vp]),
                "dpma_derived_moments": (ip, [vp, ip, ip, ctypes.POINTER(ctypes.c_double), vp,
                                              vp]),
                "dpma_server_create": (ip, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
                "dpma_server_submit": (ip, [vp, ctypes.POINTER(VolumeDesc),
                                            ctypes.POINTER(ctypes.c_uint64)]),
                "dpma_server_submit_keyed": (ip, [vp, ctypes.POINTER(VolumeDesc), ctypes.c_uint64,
                                                  ctypes.POINTER(ctypes.c_uint64)]),
                "dpma_server_wait": (ip, [vp, ctypes.c_uint64, i64, vp]),
                "dpma_server_poll": (ip, [vp, ctypes.c_uint64]),
                "dpma_server_stats": (ip, [vp, ctypes.POINTER(ServerCounters), ip]),
                "dpma_server_destroy": (ip, [vp]),
            }
            for name, (res, args) in sigs.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise DpmaError(rc, lib().dpma_last_error().decode())


# ---------------------------------------------------------------- helpers


def last_float_path() -> int:
    """0 if the calling thread's last synchronous float32 call was served by
    the quantised integer-lane pipeline; otherwise the flags that sent it to
    the compensated fallback (1: a voxel beyond the grid, 2: an error bound
    above the tolerance)."""
    return lib().dpma_last_float_path()


def set_wait_budget(cycles: int):
    """Test hook: cycles a bounded device wait spins before it gives up (0:
    the default)."""
    _check(lib().dpma_set_wait_budget(cycles))


def num_moments(K: int) -> int:
    return lib().dpma_num_moments(K)


def num_images(K: int) -> int:
    return lib().dpma_num_images(K)


def moment_index(p: int, q: int, r: int) -> int:
    return lib().dpma_moment_index(p, q, r)


def image_geometry(k: int, L: int, M: int, N: int) -> tuple[int, int, int, int]:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().dpma_image_geometry(k, L, M, N, *[ctypes.byref(x) for x in v]))
    return tuple(int(x.value) for x in v)


def images_size(L, M, N, dtype: int, K: int) -> int:
    return int(lib().dpma_images_size(L, M, N, dtype, K))


def workspace_size(L, M, N, dtype: int, K: int) -> int:
    return int(lib().dpma_workspace_size(L, M, N, dtype, K))


def combine_plan(K: int, n: int):
    """(D, img, a, C) of the exact degree-n combine for order K."""
    nm = ctypes.c_int()
    D = ctypes.c_int64()
    img = (ctypes.c_int32 * 66)()
    a = (ctypes.c_int32 * 66)()
    C = (ctypes.c_int64 * (66 * 66))()
    _check(lib().dpma_combine_plan(K, n, ctypes.byref(nm), ctypes.byref(D), img, a, C))
    m = nm.value
    Cm = np.array(C[: m * m], dtype=np.int64).reshape(m, m)
    return int(D.value), list(img[:m]), list(a[:m]), Cm


def int128_to_ints(words) -> list[int]:
    """Little-endian int128 values given as (lo, hi) int64 pairs -> Python ints."""
    w = np.asarray(words, dtype=np.int64).reshape(-1, 2)
    return [((int(hi) << 64) | (int(lo) & 0xFFFFFFFFFFFFFFFF)) for lo, hi in w]


def dtype_code(t) -> int:
    """Library dtype of a torch tensor or numpy array (uint16 may arrive as int16 bits)."""
    name = str(getattr(t, "dtype", t)).replace("torch.", "")
    if name == "uint8":
        return U8
    if name in ("uint16",):
        return U16
    if name == "float32":
        return F32
    raise TypeError(f"unsupported volume dtype {name}; use uint8, uint16 or float32")


def _shape(vol):
    if vol.dim() != 3:
        raise ValueError("volume must be 3-D (N, M, L)")
    if not vol.is_contiguous():
        raise ValueError("volume must be contiguous (x fastest)")
    N, M, L = vol.shape
    return int(L), int(M), int(N)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


# ------------------------------------------------------------- hot path


def moments(volume, K: int, dtype: int | None = None, out=None):
    """All moments M_pqr, p+q+r <= K, of a CUDA volume (synchronous).

    ``volume``: CUDA tensor (N, M, L); pass ``dtype=U16`` when uint16 data
    is held in an int16 tensor.  Returns exact ints or a float64 tensor.
    """
    import torch
    dt = dtype_code(volume) if dtype is None else dtype
    L, M, N = _shape(volume)
    nm = lib().dpma_num_moments(K)
    if nm == 0:
        raise DpmaError(1, "K must lie in 0..10")
    if out is None:
        out = torch.empty((nm, 2) if dt != F32 else (nm,),
                          dtype=torch.int64 if dt != F32 else torch.float64, device=volume.device)
    with torch.cuda.device(volume.device):
        _check(lib().dpma_moments(ctypes.c_void_p(volume.data_ptr()), L, M, N, dt, K,
                                  ctypes.c_void_p(out.data_ptr())))
    return out


def moments_values(volume, K: int, dtype: int | None = None):
    """Like :func:`moments` but returns host values (ints or float64 numpy)."""
    dt = dtype_code(volume) if dtype is None else dtype
    out = moments(volume, K, dt)
    if dt == F32:
        return out.cpu().numpy()
    return int128_to_ints(out.cpu().numpy())


def moments_async(volume, K: int, out, dtype: int | None = None, stream=None, workspace=None):
    """Enqueue the three steps on ``stream`` (default: torch's current stream)."""
    dt = dtype_code(volume) if dtype is None else dtype
    L, M, N = _shape(volume)
    ws_ptr = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else None
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().dpma_moments_async(ctypes.c_void_p(volume.data_ptr()), L, M, N, dt, K,
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream),
                                    ws_ptr, ws_bytes))
    return out


def moments_host(volume: np.ndarray, K: int, dtype: int | None = None, out: np.ndarray | None = None):
    """End to end from host memory (copies in, computes, copies out)."""
    vol = np.ascontiguousarray(volume)
    dt = dtype_code(vol) if dtype is None else dtype
    N, M, L = vol.shape
    nm = lib().dpma_num_moments(K)
    if out is None:
        out = np.empty((nm, 2) if dt != F32 else (nm,), dtype=np.int64 if dt != F32 else np.float64)
    _check(lib().dpma_moments_host(ctypes.c_void_p(vol.ctypes.data), L, M, N, dt, K,
                                   ctypes.c_void_p(out.ctypes.data)))
    return out


def project(volume, K: int, dtype: int | None = None, stream=None):
    """Step 1 alone: the projection images as a list of CPU numpy arrays.

    Integer volumes give uint64 arrays [S_k, F_k]; float volumes give float64
    arrays (the library's float images are doubles).
    """
    import torch
    dt = dtype_code(volume) if dtype is None else dtype
    L, M, N = _shape(volume)
    nbytes = images_size(L, M, N, dt, K)
    buf = torch.empty(nbytes // 4, dtype=torch.int32, device=volume.device)
    _check(lib().dpma_project(ctypes.c_void_p(volume.data_ptr()), L, M, N, dt, K,
                              ctypes.c_void_p(buf.data_ptr()), _stream_ptr(stream)))
    torch.cuda.synchronize(volume.device)
    host = buf.cpu().numpy()
    imgs, at = [], 0
    for k in range(num_images(K)):
        S, F, _, _ = image_geometry(k, L, M, N)
        if dt == F32:
            imgs.append(host.view(np.float64)[at:at + S * F].copy().reshape(S, F))
            at += S * F
        else:
            imgs.append(host.view(np.uint32)[at:at + S * F].astype(np.uint64).reshape(S, F))
            at += S * F
    return imgs


def image_moments_of(volume, K: int, dtype: int | None = None):
    """Steps 1+2 through the C ABI: per-image 2-D moments (ints or float64)."""
    import torch
    dt = dtype_code(volume) if dtype is None else dtype
    L, M, N = _shape(volume)
    P = num_images(K)
    npairs = (K + 1) * (K + 2) // 2
    imgs = torch.empty(images_size(L, M, N, dt, K) // 4, dtype=torch.int32, device=volume.device)
    st = _stream_ptr(None)
    _check(lib().dpma_project(ctypes.c_void_p(volume.data_ptr()), L, M, N, dt, K,
                              ctypes.c_void_p(imgs.data_ptr()), st))
    m2d = torch.empty(P * npairs * (2 if dt == F32 else 4), dtype=torch.int32,
                      device=volume.device)
    _check(lib().dpma_image_moments(ctypes.c_void_p(imgs.data_ptr()), L, M, N, dt, K,
                                    ctypes.c_void_p(m2d.data_ptr()), st, None, 0))
    torch.cuda.synchronize(volume.device)
    h = m2d.cpu().numpy()
    if dt == F32:
        f = h.view(np.float32).reshape(P, npairs, 2).astype(np.float64)
        return f[:, :, 0] + f[:, :, 1]
    vals = int128_to_ints(h.view(np.int64))
    return [vals[k * npairs:(k + 1) * npairs] for k in range(P)]


def image_moments_drt_of(volume, K: int, dtype: int | None = None, images=None, status=None):
    """Steps 1+2 through the C ABI with the discrete Radon step 2
    (dpma_image_moments_drt): per-image 2-D moments as Python ints.  With
    ``images`` (a device buffer as dpma_project writes it) step 1 is skipped;
    ``status`` (an int32 device tensor) receives a remainder flag."""
    import torch
    dt = dtype_code(volume) if dtype is None else dtype
    L, M, N = _shape(volume)
    P = num_images(K)
    npairs = (K + 1) * (K + 2) // 2
    st = _stream_ptr(None)
    if images is None:
        images = torch.empty(images_size(L, M, N, dt, K) // 4, dtype=torch.int32,
                             device=volume.device)
        _check(lib().dpma_project(ctypes.c_void_p(volume.data_ptr()), L, M, N, dt, K,
                                  ctypes.c_void_p(images.data_ptr()), st))
    m2d = torch.empty(P * npairs * 4, dtype=torch.int32, device=volume.device)
    nws = lib().dpma_drt_workspace_size(L, M, N, dt, K)
    ws = torch.empty(max(nws, 1), dtype=torch.uint8, device=volume.device)
    _check(lib().dpma_image_moments_drt(ctypes.c_void_p(images.data_ptr()), L, M, N, dt, K,
                                        ctypes.c_void_p(m2d.data_ptr()), st,
                                        ctypes.c_void_p(ws.data_ptr()), nws,
                                        None if status is None
                                        else ctypes.c_void_p(status.data_ptr())))
    torch.cuda.synchronize(volume.device)
    vals = int128_to_ints(m2d.cpu().numpy().view(np.int64))
    return [vals[k * npairs:(k + 1) * npairs] for k in range(P)]


def drt_plan(n: int):
    """Host helper: directions [(alpha, beta)] and the exact solve (E rows,
    D) of degree n of the discrete Radon step 2."""
    a = (ctypes.c_int * (n + 1))()
    b = (ctypes.c_int * (n + 1))()
    E = (ctypes.c_int64 * ((n + 1) * (n + 1)))()
    D = (ctypes.c_int64 * (n + 1))()
    _check(lib().dpma_drt_plan(n, a, b, E, D))
    return ([(a[j], b[j]) for j in range(n + 1)],
            [[E[r * (n + 1) + j] for j in range(n + 1)] for r in range(n + 1)], list(D))


def moments_noalloc(volume, K: int, out, dtype: int | None = None, stream=None):
    """All moments through the entry point that allocates no device memory.

    For callers that cannot call cudaMalloc; the library's workspace is a
    static 32 MiB device array shared by every call (see include/dpma.h).
    Enqueued on ``stream`` (default: torch's current stream).
    """
    dt = dtype_code(volume) if dtype is None else dtype
    L, M, N = _shape(volume)
    _check(lib().dpma_moments_noalloc(ctypes.c_void_p(volume.data_ptr()), L, M, N, dt, K,
                                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def moments_from_projections(images, L: int, M: int, N: int, K: int, dtype: int, stream=None):
    """3-D moments from projection images already on the device.

    ``images``: a CUDA tensor holding the first max(3, K+1) images back to
    back (uint32 pixels for integer dtypes, float64 for F32), as
    :func:`project` lays them out.  Returns exact ints or a float64 numpy array.
    """
    import torch
    nm = num_moments(K)
    out = torch.empty((nm, 2) if dtype != F32 else (nm,),
                      dtype=torch.int64 if dtype != F32 else torch.float64, device=images.device)
    _check(lib().dpma_moments_from_projections(ctypes.c_void_p(images.data_ptr()), L, M, N, dtype,
                                               K, ctypes.c_void_p(out.data_ptr()),
                                               _stream_ptr(stream)))
    h = out.cpu().numpy()
    return h if dtype == F32 else int128_to_ints(h)


def derived_moments(moments, K: int, dtype: int, spacing=None, stream=None) -> dict:
    """Centroid, mu_pqr, eta_pqr (Eq. 17) and physical-unit mu'_pqr (Sec. 4).

    ``moments``: the CUDA tensor a moment call returned.  Returns numpy arrays.
    """
    import torch
    nm = num_moments(K)
    out = torch.empty(3 + 3 * nm, dtype=torch.float64, device=moments.device)
    sp = (ctypes.c_double * 3)(*spacing) if spacing is not None else None
    _check(lib().dpma_derived_moments(ctypes.c_void_p(moments.data_ptr()), dtype, K, sp,
                                      ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    torch.cuda.synchronize(moments.device)
    h = out.cpu().numpy()
    return {"centroid": h[:3], "mu": h[3:3 + nm], "eta": h[3 + nm:3 + 2 * nm],
            "mu_phys": h[3 + 2 * nm:]}


# ------------------------------------------------------------ profiling


def stage_timing(enable: bool) -> None:
    """Record CUDA events around each stage of the hot-path calls."""
    _check(lib().dpma_stage_timing(1 if enable else 0))


def stage_times(reset: bool = True):
    """(ms[4], launches[4]) per stage: 0 clear, 1 projection, 2 image moments, 3 combine."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int64 * 4)()
    _check(lib().dpma_stage_times(ms, n, 1 if reset else 0))
    return list(ms), list(n)


# ------------------------------------------------------------- batches


def _descs(volumes, Ks, dtypes=None):
    """Descriptor array and output layout for CUDA volumes with orders ``Ks``."""
    n = len(volumes)
    arr = (VolumeDesc * max(1, n))()
    offsets, at = [], 0
    for i, (v, K) in enumerate(zip(volumes, Ks)):
        dt = dtype_code(v) if dtypes is None or dtypes[i] is None else dtypes[i]
        L, M, N = _shape(v)
        arr[i] = VolumeDesc(v.data_ptr(), L, M, N, dt, K, at)
        offsets.append(at)
        at += num_moments(K) * 16
    return arr, offsets, at


class Batch:
    """A planned batch of CUDA volumes (``dpma_batch_*``); ``run`` is graph-capturable."""

    def __init__(self, volumes, Ks, dtypes=None, autotune: bool = False):
        self.volumes = list(volumes)  # keep the device buffers alive
        self.Ks = list(Ks)
        self.dtypes = [dtype_code(v) if dtypes is None or dtypes[i] is None else dtypes[i]
                       for i, v in enumerate(self.volumes)]
        self.descs, self.offsets, self.out_bytes = _descs(self.volumes, self.Ks, self.dtypes)
        h = ctypes.c_void_p()
        _check(lib().dpma_batch_create(self.descs, len(self.volumes),
                                       BATCH_AUTOTUNE if autotune else 0, ctypes.byref(h)))
        self.handle = h

    def info(self, what: int) -> int:
        return lib().dpma_batch_info(self.handle, what)

    def out_buffer(self, device=None):
        import torch
        dev = device if device is not None else self.volumes[0].device
        return torch.zeros(max(16, self.out_bytes) // 8, dtype=torch.int64, device=dev)

    def run(self, out, stream=None):
        _check(lib().dpma_batch_run(self.handle, ctypes.c_void_p(out.data_ptr()),
                                    _stream_ptr(stream)))
        return out

    def status(self, stream=None):
        _check(lib().dpma_batch_status(self.handle, _stream_ptr(stream)))

    def values(self, out):
        """Per volume: exact ints (integer volumes) or float64 numpy (float32 volumes)."""
        h = out.cpu().numpy()
        res = []
        for off, K, dt in zip(self.offsets, self.Ks, self.dtypes):
            nm = num_moments(K)
            w = h[off // 8: off // 8 + 2 * nm]
            res.append(w.view(np.float64)[:nm].copy() if dt == F32 else int128_to_ints(w))
        return res

    def close(self):
        if self.handle:
            lib().dpma_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def moments_batched(volumes, Ks, dtypes=None, stream=None):
    """One-shot batch (``dpma_moments_batched``): list of per-volume moment values."""
    import torch
    descs, offsets, nbytes = _descs(volumes, Ks, dtypes)
    out = torch.zeros(max(16, nbytes) // 8, dtype=torch.int64, device=volumes[0].device)
    _check(lib().dpma_moments_batched(descs, len(volumes), ctypes.c_void_p(out.data_ptr()),
                                      _stream_ptr(stream)))
    h = out.cpu().numpy()
    res = []
    for i, (off, K) in enumerate(zip(offsets, Ks)):
        nm = num_moments(K)
        w = h[off // 8: off // 8 + 2 * nm]
        res.append(w.view(np.float64)[:nm].copy() if descs[i].dtype == F32 else int128_to_ints(w))
    return res


# -------------------------------------------------------------- serving


class Server:
    """Continuous-batching moment server (``dpma_server_*``) on the current device.

    ``submit`` takes a host numpy volume (copied before it returns) and its
    order K and gives a ticket; ``wait`` returns the moments (exact ints for
    integer volumes, float64 numpy for float32 ones).
    """

    def __init__(self, device_bytes=0, max_inflight=0, streams=0, max_group=0, max_pending=0):
        cfg = ServerConfig(device_bytes, max_inflight, streams, max_group, max_pending)
        h = ctypes.c_void_p()
        _check(lib().dpma_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._meta = {}

    def submit(self, volume: np.ndarray, K: int, dtype: int | None = None, key: int = 0) -> int:
        """Queue one request; ``key`` (non-zero) names the volume so that its
        projection images can stay resident for later requests at K or lower."""
        vol = np.ascontiguousarray(volume)
        dt = dtype_code(vol) if dtype is None else dtype
        N, M, L = vol.shape
        d = VolumeDesc(vol.ctypes.data, L, M, N, dt, K, 0)
        t = ctypes.c_uint64()
        _check(lib().dpma_server_submit_keyed(self.handle, ctypes.byref(d), key, ctypes.byref(t)))
        self._meta[t.value] = (K, dt)
        return t.value

    def poll(self, ticket: int) -> int:
        return lib().dpma_server_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_ms: int = -1):
        K, dt = self._meta[ticket]
        nm = num_moments(K)
        out = np.empty((nm, 2) if dt != F32 else (nm,), dtype=np.int64 if dt != F32 else np.float64)
        rc = lib().dpma_server_wait(self.handle, ticket, timeout_ms, ctypes.c_void_p(out.ctypes.data))
        if rc != 5:
            self._meta.pop(ticket, None)
        _check(rc)
        return out if dt == F32 else int128_to_ints(out)

    def stats(self, reset: bool = False) -> dict:
        c = ServerCounters()
        _check(lib().dpma_server_stats(self.handle, ctypes.byref(c), 1 if reset else 0))
        return {n: getattr(c, n) for n, _ in ServerCounters._fields_}

    def close(self):
        if self.handle:
            lib().dpma_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
