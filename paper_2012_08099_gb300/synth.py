"""Seeded synthetic volumes (input generation only, no moment arithmetic).

The paper measures on MRI/CT volumes (Sec. 4, brain MRI 512x512x230) and on
1 MB - 1 GB volumes from public volume datasets (Sec. 5, Table 1) that are
not available here.  These generators stand in for them; both the CUDA path
and the CPU oracle consume the same arrays.

Every array is ``V[z, y, x]`` (shape ``(N, M, L)``, x fastest) and is drawn
from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_volume(shape, dtype, seed: int, low=None, high=None) -> np.ndarray:
    """I.i.d. uniform voxels.

    uint8/uint16 default to the full range of the type; float32 defaults to
    [0, 1000).  ``shape`` is (N, M, L).
    """
    g = _rng(seed)
    dt = np.dtype(dtype)
    if dt.kind == "u":
        lo = 0 if low is None else low
        hi = (np.iinfo(dt).max + 1) if high is None else high
        return g.integers(lo, hi, size=shape, dtype=dt)
    if dt == np.float32:
        lo = 0.0 if low is None else low
        hi = 1000.0 if high is None else high
        return (g.random(size=shape, dtype=np.float32) * np.float32(hi - lo) + np.float32(lo))
    raise TypeError(f"unsupported dtype {dt}")


def _uniform_rotation(g: np.random.Generator) -> np.ndarray:
    """Rotation matrix from a uniformly distributed unit quaternion."""
    u1, u2, u3 = g.random(3)
    a = math.sqrt(1 - u1) * math.sin(2 * math.pi * u2)
    b = math.sqrt(1 - u1) * math.cos(2 * math.pi * u2)
    c = math.sqrt(u1) * math.sin(2 * math.pi * u3)
    d = math.sqrt(u1) * math.cos(2 * math.pi * u3)
    w, x, y, z = d, a, b, c
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def ct_phantom_u16(
    L: int,
    M: int,
    N: int,
    seed: int,
    n_ellipsoids: int = 20,
    semi_axes=(10.0, 80.0),
    density=(200, 4000),
    background=(0, 50),
    noise_sigma: float = 20.0,
    vmax: int = 4095,
    axis_scale: float = 1.0,
) -> np.ndarray:
    """CT-like uint16 phantom.

    Background i.i.d. uniform integers in ``background``; ``n_ellipsoids``
    randomly rotated (uniform quaternion) ellipsoids with semi-axes uniform in
    ``semi_axes`` (times ``axis_scale``), centres uniform in the box and
    densities uniform in ``density``; overlaps add.  Then N(0, sigma^2) noise,
    rounded to nearest and clipped to [0, vmax].
    """
    g = _rng(seed)
    acc = g.integers(background[0], background[1] + 1, size=(N, M, L)).astype(np.float32)
    for _ in range(n_ellipsoids):
        ax = g.uniform(semi_axes[0], semi_axes[1], size=3) * axis_scale
        ctr = g.uniform([0, 0, 0], [L, M, N])
        rot = _uniform_rotation(g)
        dens = float(g.integers(density[0], density[1] + 1))
        r = float(ax.max())
        lo = np.maximum(np.floor(ctr - r).astype(int), 0)
        hi = np.minimum(np.ceil(ctr + r).astype(int) + 1, [L, M, N])
        if np.any(hi <= lo):
            continue
        xs = np.arange(lo[0], hi[0], dtype=np.float32) - np.float32(ctr[0])
        ys = np.arange(lo[1], hi[1], dtype=np.float32) - np.float32(ctr[1])
        zs = np.arange(lo[2], hi[2], dtype=np.float32) - np.float32(ctr[2])
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        rt = rot.T.astype(np.float32)
        q = np.zeros(X.shape, dtype=np.float32)
        for k in range(3):
            u = rt[k, 0] * X + rt[k, 1] * Y + rt[k, 2] * Z
            q += (u / np.float32(ax[k])) ** 2
        acc[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += np.where(q <= 1.0, np.float32(dens), 0)
    acc += g.standard_normal(size=acc.shape, dtype=np.float32) * np.float32(noise_sigma)
    np.rint(acc, out=acc)
    np.clip(acc, 0, vmax, out=acc)
    return acc.astype(np.uint16)


def mri_like_f32(
    L: int,
    M: int,
    N: int,
    seed: int,
    n_blobs: int = 50,
    sigma=(5.0, 60.0),
    amplitude=(50.0, 1000.0),
    noise_sigma: float = 10.0,
) -> np.ndarray:
    """MRI-like float32 volume.

    Sum of ``n_blobs`` isotropic Gaussian blobs (sigma uniform in ``sigma``,
    amplitude uniform in ``amplitude``, centres uniform in the box) with
    Rician noise: sqrt((S + n1)^2 + n2^2), n1, n2 ~ N(0, noise_sigma^2).
    Each blob is an outer product of three 1-D Gaussians, so the clean
    signal is one (N x B) @ (B x M*L) product.
    """
    g = _rng(seed)
    sig = g.uniform(sigma[0], sigma[1], size=n_blobs)
    amp = g.uniform(amplitude[0], amplitude[1], size=n_blobs)
    ctr = g.uniform([0, 0, 0], [L, M, N], size=(n_blobs, 3))

    def gauss(n, c):
        t = np.arange(n, dtype=np.float64)[None, :] - c[:, None]
        return np.exp(-0.5 * (t / sig[:, None]) ** 2)

    gx = gauss(L, ctr[:, 0]).astype(np.float32)
    gy = gauss(M, ctr[:, 1]).astype(np.float32)
    gz = (gauss(N, ctr[:, 2]) * amp[:, None]).astype(np.float32)
    yx = (gy[:, :, None] * gx[:, None, :]).reshape(n_blobs, M * L)
    s = (gz.T @ yx).reshape(N, M, L)
    del yx
    n1 = g.standard_normal(size=s.shape, dtype=np.float32)
    n1 *= np.float32(noise_sigma)
    s += n1
    np.square(s, out=s)
    n1[...] = g.standard_normal(size=s.shape, dtype=np.float32)
    n1 *= np.float32(noise_sigma)
    np.square(n1, out=n1)
    s += n1
    del n1
    np.sqrt(s, out=s)
    return s


def roi_mask_u8(L: int, M: int, N: int, fill: float) -> np.ndarray:
    """Binary {0,1} mask holding one axis-aligned ellipsoid centred in its box.

    The ellipsoid's semi-axes are proportional to the half sizes of the box;
    its scale is chosen so that the fraction of voxels inside is ``fill``
    (fills above pi/6 give ellipsoids clipped by the box).  The scale is the
    ``fill``-quantile of the voxels' normalised radii.
    """
    xs = (np.arange(L) + 0.5 - L / 2) / (L / 2)
    ys = (np.arange(M) + 0.5 - M / 2) / (M / 2)
    zs = (np.arange(N) + 0.5 - N / 2) / (N / 2)
    rho = zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2
    flat = np.sort(rho, axis=None)
    k = min(max(int(round(fill * flat.size)), 1), flat.size) - 1
    return (rho <= flat[k]).astype(np.uint8)


@dataclass
class RoiBatch:
    shapes: list  # (N, M, L) per ROI
    volumes: list  # uint8 arrays


def roi_batch(count: int, seed: int, size_range=(8, 96), fill_range=(0.2, 0.8)) -> RoiBatch:
    """``count`` binary ROI masks with per-axis sizes log-uniform in ``size_range``."""
    g = _rng(seed)
    lo, hi = math.log(size_range[0]), math.log(size_range[1])
    shapes, vols = [], []
    for _ in range(count):
        L, M, N = (int(round(math.exp(v))) for v in g.uniform(lo, hi, size=3))
        fill = float(g.uniform(fill_range[0], fill_range[1]))
        vols.append(roi_mask_u8(L, M, N, fill))
        shapes.append((N, M, L))
    return RoiBatch(shapes, vols)


@dataclass
class Request:
    arrival_s: float
    K: int
    volume: np.ndarray


def serving_stream(
    count: int,
    seed: int,
    rate_hz: float = 200.0,
    xy_range=(32, 512),
    z_range=(32, 300),
    orders=(3, 4, 6, 8),
) -> list:
    """Poisson request stream of uint16 phantoms with mixed sizes and orders.

    Inter-arrival times are exponential with mean 1/rate_hz; x and y sizes
    log-uniform in ``xy_range``, z log-uniform in ``z_range``; the order K is
    uniform over ``orders``; each volume is a :func:`ct_phantom_u16` with
    semi-axes scaled by min(dim)/256.
    """
    g = _rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(g.exponential(1.0 / rate_hz))
        L = int(round(math.exp(g.uniform(math.log(xy_range[0]), math.log(xy_range[1])))))
        M = int(round(math.exp(g.uniform(math.log(xy_range[0]), math.log(xy_range[1])))))
        N = int(round(math.exp(g.uniform(math.log(z_range[0]), math.log(z_range[1])))))
        K = int(orders[int(g.integers(0, len(orders)))])
        vol = ct_phantom_u16(L, M, N, seed=seed * 100003 + i, axis_scale=min(L, M, N) / 256.0)
        out.append(Request(t, K, vol))
    return out
