"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only input generation (random fields, blurring, rank
spacing); none of the persistence arithmetic.  Both the CUDA path's tests and
the oracle's tests draw their inputs from here.

The paper's synthetic inputs are i.i.d. uniform images (Sec. 5.1); its real
2D and 3D datasets are not available, and white noise blurred with a Gaussian
stands in for them (smooth fields with few critical points).

Recipes (numpy PCG64 ``default_rng(seed)``):
  uniform(shape, seed)       : rng.random(shape, float32) in [0, 1)
  blurred(shape, sigma, seed): rng.standard_normal(shape) (float64), separable
                               Gaussian blur, truncated at 4 sigma, reflect
                               boundary, min-max normalised to [0, 1], float32
  quantised(x)               : floor(x * 255 + 0.5) stored as float32 (256
                               levels, heavy ties)
  rank_spaced(x)             : each value replaced by rank * 2**-8 (ranks by
                               value then linear index); exact in float32 for
                               fewer than 2**24 pixels, same refined order as x
  batch(seed)                : 64 2D images with sides drawn from [128, 1024]
                               and 8 volumes with sides drawn from [64, 192];
                               blurred fields (sigma 4 in 2D, 2 in 3D) from
                               seeds 1000 + i, then rank-spaced.
"""
from __future__ import annotations

import numpy as np

try:  # scipy is present on both machines; the numpy fallback is equivalent, only slower
    from scipy.ndimage import gaussian_filter1d as _gf1d
except Exception:  # pragma: no cover
    _gf1d = None


def uniform(shape, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).random(tuple(shape), dtype=np.float32)


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(4.0 * sigma + 0.5)
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def _blur_axis(a: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    if _gf1d is not None:
        return _gf1d(a, sigma, axis=axis, mode="reflect", truncate=4.0)
    k = _gauss_kernel(sigma)
    r = len(k) // 2
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    p = np.pad(a, pad, mode="symmetric")
    out = np.zeros_like(a)
    n = a.shape[axis]
    for i, w in enumerate(k):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(i, i + n)
        out += w * p[tuple(sl)]
    return out


def blurred(shape, sigma: float, seed: int = 0) -> np.ndarray:
    a = np.random.default_rng(seed).standard_normal(tuple(shape))
    for ax in range(a.ndim):
        a = _blur_axis(a, sigma, ax)
    lo, hi = a.min(), a.max()
    a = (a - lo) / (hi - lo) if hi > lo else np.zeros_like(a)
    return a.astype(np.float32)


def quantised(x: np.ndarray) -> np.ndarray:
    return np.floor(np.asarray(x, dtype=np.float64) * 255.0 + 0.5).astype(np.float32)


def rank_spaced(x: np.ndarray) -> np.ndarray:
    flat = np.asarray(x, dtype=np.float32).ravel()
    order = np.lexsort((np.arange(flat.size), flat))  # by value, then linear index
    ranks = np.empty(flat.size, dtype=np.int64)
    ranks[order] = np.arange(flat.size)
    return (ranks.astype(np.float64) * 2.0 ** -8).astype(np.float32).reshape(np.shape(x))


def batch_shapes(seed: int = 0, n2d: int = 64, n3d: int = 8):
    rng = np.random.default_rng(seed)
    s2 = [tuple(int(v) for v in rng.integers(128, 1025, 2)) for _ in range(n2d)]
    rng = np.random.default_rng(seed)
    s3 = [tuple(int(v) for v in rng.integers(64, 193, 3)) for _ in range(n3d)]
    return s2, s3


def batch(seed: int = 0, n2d: int = 64, n3d: int = 8, scale: float = 1.0):
    """The batched workload: a list of float32 arrays (2D images, then volumes).

    `scale` < 1 shrinks every side (at least 2) for quick tests with the same recipe.
    """
    s2, s3 = batch_shapes(seed, n2d, n3d)
    items = []
    for i, s in enumerate(s2 + s3):
        s = tuple(max(2, int(round(v * scale))) for v in s)
        sigma = 4.0 if len(s) == 2 else 2.0
        items.append(rank_spaced(blurred(s, sigma, 1000 + i)))
    return items


# Named workloads used by the tests and the benchmark.
def config(name: str):
    if name == "2d_64_uniform":
        return [uniform((64, 64), 0)]
    if name == "2d_2048_grf":
        g = blurred((2048, 2048), 8.0, 0)
        return [g, quantised(g)]
    if name == "3d_128":
        return [uniform((128, 128, 128), 0), blurred((128, 128, 128), 2.0, 1)]
    if name == "3d_512_blurred":
        return [blurred((512, 512, 512), 3.0, 0)]
    if name == "batch":
        return batch(0)
    raise KeyError(name)
