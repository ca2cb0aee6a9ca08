"""Analytic test objects shared by the oracle pins and the GPU parity tests.

Inputs only: smooth objects with compact support rendered at integer
positions, so that integer shifts of them are exact (no interpolation).
"""
import numpy as np


def _bump(u, c, r):
    """cos^2 window: C^1, exactly zero for |u - c| >= r."""
    a = np.clip((u - c) / r, -1.0, 1.0)
    return np.cos(0.5 * np.pi * a) ** 2


def blob_object(shape, margin, seed=0, n_blobs=12):
    """Callable O(x, y, z) that is exactly 0 within `margin` of the transverse and axial edges."""
    h, w, d = shape
    rng = np.random.default_rng(seed)
    blobs = []
    for _ in range(n_blobs):
        r = rng.uniform(2.5, 4.0, size=3)
        c = [rng.uniform(margin + r[0], w - 1 - margin - r[0]),
             rng.uniform(margin + r[1], h - 1 - margin - r[1]),
             rng.uniform(margin + r[2], d - 1 - margin - r[2])]
        blobs.append((c, r, rng.uniform(0.3, 1.0)))

    def O(x, y, z):
        out = np.zeros(np.broadcast(x, y, z).shape)
        for c, r, a in blobs:
            out += a * _bump(x, c[0], r[0]) * _bump(y, c[1], r[1]) * _bump(z, c[2], r[2])
        return out
    return O


def render(O, shape, shift):
    """Volume [h][w][d] with V[j][i][k] = O(i + sx, j + sy, k + sz)."""
    h, w, d = shape
    j, i, k = np.meshgrid(np.arange(h), np.arange(w), np.arange(d), indexing="ij")
    return O(i + shift[0], j + shift[1], k + shift[2]).astype(np.float32)


def raster_times(w, h, flyback):
    j, i = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    return j * (w + flyback) + i, i * (h + flyback) + j


def wave_object(shape, margin, seed=0, n_waves=24, min_wavelength=5.0, taper=4.0):
    """Callable O(x, y, z): a random sum of plane waves (wavelengths >= min_wavelength px)
    multiplied by a C^1 window that is exactly 0 within `margin` of every edge and 1 more
    than `margin + taper` inside.  Every interior A-scan sees structure along all axes."""
    h, w, d = shape
    rng = np.random.default_rng(seed)
    kmax = 2 * np.pi / min_wavelength
    waves = []
    for _ in range(n_waves):
        k = rng.normal(size=3)
        k *= rng.uniform(0.3, 1.0) * kmax / np.linalg.norm(k)
        waves.append((k, rng.uniform(0, 2 * np.pi), rng.uniform(0.5, 1.0)))

    def win(u, n):
        lo = np.clip((u - margin) / taper, 0.0, 1.0)
        hi = np.clip((n - 1 - margin - u) / taper, 0.0, 1.0)
        return np.sin(0.5 * np.pi * lo) ** 2 * np.sin(0.5 * np.pi * hi) ** 2

    def O(x, y, z):
        x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
        s = np.zeros(x.shape)
        for k, ph, a in waves:
            s += a * np.cos(k[0] * x + k[1] * y + k[2] * z + ph)
        return (1.0 + 0.25 * s) * win(x, w) * win(y, h) * win(z, d)
    return O
