"""Seeded synthetic OCTA (amplitude decorrelation) volumes with their OCT
volumes, for the saccade detection and en-face projection steps (Sec. 2.2,
2.3).  Rendering only: no projection arithmetic here.

The decorrelation model follows the paper's description of its input: high
values where the OCT signal is low (vitreous above the retina, deep choroid
below it), low values in the retinal tissue between vessels, vessel trees
(widths 1-3 px) as high values in ``n_slabs`` thin depth slabs inside the
retina, additive noise, and ``n_saturated`` B-scans (with their neighbours)
saturated by saccadic motion (uniformly high over the whole B-scan).
"""
import math

import numpy as np
from scipy.special import ndtr

from .generator import _Retina, _rasterise, _sample_map, _vessel_segments


def make_octa_scan(w, h, d, fast_axis=0, n_layers=8, n_slabs=2, n_saturated=2, seed=0):
    """Returns dict(A=[h][w][d] decorrelation, S=[h][w][d] OCT (float32),
    saturated=sorted B-scan indices, fast_axis)."""
    rng = np.random.default_rng(seed)
    retina = _Retina(rng, w, h, d, n_layers)
    slab_maps = [_rasterise(_vessel_segments(rng, w, h), w, h) for _ in range(n_slabs)]
    nb = h if fast_axis == 0 else w
    sat = np.sort(rng.choice(nb, size=min(n_saturated, nb), replace=False)) if n_saturated else np.zeros(0, int)
    srng = np.random.default_rng(seed * 104729 + 17)
    A = np.empty((h, w, d), np.float32)
    S = np.empty((h, w, d), np.float32)
    z = np.arange(d, dtype=np.float32)
    for j0 in range(0, h, 16):
        j1 = min(h, j0 + 16)
        jj, ii = np.meshgrid(np.arange(j0, j1, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
        clean = retina.render(ii, jj, np.zeros_like(ii), d)
        S[j0:j1] = clean * srng.rayleigh(math.sqrt(2.0 / math.pi), size=clean.shape).astype(np.float32)
        surf = retina.surfaces(ii, jj).astype(np.float32)
        dec = np.float32(0.05) + np.float32(0.85) * np.exp(-clean / np.float32(0.12))
        dec += np.float32(0.6) * ndtr((z - surf[..., -1:] - 8.0) / 3.0).astype(np.float32)  # deep choroid
        for s, mp in enumerate(slab_maps):  # vessel slabs between the upper surfaces
            centre = 0.5 * (surf[..., s + 1] + surf[..., s + 2])
            prof = np.exp(-((z - centre[..., None]) ** 2) / (2.0 * 2.0 ** 2)).astype(np.float32)
            dec += np.float32(0.7) * _sample_map(mp, ii, jj)[..., None] * prof
        dec += srng.normal(0.0, 0.03, size=dec.shape).astype(np.float32)
        A[j0:j1] = np.clip(dec, 0.0, 1.0)
    for b in sat:
        noise = np.clip(0.9 + srng.normal(0.0, 0.03, size=(w if fast_axis == 0 else h, d)), 0.0, 1.0)
        if fast_axis == 0:
            A[b] = noise.astype(np.float32)
        else:
            A[:, b] = noise.astype(np.float32)
    return dict(A=A, S=S, saturated=sat, fast_axis=fast_axis)
