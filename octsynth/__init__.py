"""Seeded synthetic orthogonal-raster OCT/OCTA scan pairs.

Input generator shared by the tests, the smoke check and the benchmark.  It
renders inputs only: it contains none of the registration method's
arithmetic (no interpolation of volumes, no loss, no objective).

The real scans of the paper (500x500 A-scans x 465 samples, Sec. 3.3; wide
field 800x800x433) are clinical data and not available; these volumes stand
in for them with the same structure:

* a retina of ``n_layers`` Gaussian-smoothed intensity bands on curved
  surfaces (a quadratic bowl plus one Gaussian drusen-like bump of 6 px),
  normalised to [0, 1] and multiplied by unit-mean Rayleigh speckle,
  independently per acquired voxel and per scan;
* an en-face angiography image: random branching vessel trees (widths
  1-3 px) in ``n_slabs`` depth slabs, projected by the depth mean;
* eye motion per acquisition slot: Gaussian random-walk drift, Poisson-timed
  transverse saccades and a 1 Hz axial sinusoid of 2 px amplitude;
* B-scans within 2 of a saccade carry saturated angiography and validity 0
  (Sec. 2.2); as in the paper's projection step they are then replaced by the
  nearest valid B-scan (Sec. 2.3);
* sampling-time maps: raster order with a flyback of 25 % of a B-scan
  (500 x 500 x 5 repeats at 400 kHz take about 3.9 s, Sec. 3.3).

``make_octa_scan`` renders one scan's 3-D angiography (amplitude
decorrelation) and OCT volumes for the saccade detection and en-face
projection steps (Sec. 2.2, 2.3).

All arrays are in the common frame: volumes ``[h][w][d]`` (depth contiguous),
images and time maps ``[h][w]``; ``vx`` has one value per row (the X-fast
scan's B-scans are rows), ``vy`` one per column.
"""
from .generator import (CONFIGS, fingerprint, fingerprints_match, make_config, make_pair,  # noqa: F401
                        true_displacement)
from .octa import make_octa_scan  # noqa: F401
