"""FP64 CPU oracle for the orthogonal-raster OCT/OCTA registration objective.

TEST INFRASTRUCTURE ONLY: the plain reference the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the
CUDA library in ``paper_2010_06931_gb300``.

The arithmetic lives in ``octmc_oracle.c`` (the objective, its gradient, the
pyramid, L-BFGS and the final merge) and ``octa_oracle.c`` (saccade
validity and the en-face OCTA projection, Sec. 2.2-2.3), plain C in double
precision; this module compiles them on demand, loads them with ctypes and
adds the multi-resolution driver (pyramid -> per-level eta -> L-BFGS ->
prolongation), Sec. 2.1 of Ploner et al. (arXiv 2010.06931).
"""
from .oracle import (  # noqa: F401
    OracleProblem, build, cr_weights, interp1, validity_interp, interp2, interp3, loss, chain,
    pyramid_volume, pyramid_image, pyramid_line, pyramid_time, prolong,
    lbfgs_direction, lbfgs_minimize, num_threads, LOSS_PSEUDO_HUBER, LOSS_SSD, prealign_prolong,
    saccade_validity, median3, rank_filter, percentile, bscan_median_subtract, replace_invalid, enface,
)
