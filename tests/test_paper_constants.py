"""The constants the paper fixes (tests/golden/paper_constants.txt, each with
its citation) are the defaults of the library, of its binding and of the
oracle, and the oracle's projection steps follow them."""
import ctypes
import inspect
import os
import shutil

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def constants():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_constants.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("="))
            out[k] = float(v)
    return out


K = constants()


def test_oracle_defaults():
    sig = inspect.signature(O.OracleProblem.__init__).parameters
    assert sig["eps_h"].default == K["eps_h"]
    assert sig["delta0"].default == K["delta0"]
    assert sig["alpha"].default == K["alpha"]
    ef = inspect.signature(O.enface).parameters
    assert ef["q_lo"].default == K["quantile_low"] and ef["q_hi"].default == K["quantile_high"]
    assert ef["thresh"].default == K["mask_threshold"]
    rf = inspect.signature(O.rank_filter).parameters
    assert rf["width"].default == K["rank_width"] and rf["rank"].default == K["rank"]


def test_binding_defaults():
    import paper_2010_06931_gb300 as octmc
    sig = inspect.signature(octmc.Problem.__init__).parameters
    assert sig["eps_h"].default == K["eps_h"] and sig["delta0"].default == K["delta0"]
    assert sig["alpha"].default == K["alpha"]
    ef = inspect.signature(octmc.enface).parameters
    assert ef["q_lo"].default == K["quantile_low"] and ef["q_hi"].default == K["quantile_high"]
    assert ef["thresh"].default == K["mask_threshold"]


def test_library_defaults():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_2010_06931_gb300 import _native as N
    d = N.Desc()
    N.lib().octmc_desc_defaults(ctypes.byref(d))
    assert d.eps_h == K["eps_h"] and d.delta0 == K["delta0"] and d.alpha == K["alpha"]


def test_validity_dilation_and_median_radius_follow_the_constants():
    nb, r = 24, int(K["validity_dilation"])
    A = np.full((nb, 5, 4), 0.3, np.float32)
    A[11] = 0.95  # one saturated B-scan among 24: well above mu + 3 sigma
    v, m = O.saccade_validity(A, 0)
    assert m[11] > m.mean() + K["validity_sigmas"] * m.std()
    assert np.array_equal(np.where(v == 0)[0], np.arange(11 - r, 12 + r))
    # a median of radius 1 removes a single outlier but keeps a 2-voxel-thick slab
    B = np.zeros((7, 7, 9), np.float32)
    B[3, 3, 4] = 1.0
    B[:, :, 6:8] = 1.0
    M = O.median3(B)
    assert M[3, 3, 4] == 0.0 and np.all(M[:, :, 6:8] == 1.0)
