"""Pins of the oracle's final resampling and merging (Sec. 2.1, 2.5; readings
in the oracle source): zero motion gives density 1 and the plain average; a
hand-built gap gives the hand-computed density and weights; a double gap
keeps the less oversampled scan; invalid angiography B-scans drop out."""
import numpy as np
import pytest

import oracle as O
from octsynth import make_pair


def small(w=6, h=7, d=8, seed=2):
    return make_pair(w, h, d, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=seed)


def problem(p):
    return O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"])


def test_zero_motion_is_the_plain_average():
    p = small()
    P = problem(p)
    r = P.merge(np.zeros(P.shape_disp()))
    assert np.array_equal(r["density"], np.ones_like(r["density"]))
    assert np.all(r["weights"] == 0.5)
    ref = (0.5 * p["sx"].astype(np.float64) + 0.5 * p["sy"].astype(np.float64)).astype(np.float32)
    assert np.array_equal(r["merged"], ref)
    assert np.array_equal(r["cx"], p["sx"]) and np.array_equal(r["cy"], p["sy"])
    # angio: validity-weighted average of the two images at the nodes
    vx, vy = p["vx"][:, None].astype(np.float64), p["vy"][None, :].astype(np.float64)
    a = np.where(vx + vy > 0, (vx * p["ax"] + vy * p["ay"]) / np.maximum(vx + vy, 1e-300), 0.0)
    assert np.allclose(r["angio"], a, atol=1e-6)


def test_gap_density_and_weights_by_hand():
    p = small(w=4, h=6)
    P = problem(p)
    D = np.zeros(P.shape_disp())
    D[0, 1, 3, :] = -1.0  # X rows 2 and 3 both sample input row 2: a one-row gap at row 3
    r = P.merge(D, beta=2.0, tau=0.05)
    rho = r["density"][0]
    assert np.allclose(rho[2], 2.0) and np.allclose(rho[3], 2.0)
    assert np.allclose(np.delete(rho, [2, 3], axis=0), 1.0)
    wx = np.exp(-2.0) / (1.0 + np.exp(-2.0))
    assert np.allclose(r["weights"][0, 2:4], wx, rtol=1e-6) and np.allclose(r["weights"][1, 2:4], 1 - wx, rtol=1e-6)
    m = r["merged"][3].astype(np.float64)
    ref = wx * p["sx"][2].astype(np.float64) + (1 - wx) * p["sy"][3].astype(np.float64)
    assert np.allclose(m, ref, rtol=1e-6, atol=1e-7)


def test_double_gap_keeps_the_less_oversampled_scan():
    p = small(w=4, h=9)
    P = problem(p)
    D = np.zeros(P.shape_disp())
    D[0, 1, 3:6, :] = np.array([-1.0, -2.0, -3.0])[:, None]  # X rows 2..5 all sample row 2: density 4
    D[1, 1, 4:6, :] = np.array([-1.0, -2.0])[:, None]      # Y rows 3..5 sample row 3: density 3
    r = P.merge(D, beta=2.0, tau=0.05)
    # at rows 4, 5 both weights (e^-6, e^-4) are below tau: the Y scan (less oversampled) remains
    assert np.all(r["weights"][1, 4:6] == 1.0) and np.all(r["weights"][0, 4:6] == 0.0)
    # at row 3 X (e^-6) is clipped and Y (e^-4 < 0.05 too): Y kept; at row 2 only X is high
    assert np.all(r["weights"][1, 3] == 1.0)
    assert np.allclose(r["weights"][0, 2], np.exp(-6.0) / (np.exp(-6.0) + 1.0) if np.exp(-6.0) >= 0.05 else 0.0)


def test_invalid_angio_bscans_drop_out():
    p = small(w=5, h=6)
    p["vx"] = np.ones(6, np.float32)
    p["vx"][2] = 0.0
    P = problem(p)
    r = P.merge(np.zeros(P.shape_disp()))
    vy = p["vy"][None, :].astype(np.float64)
    # row 2 of X is invalid: the merged angio there is Y's where Y is valid
    ok = vy[0] > 0
    assert np.allclose(r["angio"][2, ok], p["ay"][2, ok], atol=1e-6)
