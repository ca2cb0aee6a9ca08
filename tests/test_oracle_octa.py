"""Pins of the oracle's saccade validity (Sec. 2.2) and en-face OCTA
projection (Sec. 2.3): the filters against scipy.ndimage, the percentile
against numpy, closed forms on ramps, and hand-built volumes whose
validity, masks and en-face values are known."""
import numpy as np
import pytest

import oracle as O

nd = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("shape", [(5, 6, 7), (1, 9, 4), (8, 1, 1), (3, 4, 33)])
def test_median3_is_the_nearest_mode_median_filter(shape):
    A = np.random.default_rng(sum(shape)).random(shape).astype(np.float32)
    assert np.array_equal(O.median3(A), nd.median_filter(A, size=3, mode="nearest"))


def test_median3_removes_an_isolated_outlier():
    A = np.full((6, 7, 8), 0.25, np.float32)
    A[3, 4, 5] = 100.0
    assert np.all(O.median3(A) == 0.25)


@pytest.mark.parametrize("axis", [0, 1])
def test_rank_filter_is_scipy_rank_filter(axis):
    A = np.random.default_rng(7 + axis).random((20, 23, 5)).astype(np.float32)
    size = (1, 15, 1) if axis == 0 else (15, 1, 1)
    assert np.array_equal(O.rank_filter(A, axis), nd.rank_filter(A, rank=2, size=size, mode="nearest"))


def test_rank3_of_15_on_a_ramp_is_the_sample_five_back():
    w = 30
    A = np.broadcast_to(np.arange(w, dtype=np.float32)[None, :, None], (3, w, 2)).copy()
    R = O.rank_filter(A, 0)
    expect = np.clip(np.arange(w) - 5, 0, w - 1).astype(np.float32)
    assert np.array_equal(R[1, :, 0], expect)
    # along y the x-ramp is constant, so it passes unchanged
    assert np.array_equal(O.rank_filter(A, 1), A)


@pytest.mark.parametrize("n", [1, 2, 7, 1000])
def test_percentile_is_numpy_linear(n):
    x = np.random.default_rng(n).normal(size=n).astype(np.float32)
    x[: n // 3] = x[0]  # ties
    for q in (0.0, 0.05, 0.5, 0.95, 1.0):
        assert O.percentile(x, q) == pytest.approx(np.percentile(x.astype(np.float64), 100 * q), rel=1e-15, abs=0)


def test_percentile_closed_form_on_0_to_n_minus_1():
    x = np.random.default_rng(0).permutation(101).astype(np.float32)
    assert O.percentile(x, 0.05) == pytest.approx(5.0)
    assert O.percentile(x, 0.95) == pytest.approx(95.0)
    assert O.percentile(x, 0.123) == pytest.approx(12.3)


@pytest.mark.parametrize("fast_axis", [0, 1])
def test_saccade_validity_flags_a_saturated_bscan_and_two_neighbours(fast_axis):
    h, w, d = (20, 6, 4) if fast_axis == 0 else (6, 20, 4)
    A = np.full((h, w, d), 0.3, np.float32)
    if fast_axis == 0:
        A[7] = 0.9
    else:
        A[:, 7] = 0.9
    v, m = O.saccade_validity(A, fast_axis)
    assert m[7] == pytest.approx(0.9) and m[0] == pytest.approx(0.3)
    expect = np.ones(20, np.float32)
    expect[5:10] = 0
    assert np.array_equal(v, expect)


def test_saccade_validity_threshold_is_three_sigma():
    # one outlier among nb B-scans exceeds mu + 3 sigma only if nb > 10
    for nb, flagged in ((10, False), (11, True)):
        A = np.zeros((nb, 3, 2), np.float32)
        A[4] = 1.0
        v, _ = O.saccade_validity(A, 0)
        assert (v[4] == 0) == flagged, nb


@pytest.mark.parametrize("fast_axis", [0, 1])
def test_bscan_median_subtraction(fast_axis):
    E = np.random.default_rng(3).random((5, 6)).astype(np.float32)
    out = O.bscan_median_subtract(E, fast_axis)
    lines = out if fast_axis == 0 else out.T
    src = E if fast_axis == 0 else E.T
    for b in range(lines.shape[0]):
        s = np.sort(src[b].astype(np.float64))
        med = 0.5 * (s[len(s) // 2 - 1] + s[len(s) // 2]) if len(s) % 2 == 0 else s[len(s) // 2]
        assert np.allclose(lines[b], (src[b] - med).astype(np.float32), atol=1e-7)


def test_replace_invalid_takes_the_nearest_valid_bscan():
    E = np.arange(5, dtype=np.float32)[:, None].repeat(3, axis=1)
    out = O.replace_invalid(E, 0, np.array([1, 0, 0, 1, 0], np.float32))
    assert np.array_equal(out[:, 0], [0, 0, 3, 3, 3])
    out = O.replace_invalid(E.T.copy(), 1, np.array([0, 1, 0, 0, 1], np.float32))
    assert np.array_equal(out[0], [1, 1, 1, 4, 4])  # B-scan 2: tie between 1 and 3 -> 1
    assert np.array_equal(O.replace_invalid(E, 0, np.zeros(5, np.float32)), E)


@pytest.mark.parametrize("fast_axis", [0, 1])
def test_enface_of_a_hand_built_retina_slab(fast_axis):
    h, w, d = 24, 20, 40
    A = np.full((h, w, d), 0.9, np.float32)   # vitreous / choroid: high decorrelation
    S = np.zeros((h, w, d), np.float32)
    A[:, :, 10:20] = 0.1                       # retina: low decorrelation ...
    S[:, :, 10:20] = 1.0                       # ... and high OCT signal
    rng = np.random.default_rng(5)
    vessel = rng.random((h, w)) < 0.2          # single-voxel vessels in the middle of the slab
    A[:, :, 15][vessel] = 0.5
    v = np.ones(h if fast_axis == 0 else w, np.float32)
    E, info, F = O.enface(A, S, fast_axis, v, want_filtered=True)
    # the filters erase the isolated vessels: the filtered retina is 0.1, the rest 0.9
    assert np.all(F[:, :, 10:20] == np.float32(0.1)) and np.all(F[:, :, :10] == np.float32(0.9))
    assert info["p_lo"] == pytest.approx(0.1, abs=1e-7) and info["p_hi"] == pytest.approx(0.9, abs=1e-7)
    assert info["t_oct"] == pytest.approx(10.0 / d)
    assert info["kept"] == h * w * 10
    raw = (np.float64(0.1) * 9 + np.where(vessel, 0.5, 0.1)) / 10.0
    lines = raw if fast_axis == 0 else raw.T
    med = np.median(lines, axis=1, keepdims=True)
    expect = lines - med
    got = E if fast_axis == 0 else E.T
    assert np.allclose(got, expect, atol=1e-6)
