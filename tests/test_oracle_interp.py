"""Pins of the oracle's interpolator and loss (CPU only).

The paper asks for "Hermitian interpolation" with continuous first
derivatives (Sec. 2.1, Eq. 2; Sec. 2.2, Eq. 7).  Reading: cubic Hermite with
central-difference tangents (Catmull-Rom), edge samples replicated.  These
tests pin it against properties the mathematics fixes, not against a retyped
formula: interpolation at the nodes, exact reproduction of quadratics,
hand-derived values at the edges, C^1 continuity, and consistency of the
analytic derivative with central differences.
"""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("t", [0.0, 0.1, 0.37, 0.5, 0.81, 0.999])
def test_weights_partition_and_moments(t):
    w, dw = O.cr_weights(t)
    # partition of unity and first moment (linear precision): sum w = 1, sum w n = t
    n = np.array([-1.0, 0.0, 1.0, 2.0])
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs((w * n).sum() - t) < 1e-15
    # second moment: cubic convolution with a = -1/2 reproduces quadratics
    assert abs((w * n ** 2).sum() - t * t) < 1e-15
    assert abs(dw.sum()) < 1e-15
    assert abs((dw * n).sum() - 1.0) < 1e-14
    assert abs((dw * n ** 2).sum() - 2 * t) < 1e-14


def test_weights_closed_forms():
    # t = 0: interpolation at the node
    w, dw = O.cr_weights(0.0)
    assert np.array_equal(w, [0.0, 1.0, 0.0, 0.0])
    # derivative at a node is the central difference (p_{n+1} - p_{n-1}) / 2
    assert np.allclose(dw, [-0.5, 0.0, 0.5, 0.0], atol=0, rtol=0)
    # t = 1/2: the classic (-1, 9, 9, -1)/16 midpoint stencil
    w, dw = O.cr_weights(0.5)
    assert np.allclose(w, np.array([-1, 9, 9, -1]) / 16.0, atol=1e-16)
    # its derivative stencil (1, -11, 11, -1)/8: exact for p_n = n (gives 1) and n^2 (gives 2t = 1)
    assert np.allclose(dw, np.array([1, -11, 11, -1]) / 8.0, atol=1e-16)


def test_interp1_nodes_quadratic_and_edges():
    rng = np.random.default_rng(1)
    v = rng.normal(size=11).astype(np.float32)
    for i in range(11):
        val, _ = O.interp1(v, float(i))
        assert val == float(v[i])
    q = (0.3 * np.arange(11) ** 2 - 1.1 * np.arange(11) + 0.7).astype(np.float32)
    for u in [1.0, 2.25, 4.5, 7.9, 8.999]:  # stencil inside the grid
        val, du = O.interp1(q, u)
        assert abs(val - (0.3 * u * u - 1.1 * u + 0.7)) < 1e-5
        assert abs(du - (0.6 * u - 1.1)) < 1e-5
    # edge replication, value by hand: u = -0.5 uses p0, p0, p0, p1 with (-1, 9, 9, -1)/16
    val, du = O.interp1(v, -0.5)
    assert abs(val - ((17.0 / 16.0) * v[0] - (1.0 / 16.0) * v[1])) < 1e-7
    # constant beyond -1 and at/after n
    for u in (-1.0, -3.7, -1e9):
        val, du = O.interp1(v, u)
        assert val == pytest.approx(float(v[0]), abs=1e-7) and du == pytest.approx(0.0, abs=1e-7)
    for u in (11.0, 12.2, 1e9):
        val, du = O.interp1(v, u)
        assert val == pytest.approx(float(v[-1]), abs=1e-7) and du == pytest.approx(0.0, abs=1e-7)


def test_interp1_c1_continuity_at_nodes():
    rng = np.random.default_rng(2)
    v = rng.normal(size=9).astype(np.float32)
    for n in range(1, 8):
        _, dl = O.interp1(v, n - 1e-9)
        _, dr = O.interp1(v, n + 1e-9)
        assert abs(dl - dr) < 1e-6
        assert abs(dr - 0.5 * (float(v[n + 1]) - float(v[n - 1]))) < 1e-6


def test_interp2_interp3_separable_quadratic():
    # a separable quadratic in each axis is reproduced exactly, with its gradient
    h, w, d = 9, 10, 11
    qx = lambda x: 0.2 * x * x - x + 1.0
    qy = lambda y: -0.1 * y * y + 0.5 * y + 2.0
    qz = lambda z: 0.05 * z * z + 0.3 * z - 1.0
    j, i, k = np.meshgrid(np.arange(h), np.arange(w), np.arange(d), indexing="ij")
    vol = (qx(i) * qy(j) * qz(k)).astype(np.float64)
    img = (qx(i[:, :, 0]) * qy(j[:, :, 0])).astype(np.float64)
    rng = np.random.default_rng(3)
    for _ in range(20):
        x, y, z = rng.uniform(1, w - 2.01), rng.uniform(1, h - 2.01), rng.uniform(1, d - 2.01)
        val, g = O.interp3(vol.astype(np.float32), x, y, z)
        ref = qx(x) * qy(y) * qz(z)
        assert abs(val - ref) < 2e-5 * max(1, abs(ref))
        gref = [(0.4 * x - 1) * qy(y) * qz(z), qx(x) * (-0.2 * y + 0.5) * qz(z), qx(x) * qy(y) * (0.1 * z + 0.3)]
        assert np.allclose(g, gref, rtol=1e-4, atol=1e-4)
        val2, g2 = O.interp2(img.astype(np.float32), x, y)
        assert abs(val2 - qx(x) * qy(y)) < 2e-5 * max(1, abs(qx(x) * qy(y)))
        assert np.allclose(g2, gref[:2] / np.array(qz(z)), rtol=1e-4, atol=1e-4)


def test_interp3_gradient_vs_central_differences():
    rng = np.random.default_rng(4)
    vol = rng.normal(size=(6, 7, 8)).astype(np.float32)
    for _ in range(30):
        x, y, z = rng.uniform(-1.5, 7.5), rng.uniform(-1.5, 6.5), rng.uniform(-1.5, 8.5)
        _, g = O.interp3(vol, x, y, z)
        e = 1e-6
        fd = [(O.interp3(vol, x + e, y, z)[0] - O.interp3(vol, x - e, y, z)[0]) / (2 * e),
              (O.interp3(vol, x, y + e, z)[0] - O.interp3(vol, x, y - e, z)[0]) / (2 * e),
              (O.interp3(vol, x, y, z + e)[0] - O.interp3(vol, x, y, z - e)[0]) / (2 * e)]
        assert np.allclose(g, fd, atol=1e-6)


def test_interp3_brute_force_tensor_product():
    # the 3-D interpolant equals 1-D interpolation applied axis by axis
    rng = np.random.default_rng(5)
    vol = rng.normal(size=(5, 6, 7)).astype(np.float32)
    x, y, z = 2.3, 1.7, 4.6
    val, _ = O.interp3(vol, x, y, z)
    # along z for each (j, i), then x per row, then y
    col = np.array([[O.interp1(vol[j, i], z)[0] for i in range(6)] for j in range(5)], dtype=np.float64)
    row = np.array([O.interp1(col[j].astype(np.float32), x)[0] for j in range(5)])
    # interp1 takes float32 samples: compare with a tolerance covering that rounding
    ref = O.interp1(row.astype(np.float32), y)[0]
    assert abs(val - ref) < 1e-5


def test_loss_closed_forms():
    eps = 1e-3
    assert O.loss(0.0, eps) == (0.0, 0.0)
    v, dv = O.loss(eps, eps)
    assert v == pytest.approx(eps * (np.sqrt(2.0) - 1.0), rel=1e-14)
    assert dv == pytest.approx(1.0 / np.sqrt(2.0), rel=1e-14)
    # far from 0 the pseudo-Huber loss approaches |x| - eps (Eq. 4)
    v, dv = O.loss(-2.0, eps)
    assert v == pytest.approx(2.0 - eps, abs=1e-6) and dv == pytest.approx(-1.0, abs=1e-6)
    # symmetric; the stable form equals the defining form where the latter is accurate
    for x in (3e-4, 2e-3, 0.05, 0.7):
        a, da = O.loss(x, eps)
        b, db = O.loss(-x, eps)
        assert a == b and da == -db
        assert a == pytest.approx(eps * (np.sqrt(1 + (x / eps) ** 2) - 1), rel=1e-12)
    # squared-difference loss
    assert O.loss(0.3, eps, O.LOSS_SSD) == pytest.approx((0.09, 0.6), rel=1e-15)
    # small-|x| limit of pseudo-Huber is x^2 / (2 eps), i.e. SSD / (2 eps)
    v, _ = O.loss(1e-7, eps)
    assert v == pytest.approx(1e-14 / (2 * eps), rel=1e-6)


# ---------------------------------------------------------------- validity (Eq. 7, 8)
# Reading: the validity line is resampled by the cubic Hermite interpolant
# with zero node tangents, so that delta stays within [0, delta_0]: 0 where a
# scan is invalid, delta_0 where both are valid, a smooth fade in between
# (Sec. 2.2).  Pinned by the properties that fix it: it passes through the
# nodes with zero slope there (C^1 across nodes), never leaves the range of
# its two nodes, is the Hermite basis function 3 t^2 - 2 t^3 on a unit step,
# and replicates the edge samples.

def test_validity_nodes_slope_and_edges():
    rng = np.random.default_rng(3)
    v = rng.uniform(0, 1, 9).astype(np.float32)
    for n in range(9):
        val, du = O.validity_interp(v, float(n))
        assert val == float(v[n]) and du == 0.0
    for u in (-3.0, -1.0, -0.25):
        assert O.validity_interp(v, u) == (float(v[0]), 0.0)
    for u in (8.0, 8.6, 11.0):
        assert O.validity_interp(v, u) == (float(v[8]), 0.0)


def test_validity_step_is_the_hermite_basis_and_never_overshoots():
    v = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
    for t in np.linspace(0.0, 1.0, 41):
        val, du = O.validity_interp(v, 2.0 + t)
        assert val == pytest.approx(t * t * (3 - 2 * t), abs=1e-15)
        assert du == pytest.approx(6 * t * (1 - t), abs=1e-14)
    # the Catmull-Rom interpolant of the same step dips below 0 between the zeros
    assert O.interp1(v, 1.5)[0] < -0.05
    rng = np.random.default_rng(4)
    w = (rng.uniform(size=30) > 0.4).astype(np.float32)
    for u in rng.uniform(-2, 31, 400):
        val, _ = O.validity_interp(w, u)
        b = int(np.clip(np.floor(u), 0, 29))
        lo, hi = sorted((float(w[b]), float(w[min(b + 1, 29)])))
        assert lo <= val <= hi


def test_validity_derivative_matches_central_differences():
    rng = np.random.default_rng(5)
    v = rng.uniform(0, 1, 12).astype(np.float32)
    for u in rng.uniform(0.05, 10.95, 50):
        if abs(u - round(u)) < 1e-3:
            continue
        e = 1e-6
        fd = (O.validity_interp(v, u + e)[0] - O.validity_interp(v, u - e)[0]) / (2 * e)
        assert O.validity_interp(v, u)[1] == pytest.approx(fd, rel=1e-7, abs=1e-9)
