"""Pins of the oracle's pyramid, prolongation, L-BFGS direction and L-BFGS
minimiser (CPU only).

Sec. 2.1: a factor-2 multi-resolution pyramid, zero displacements at the
coarsest level, L-BFGS per level.  Readings (box mean, centre-aligned
bilinear prolongation, two-loop recursion, weak-Wolfe bisection line search
and its stopping rules) are pinned by closed forms, by properties the
mathematics fixes (the secant equation of the BFGS update) and by textbook
minimisation problems with known minimisers.
"""
import numpy as np
import pytest

import oracle as O


def test_pyramid_constant_and_mean():
    v = np.full((6, 8, 10), 0.37, dtype=np.float32)
    assert np.all(O.pyramid_volume(v) == np.float32(0.37))
    rng = np.random.default_rng(0)
    v = rng.uniform(size=(6, 8, 10)).astype(np.float32)
    out = O.pyramid_volume(v)
    assert out.shape == (3, 4, 5)
    assert out.astype(np.float64).mean() == pytest.approx(v.astype(np.float64).mean(), rel=1e-6)
    # one output by hand: the mean of its 2x2x2 block
    assert out[1, 2, 3] == np.float32(v[2:4, 4:6, 6:8].astype(np.float64).mean())


def test_pyramid_odd_sizes_repeat_the_edge():
    v = np.arange(3 * 5 * 3, dtype=np.float32).reshape(3, 5, 3)
    out = O.pyramid_volume(v)
    assert out.shape == (2, 3, 2)
    # last row/column/depth: the missing neighbour repeats the edge sample
    blk = v[2:3, 4:5, 2:3]
    assert out[1, 2, 1] == np.float32(blk.astype(np.float64).mean())
    blk = np.stack([v[2, 4, 0:2], v[2, 4, 0:2]])  # y repeats row 2, x repeats column 4
    assert out[1, 2, 0] == np.float32(blk.mean())
    img = np.arange(15, dtype=np.float32).reshape(3, 5)
    o2 = O.pyramid_image(img)
    assert o2[1, 2] == img[2, 4] and o2[0, 0] == np.float32(img[0:2, 0:2].mean())
    assert np.array_equal(O.pyramid_line(np.array([1, 3, 5], np.float32)), np.array([2, 5], np.float32))
    t = np.arange(20, dtype=np.float64).reshape(4, 5)
    assert O.pyramid_time(t)[1, 1] == t[2:4, 2:4].mean()


def test_prolong_constant_and_linear():
    wc, hc, wf, hf = 5, 4, 10, 8
    c = np.zeros((2, 3, hc, wc))
    c[0, 1] = 0.75
    f = O.prolong(c, hf, wf)
    assert np.all(f[0, 1] == 1.5) and np.all(f[1] == 0)
    # a linear coarse field a*i + b maps to a*(i - 1/2) + 2b inside the clamped border
    a, b = 0.3, -0.2
    c = np.zeros((2, 3, hc, wc))
    c[1, 0] = a * np.arange(wc)[None, :] + b
    f = O.prolong(c, hf, wf)
    i = np.arange(1, wf - 1)
    assert np.allclose(f[1, 0][:, 1:-1], a * (i - 0.5) + 2 * b, rtol=1e-14)
    assert np.allclose(f[1, 0][:, 0], 2 * b)  # clamped at the left edge


def test_lbfgs_direction_properties():
    rng = np.random.default_rng(4)
    n = 40
    g = rng.normal(size=n)
    assert np.array_equal(O.lbfgs_direction([], [], g), -g)
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)
    S = [rng.normal(size=n) for _ in range(6)]
    Y = [A @ s for s in S]
    # secant equation of the latest update: H y_k = s_k
    assert np.allclose(O.lbfgs_direction(S, Y, Y[-1]), -S[-1], rtol=1e-12, atol=1e-12)
    # H is symmetric positive definite
    u, v = rng.normal(size=n), rng.normal(size=n)
    Hu, Hv = -O.lbfgs_direction(S, Y, u), -O.lbfgs_direction(S, Y, v)
    assert np.dot(v, Hu) == pytest.approx(np.dot(u, Hv), rel=1e-12)
    assert np.dot(u, Hu) > 0
    # with one pair H = gamma-scaled BFGS update of gamma*I, gamma = s'y/y'y
    s, y = S[0], Y[0]
    gam, rho = s @ y / (y @ y), 1.0 / (s @ y)
    Vm = np.eye(n) - rho * np.outer(y, s)
    H = Vm.T @ (gam * np.eye(n)) @ Vm + rho * np.outer(s, s)
    assert np.allclose(O.lbfgs_direction([s], [y], g), -H @ g, rtol=1e-12, atol=1e-12)


def _quadratic(a, b, offset=0.0):
    # f = offset + 1/2 x'Ax - b'x with A = diag(a): minimiser b / a
    return lambda x: (offset + 0.5 * x @ (a * x) - b @ x, a * x - b)


def _rosenbrock(x):
    r = x[1] - x[0] ** 2
    return 100.0 * r * r + (1.0 - x[0]) ** 2, np.array([-400.0 * x[0] * r - 2.0 * (1.0 - x[0]), 200.0 * r])


def test_lbfgs_minimize_quadratic_reaches_the_closed_form_minimiser():
    rng = np.random.default_rng(3)
    a, b = rng.uniform(1.0, 10.0, 50), rng.normal(size=50)
    x, st = O.lbfgs_minimize(_quadratic(a, b), np.zeros(50), gtol=1e-10, ftol=0.0)
    assert st["status"] == 0 and st["iters"] < 200
    assert np.allclose(x, b / a, rtol=0.0, atol=1e-9)


def test_lbfgs_minimize_rosenbrock():
    # the textbook start (-1.2, 1); minimiser (1, 1)
    x, st = O.lbfgs_minimize(_rosenbrock, [-1.2, 1.0], gtol=1e-6, ftol=0.0, max_iter=500)
    assert st["status"] == 0, st
    assert np.allclose(x, [1.0, 1.0], rtol=0.0, atol=1e-5)
    assert st["f"] < 1e-10


def test_lbfgs_first_trial_is_a_unit_step_along_minus_g():
    # empty history: the first trial point is x0 - g0 / ||g0||_2
    rng = np.random.default_rng(5)
    a, b = rng.uniform(1.0, 4.0, 7), rng.normal(size=7)
    fg = _quadratic(a, b)
    seen = []

    def rec(x):
        seen.append(x.copy())
        return fg(x)

    x0 = rng.normal(size=7)
    O.lbfgs_minimize(rec, x0, max_iter=1, gtol=0.0, ftol=0.0)
    g0 = fg(x0)[1]
    assert np.allclose(seen[0], x0, rtol=0.0, atol=0.0)
    assert np.allclose(seen[1], x0 - g0 / np.linalg.norm(g0), rtol=0.0, atol=1e-14)


def test_lbfgs_iteration_cap_and_relative_decrease_stops():
    x, st = O.lbfgs_minimize(_rosenbrock, [-1.2, 1.0], max_iter=5, gtol=0.0, ftol=0.0)
    assert st["status"] == 1 and st["iters"] == 5
    # a large constant offset makes every relative decrease smaller than ftol:
    # the solve stops (status 0) after 3 such iterations, before max|g| <= gtol
    rng = np.random.default_rng(6)
    a, b = rng.uniform(1.0, 10.0, 20), rng.normal(size=20)
    fg = _quadratic(a, b, offset=1e12)
    x, st = O.lbfgs_minimize(fg, np.zeros(20), gtol=1e-6, ftol=1e-9)
    assert st["status"] == 0 and st["iters"] == 3
    assert np.abs(fg(x)[1]).max() > 1e-6
    # with the relative-decrease test off the same problem runs on to the gradient test
    x, st = O.lbfgs_minimize(_quadratic(a, b), np.zeros(20), gtol=1e-6, ftol=0.0)
    assert st["status"] == 0 and st["iters"] > 3 and np.abs(_quadratic(a, b)(x)[1]).max() <= 1e-6
