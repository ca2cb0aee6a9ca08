"""Pins of the oracle's objective and gradient (CPU only).

Objective: f = eta S^str + S^ang/eta + alpha R + M (Eq. 1, 5, 6, 9), with the
residual of Eq. 2, the loss of Eq. 4, validity and delta of Eq. 7-8 and eta of
Eq. 10.  Pinned by invariants and closed forms: zero at identical inputs, the
delta_0 = 0 reduction, the X<->Y transpose symmetry, central differences,
the eta equalisation property, exact zeros at a known translation, closed
forms of R and M, and known synthetic motion.
"""
import numpy as np
import pytest

import oracle as O
from octsynth import make_pair, make_config, true_displacement
from tests.analytic import raster_times, render, wave_object


def small_pair(seed=5, w=9, h=7, d=11):
    return make_pair(w, h, d, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0,
                     drift_sigma=0.05, seed=seed)


def problem(p, **kw):
    return O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"], **kw)


def test_identical_inputs_give_exact_zero():
    p = small_pair()
    P = O.OracleProblem(p["sx"], p["sx"].copy(), p["tx"], p["ty"], p["ax"], p["ax"].copy(),
                        p["vx"], p["vy"])
    P.eta = 0.7
    f, g, terms = P.eval(np.zeros(P.shape_disp()))
    assert f == 0.0 and np.all(g == 0.0) and np.all(terms[:5] == 0.0)


def test_delta0_zero_removes_angio():
    p = small_pair()
    rng = np.random.default_rng(0)
    D = rng.normal(0, 0.6, (2, 3, 7, 9))
    P1 = problem(p, delta0=0.0)
    q = dict(p)
    q["ax"] = rng.uniform(size=p["ax"].shape).astype(np.float32)
    q["ay"] = rng.uniform(size=p["ay"].shape).astype(np.float32)
    P2 = problem(q, delta0=0.0)
    P1.eta = P2.eta = 1.3
    f1, g1, t1 = P1.eval(D)
    f2, g2, t2 = P2.eval(D)
    assert f1 == f2 and np.array_equal(g1, g2) and t1[1] == 0.0
    # and with delta = 0 and eta = 1 the structural term is the basic Eq. 3 sum
    P3 = problem(p, delta0=0.0, alpha=0.0)
    P3.mu = 0.0
    f3, _, t3 = P3.eval(D)
    ref = 0.0
    for j in range(7):
        for i in range(9):
            for k in range(11):
                a, _ = O.interp3(p["sx"], i + D[0, 0, j, i], j + D[0, 1, j, i], k + D[0, 2, j, i])
                b, _ = O.interp3(p["sy"], i + D[1, 0, j, i], j + D[1, 1, j, i], k + D[1, 2, j, i])
                ref += O.loss(a - b, 1e-3)[0]
    assert f3 == pytest.approx(ref, rel=1e-12)


def transpose_problem(p):
    """The same acquisition seen with the x and y axes exchanged: X and Y swap roles."""
    T3 = lambda v: np.ascontiguousarray(np.transpose(v, (1, 0, 2)))
    T2 = lambda v: np.ascontiguousarray(v.T)
    return dict(sx=T3(p["sy"]), sy=T3(p["sx"]), ax=T2(p["ay"]), ay=T2(p["ax"]),
                vx=p["vy"].copy(), vy=p["vx"].copy(), tx=T2(p["ty"]), ty=T2(p["tx"]))


def transpose_disp(D):
    """D'[X] = transposed D[Y] with x/y components exchanged, and vice versa."""
    out = np.empty((2, 3) + D.shape[3:1:-1])
    for V, W in ((0, 1), (1, 0)):
        out[V, 0] = D[W, 1].T
        out[V, 1] = D[W, 0].T
        out[V, 2] = D[W, 2].T
    return out


@pytest.mark.parametrize("loss", [O.LOSS_PSEUDO_HUBER, O.LOSS_SSD])
def test_xy_transpose_symmetry(loss):
    p = small_pair()
    q = transpose_problem(p)
    rng = np.random.default_rng(1)
    D = rng.normal(0, 0.8, (2, 3, 7, 9))
    P, Q = problem(p, loss=loss), problem(q, loss=loss)
    P.eta = Q.eta = 0.9
    fp, gp, tp = P.eval(D)
    fq, gq, tq = Q.eval(transpose_disp(D))
    assert fq == pytest.approx(fp, rel=1e-12)
    assert np.allclose(tq[:4], tp[:4], rtol=1e-12)
    assert np.allclose(gq, transpose_disp(gp), rtol=1e-10, atol=1e-12)
    # eta itself is symmetric too
    assert Q.compute_eta(transpose_disp(D)) == pytest.approx(P.compute_eta(D), rel=1e-12)


@pytest.mark.parametrize("eps_h,loss,tol", [(0.1, O.LOSS_PSEUDO_HUBER, 1e-7),
                                             (1e-3, O.LOSS_PSEUDO_HUBER, 1e-4),
                                             (1e-3, O.LOSS_SSD, 1e-7)])
def test_gradient_central_differences(eps_h, loss, tol):
    p = small_pair(seed=7, w=6, h=5, d=8)
    P = problem(p, eps_h=eps_h, loss=loss, eps_r=0.3, alpha=0.7, mu=0.02)
    P.eta = 0.8
    rng = np.random.default_rng(2)
    D = rng.normal(0, 0.7, P.shape_disp())
    f, g, _ = P.eval(D)
    scale = np.abs(g).max()
    for ix in np.ndindex(*D.shape):
        # Richardson-extrapolated central difference
        fd = []
        for hstep in (2e-5, 1e-5):
            Dp, Dm = D.copy(), D.copy()
            Dp[ix] += hstep
            Dm[ix] -= hstep
            fd.append((P.eval(Dp, grad=False)[0] - P.eval(Dm, grad=False)[0]) / (2 * hstep))
        fdr = (4 * fd[1] - fd[0]) / 3
        assert abs(fdr - g[ix]) <= tol * scale + 1e-7 * abs(f) * 1e-3, (ix, fdr, g[ix])


def test_eta_equalises_the_two_terms():
    p = small_pair(seed=9)
    P = problem(p, delta0=0.5)
    D0 = np.random.default_rng(3).normal(0, 0.3, P.shape_disp())
    eta = P.compute_eta(D0)
    P.eta = eta
    _, _, t = P.eval(D0, grad=False)
    # Eq. 10 makes eta S^str_0.5 = S^ang_0.5 / eta (both at the geometric mean)
    assert eta * t[0] == pytest.approx(t[1] / eta, rel=1e-12)
    # delta_0 is 0.5 in Eq. 10 whatever the configured delta_0
    P2 = problem(p, delta0=0.2)
    assert P2.compute_eta(D0) == eta
    # no angiography: eta = 1
    P3 = O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"])
    assert P3.compute_eta(D0) == 1.0


def test_chain_of_raster_time_maps():
    w, h, fb = 5, 4, 3
    tx, ty = raster_times(w, h, fb)
    order, omega = O.chain(tx)
    assert np.array_equal(order, np.arange(w * h))  # X-fast: row-major raster
    expect = np.ones(w * h - 1)
    expect[w - 1::w] = 1.0 / (1 + fb)  # row end -> next row start spans the flyback
    assert np.allclose(omega, expect, rtol=1e-15)
    order, omega = O.chain(ty)
    j, i = np.divmod(order, w)
    assert np.array_equal(i, np.repeat(np.arange(w), h)) and np.array_equal(j, np.tile(np.arange(h), w))


def test_regulariser_and_mean_closed_forms():
    w, h, d = 5, 4, 6
    tx, ty = raster_times(w, h, 3)
    s = np.zeros((h, w, d), dtype=np.float32)
    P = O.OracleProblem(s, s, tx, ty, alpha=1.0, eps_r=0.5, mu=0.25)
    D = np.zeros(P.shape_disp())
    a = 0.2
    D[0, 0] = a * np.arange(w)[None, :]  # X volume, x component: ramp along the fast axis
    D[1, 2] = 1.5                        # Y volume, z component: constant
    f, g, t = P.eval(D)
    Lr = lambda x: O.loss(x, 0.5)[0]
    # every pair of the time chain carries the level depth d (the per-A-scan
    # scale of the data term, as in Eq. 6); flyback steps weigh 1/(1 + 3)
    R_ref = d * (h * (w - 1) * Lr(a) + (h - 1) * Lr(-a * (w - 1)) / 4.0)
    assert t[2] == pytest.approx(R_ref, rel=1e-13)
    sx_sum = D[0, 0].sum()
    M_ref = 0.25 * (sx_sum ** 2 + (1.5 * w * h) ** 2)
    assert t[3] == pytest.approx(M_ref, rel=1e-13)
    assert f == pytest.approx(R_ref + M_ref, rel=1e-13)
    # dM/dd = 2 mu (sum of the component) for every entry of that component
    assert np.allclose(g[1, 2], 2 * 0.25 * 1.5 * w * h, rtol=1e-13)


def translation_problem(loss, eps_h):
    shape = (24, 26, 20)
    h, w, d = shape
    obj = wave_object(shape, margin=2, seed=1, taper=3, min_wavelength=10)
    t = np.array([2.0, -2.0, 2.0])
    sx, sy = render(obj, shape, -t / 2), render(obj, shape, t / 2)
    tx, ty = raster_times(w, h, 4)
    # R carries the depth d; alpha = 0.1 / d keeps the regulariser at 0.1 per pair
    P = O.OracleProblem(sx, sy, tx, ty, alpha=0.1 / d, eps_h=eps_h, eps_r=0.5, loss=loss)
    sol = np.zeros(P.shape_disp())
    for c in range(3):
        sol[0, c], sol[1, c] = t[c] / 2, -t[c] / 2
    return P, sol


@pytest.mark.parametrize("loss,eps_h", [(O.LOSS_SSD, 1e-3), (O.LOSS_PSEUDO_HUBER, 1e-3)])
def test_translation_is_an_exact_global_minimum(loss, eps_h):
    P, sol = translation_problem(loss, eps_h)
    f, g, t = P.eval(sol)
    # every term is >= 0, and all vanish at the shift: a global minimum
    assert f == 0.0 and np.all(g == 0.0)
    f0, _, _ = P.eval(np.zeros(P.shape_disp()), grad=False)
    assert f0 > 1.0


def test_translation_recovered_by_the_solver():
    # the data term fixes the relative displacement d^X - d^Y; the common mode is
    # only held by R and M and converges slowly, so it is checked loosely
    P, sol = translation_problem(O.LOSS_SSD, 1e-3)
    D, st = P.solve_level(np.zeros(P.shape_disp()), max_iter=600, gtol=1e-12, ftol=1e-16)
    rel = (D[0] - D[1]) - (sol[0] - sol[1])
    assert np.abs(rel[:, 4:-4, 4:-4]).max() < 0.03
    assert np.sqrt(((D - sol) ** 2).mean()) < 0.6
    assert st["f"] < 1e-3 * P.eval(np.zeros(P.shape_disp()), grad=False)[0]


def test_delta_stays_between_zero_and_delta0():
    # Sec. 2.2: delta is delta_0 where both scans are valid, 0 where one is
    # invalid and fades smoothly in between.  Every A-scan of a 1 x h grid
    # samples the X validity at the same position u (dy^X = u - j), with
    # identical volumes and equal displacements (S^str = 0) and angio images
    # 1 and 0 (L(R_a) = L(1) everywhere), so S^ang = h d delta(u) L(1).
    h, d = 6, 4
    s = np.zeros((h, 1, d), dtype=np.float32)
    tx, ty = raster_times(1, h, 1)
    vx = np.array([1, 1, 0, 0, 1, 1], dtype=np.float32)
    P = O.OracleProblem(s, s, tx, ty, np.ones((h, 1)), np.zeros((h, 1)), vx, np.ones(1), alpha=0.0, mu=0.0)
    L1 = O.loss(1.0, 1e-3)[0]
    for u in np.linspace(-1.0, 6.0, 57):
        D = np.zeros(P.shape_disp())
        D[:, 1, :, 0] = u - np.arange(h)
        _, _, t = P.eval(D, grad=False)
        delta = t[1] / (h * d * L1)
        assert -1e-15 <= delta <= 0.5 + 1e-15
        if 2.0 <= u <= 3.0:
            assert delta == 0.0  # between two invalid B-scans
        if u <= 1.0 or u >= 4.0:
            assert delta == pytest.approx(0.5, abs=1e-15)


def test_known_motion_recovered_from_zero():
    # The method's purpose (Sec. 2.1, Eq. 1): from zero displacement, the
    # coarse-to-fine L-BFGS solve recovers known motion.  Noise-free rendering
    # of the c1 scan pair (drift and the 1 Hz axial sinusoid; no speckle, no
    # angiography noise, no saccades, so the truth is unique), the paper's
    # alpha = 0.1 and delta_0 = 0.5, three levels, each solved to the ftol
    # stopping rule.  Bar: 0.2 px RMS against the true field (A-scans more
    # than 4 px from the border), 0.2 px on the data-determined relative mode.
    p, cfg = make_config("c1", speckle=False, angio_noise=False, n_saccades=0)
    T, mask = true_displacement(p, cfg["w"], cfg["h"])
    mask[:, :4] = mask[:, -4:] = False
    mask[:, :, :4] = mask[:, :, -4:] = False
    m6 = np.broadcast_to(mask[:, None], T.shape)
    assert np.sqrt((T[m6] ** 2).mean()) > 1.0  # the motion to recover
    P = problem(p)
    D, stats = P.solve_full(3, max_iter=3000, ftol=1e-6)
    assert [s["status"] for s in stats] == [0, 0, 0]
    assert np.sqrt(((D - T)[m6] ** 2).mean()) < 0.2
    both = mask[0] & mask[1]
    rel = (D[0] - D[1]) - (T[0] - T[1])
    assert np.sqrt((rel[:, both] ** 2).mean()) < 0.2


def test_known_motion_minimum_is_near_the_truth():
    # synthetic motion with speckle: starting at the true displacement, the
    # minimiser stays close to it (a sign or index error would push it away)
    p, cfg = make_config("c1")
    T, mask = true_displacement(p, cfg["w"], cfg["h"])
    P = problem(p, alpha=1.0)
    P.eta = P.compute_eta(np.zeros(P.shape_disp()))
    D, st = P.solve_level(T, max_iter=60, set_eta=False)
    m6 = np.broadcast_to(mask[:, None], T.shape)
    assert np.sqrt(((D - T)[m6] ** 2).mean()) < 0.35
    assert st["f"] < P.eval(T, grad=False)[0]
