"""Pins of the oracle's rough axial prealignment (stage 1 of Sec. 2.1;
readings in the oracle source): the induced displacement and the tilt term
in closed form, the parameter gradient against central differences, the
level-to-level prolongation, and recovery of known per-B-scan axial offsets
and tilts from a pair rendered with them."""
import numpy as np
import pytest
from scipy.special import ndtr

import oracle as O


def profile(z, d):
    """A smooth layered depth profile (no speckle)."""
    out = np.zeros_like(z)
    for c, a in ((0.3 * d, 0.6), (0.45 * d, -0.3), (0.6 * d, 0.9), (0.75 * d, -0.8)):
        out += a * ndtr((z - c) / 1.5)
    return out.astype(np.float32)


def unseen_free(tX, tY):
    """Tilts with the three unseen modes (common x tilt, y tilt, twist)
    projected out, so the tilt term does not bias their recovery."""
    h, w = len(tX), len(tY)
    oy, ox = np.arange(h) - 0.5 * (h - 1), np.arange(w) - 0.5 * (w - 1)
    tX = tX - tX.mean()
    tY = tY - tY.mean()
    k = (tX @ oy + tY @ ox) / (oy @ oy + ox @ ox)
    return tX - k * oy, tY - k * ox


def render(w, h, d, zX, tX, zY, tY):
    k = np.arange(d, dtype=np.float64)
    cx, cy = 0.5 * (w - 1), 0.5 * (h - 1)
    jj, ii = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    shX = zX[jj] + tX[jj] * (ii - cx)
    shY = zY[ii] + tY[ii] * (jj - cy)
    sx = profile(k[None, None, :] - shX[..., None], d)
    sy = profile(k[None, None, :] - shY[..., None], d)
    tx = jj * (w + 4.0) + ii
    ty = ii * (h + 4.0) + jj
    return sx, sy, tx, ty


def problem(w=20, h=16, d=40, seed=0, **kw):
    rng = np.random.default_rng(seed)
    sx = rng.random((h, w, d)).astype(np.float32)
    sy = rng.random((h, w, d)).astype(np.float32)
    jj, ii = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    return O.OracleProblem(sx, sy, jj * (w + 4.0) + ii, ii * (h + 4.0) + jj, **kw)


def test_induced_displacement_is_offset_plus_tilt():
    P = problem()
    w, h = P.w, P.h
    prm = np.random.default_rng(1).normal(size=P.n_prealign())
    D = P.prealign_disp(prm)
    aX, tX, aY, tY = prm[:h], prm[h:2 * h], prm[2 * h:2 * h + w], prm[2 * h + w:]
    i, j = 7, 5
    assert D[0, 2, j, i] == pytest.approx(aX[j] + tX[j] * (i - 0.5 * (w - 1)))
    assert D[1, 2, j, i] == pytest.approx(aY[i] + tY[i] * (j - 0.5 * (h - 1)))
    assert np.all(D[:, :2] == 0)


def test_tilt_term_closed_form():
    P = problem()
    w, h = P.w, P.h
    prm = np.zeros(P.n_prealign())
    prm[h:2 * h] = 0.03
    prm[2 * h + w:] = -0.01
    # a common x tilt tau of the frame (X tilts tau, Y offsets tau (i - cx))
    # costs what M charges for the same displacement energy: 2 w h tau^2 vx
    vx, vy = (w * w - 1) / 12.0, (h * h - 1) / 12.0
    _, _, t = P.prealign_eval(prm)
    assert t[3] == pytest.approx(2 * w * h * (0.03 ** 2 * vx + 0.01 ** 2 * vy), rel=1e-13)
    # the twist kappa (X tilts kappa (j - cy), Y tilts kappa (i - cx)):
    # energy 2 w h kappa^2 vx vy
    oy, ox = np.arange(h) - 0.5 * (h - 1), np.arange(w) - 0.5 * (w - 1)
    prm[:] = 0.0
    prm[h:2 * h] = 0.002 * oy
    prm[2 * h + w:] = 0.002 * ox
    _, _, t = P.prealign_eval(prm)
    assert t[3] == pytest.approx(2 * w * h * 0.002 ** 2 * vx * vy, rel=1e-12)
    # and M matches it for the induced displacements of a shift
    prm[:] = 0.0
    prm[:h] = 0.7
    prm[2 * h:2 * h + w] = 0.7
    _, _, t = P.prealign_eval(prm)
    assert t[2] == pytest.approx(2 * w * h * 0.7 ** 2, rel=1e-12) and t[3] == 0.0


def test_gradient_matches_central_differences():
    P = problem(loss=O.LOSS_SSD, alpha=0.3)
    rng = np.random.default_rng(2)
    prm = rng.normal(0.0, 0.7, P.n_prealign())
    prm[P.h:2 * P.h] *= 0.05
    prm[2 * P.h + P.w:] *= 0.05
    f, g, _ = P.prealign_eval(prm)
    for idx in rng.choice(P.n_prealign(), 12, replace=False):
        e = np.zeros_like(prm)
        e[idx] = 1e-5
        fd = (P.prealign_eval(prm + e, False)[0] - P.prealign_eval(prm - e, False)[0]) / 2e-5
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-6 * abs(f)), idx


def test_prolongation_doubles_offsets_and_keeps_tilts():
    wc, hc, wf, hf = 5, 4, 10, 7
    c = np.concatenate([np.full(hc, 1.5), np.full(hc, 0.02), np.full(wc, -0.5), np.full(wc, 0.01)])
    f = O.prealign_prolong(c, wc, hc, wf, hf)
    assert np.allclose(f[:hf], 3.0) and np.allclose(f[hf:2 * hf], 0.02)
    assert np.allclose(f[2 * hf:2 * hf + wf], -1.0) and np.allclose(f[2 * hf + wf:], 0.01)
    # a ramp: fine b at (b - 1/2)/2 on the coarse grid, clamped
    c = np.concatenate([np.arange(hc, dtype=float), np.zeros(hc), np.zeros(wc), np.zeros(wc)])
    f = O.prealign_prolong(c, wc, hc, wf, hf)
    expect = 2.0 * np.clip(0.5 * np.arange(hf) - 0.25, 0, hc - 1)
    assert np.allclose(f[:hf], expect)


def test_recovers_known_offsets_and_tilts():
    w, h, d = 32, 28, 48
    j, i = np.arange(h), np.arange(w)
    zX = 1.5 * np.sin(2 * np.pi * 0.6 * j / h) + 0.4
    zY = 1.2 * np.cos(2 * np.pi * 0.5 * i / w) - 0.3
    tX, tY = unseen_free(0.03 * np.cos(2 * np.pi * j / h), 0.02 * np.sin(2 * np.pi * i / w))
    sx, sy, tx, ty = render(w, h, d, zX, tX, zY, tY)
    P = O.OracleProblem(sx, sy, tx, ty, alpha=0.01)
    prm, stats = P.prealign_full(2, max_iter=300)
    aX, gX, aY, gY = prm[:h], prm[h:2 * h], prm[2 * h:2 * h + w], prm[2 * h + w:]
    # relative axial alignment per A-scan: d^X - d^Y must equal zX_j - zY_i (+ the tilt parts)
    rel = (aX[:, None] + gX[:, None] * (i[None, :] - 0.5 * (w - 1))) - (aY[None, :] + gY[None, :] * (j[:, None] - 0.5 * (h - 1)))
    true = (zX[:, None] + tX[:, None] * (i[None, :] - 0.5 * (w - 1))) - (zY[None, :] + tY[None, :] * (j[:, None] - 0.5 * (h - 1)))
    err = np.sqrt(np.mean((rel - true) ** 2))
    assert err < 0.02, err
    assert np.abs(gX - tX).max() < 0.002 and np.abs(gY - tY).max() < 0.002
