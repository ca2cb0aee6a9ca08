"""Rough axial prealignment on the GPU (stage 1 of Sec. 2.1) against the
oracle: the induced field, the stage-1 objective and its parameter gradient,
a level solve at a fixed iteration budget, and recovery of known per-B-scan
offsets and tilts through the full coarse-to-fine solve."""
import numpy as np
import pytest

import oracle as O
from octsynth import make_config
from tests.test_oracle_prealign import render, unseen_free

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def inputs(p):
    return [p[k] for k in ("sx", "sy", "tx", "ty", "ax", "ay", "vx", "vy")]


def random_prm(P, seed):
    rng = np.random.default_rng(seed)
    prm = rng.normal(0.0, 0.8, P.n_prealign())
    prm[P.h:2 * P.h] *= 0.03
    prm[2 * P.h + P.w:] *= 0.03
    return prm


@pytest.mark.parametrize("loss", [0, 1])
def test_objective_and_gradient_match_the_oracle(loss):
    import paper_2010_06931_gb300 as octmc
    p, cfg = make_config("c1")
    G = octmc.Problem(*inputs(p), loss=loss, alpha=0.3)
    C = O.OracleProblem(*inputs(p), loss=loss, alpha=0.3)
    prm = random_prm(C, 3 + loss)
    pd = torch.from_numpy(prm).cuda()
    D = G.prealign_disp(0, pd).cpu().numpy()
    assert np.allclose(D, C.prealign_disp(prm), rtol=0, atol=1e-12)
    g = torch.empty_like(pd)
    f = G.prealign_eval(0, pd, g)
    fo, go, _ = C.prealign_eval(prm)
    assert abs(f - fo) <= 1e-5 * abs(fo)
    gn = g.cpu().numpy()
    assert np.linalg.norm(gn - go) <= 1e-4 * np.linalg.norm(go)
    assert G.prealign_eval(0, pd) == f  # objective alone: same value


def test_level_solve_matches_the_oracle_at_a_fixed_budget():
    import paper_2010_06931_gb300 as octmc
    p, cfg = make_config("c1")
    kw = dict(alpha=0.1, max_iter=10)
    G = octmc.Problem(*inputs(p), **kw)
    C = O.OracleProblem(*inputs(p), alpha=0.1)
    pd = torch.zeros(G.prealign_size(0), dtype=torch.float64, device="cuda")
    st = G.prealign_level(0, pd)
    po, so = C.prealign_level(np.zeros(C.n_prealign()), max_iter=10)
    dg = G.prealign_disp(0, pd).cpu().numpy()
    do = C.prealign_disp(po)
    rms = float(np.sqrt(np.mean((dg - do) ** 2)))
    assert rms <= 0.05, rms
    assert st["iters"] == so["iters"]
    assert st["f"] == pytest.approx(so["f"], rel=1e-4)


def test_full_prealignment_recovers_known_offsets_and_tilts():
    import paper_2010_06931_gb300 as octmc
    w, h, d = 32, 28, 48
    j, i = np.arange(h), np.arange(w)
    zX = 1.5 * np.sin(2 * np.pi * 0.6 * j / h) + 0.4
    zY = 1.2 * np.cos(2 * np.pi * 0.5 * i / w) - 0.3
    tX, tY = unseen_free(0.03 * np.cos(2 * np.pi * j / h), 0.02 * np.sin(2 * np.pi * i / w))
    sx, sy, tx, ty = render(w, h, d, zX, tX, zY, tY)
    G = octmc.Problem(sx, sy, tx, ty, alpha=0.01, levels=2, max_iter=300)
    prm, disp, stats = G.prealign_full()
    prm = prm.cpu().numpy()
    aX, gX, aY, gY = prm[:h], prm[h:2 * h], prm[2 * h:2 * h + w], prm[2 * h + w:]
    cx, cy = 0.5 * (w - 1), 0.5 * (h - 1)
    rel = (aX[:, None] + gX[:, None] * (i[None, :] - cx)) - (aY[None, :] + gY[None, :] * (j[:, None] - cy))
    true = (zX[:, None] + tX[:, None] * (i[None, :] - cx)) - (zY[None, :] + tY[None, :] * (j[:, None] - cy))
    assert np.sqrt(np.mean((rel - true) ** 2)) < 0.02
    assert np.abs(gX - tX).max() < 0.002 and np.abs(gY - tY).max() < 0.002
    D = disp.cpu().numpy()
    assert np.allclose(D[0, 2] - D[1, 2], rel, atol=1e-9)
    assert [s["level"] for s in stats] == [1, 0]


def test_repeatable():
    import paper_2010_06931_gb300 as octmc
    p, cfg = make_config("c1")
    G = octmc.Problem(*inputs(p), max_iter=15, levels=1)
    a = G.prealign_full()[0].cpu().numpy()
    b = G.prealign_full()[0].cpu().numpy()
    assert np.array_equal(a, b)
