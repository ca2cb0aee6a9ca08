"""torch.autograd over the objective (GPU): central finite differences on
random displacement components, the oracle's full gradient, both modes, and
a batch of independent pairs."""
import numpy as np
import pytest

import oracle as O
from octsynth import make_config, make_pair, true_displacement

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problems(p, **kw):
    import paper_2010_06931_gb300 as octmc
    G = octmc.Problem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"], **kw)
    C = O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"])
    return G, C


@pytest.fixture(scope="module")
def c4():
    p, cfg = make_config("c4")
    T, _ = true_displacement(p, cfg["w"], cfg["h"])
    return p, cfg, T


@pytest.mark.parametrize("mode", ["save", "recompute"])
def test_autograd_matches_oracle_and_finite_differences(c4, mode):
    from paper_2010_06931_gb300.autograd import objective
    p, cfg, T = c4
    G, C = problems(p)
    eta = 0.9
    G.set_eta(0, eta)
    C.eta = eta
    # a displacement away from the optimum: the truth plus noise
    D0 = T + np.random.default_rng(3).normal(0.0, 0.4, T.shape)
    D = torch.from_numpy(D0).cuda().requires_grad_(True)
    f = objective(G, 0, D, mode)
    f.backward()
    g = D.grad.cpu().numpy()
    fc, gc, _ = C.eval(D0)
    assert abs(f.item() - fc) <= 1e-5 * abs(fc)
    assert np.linalg.norm(g - gc) <= 1e-4 * np.linalg.norm(gc)
    # central differences, step 1e-3 px, 64 random components.  Evaluations
    # are bitwise reproducible, so the unperturbed A-scans cancel exactly and
    # the difference only carries the perturbed A-scan's float rounding.
    rng = np.random.default_rng(4)
    hstep = 1e-3
    scale = np.abs(gc).mean()
    errs = []
    with torch.no_grad():
        for _ in range(64):
            ix = tuple(int(rng.integers(0, s)) for s in D0.shape)
            Dp = torch.from_numpy(D0).cuda()
            Dp[ix] += hstep
            fp = G.eval_objective_grad(0, Dp)
            Dp[ix] -= 2 * hstep
            fm = G.eval_objective_grad(0, Dp)
            fd = (fp - fm) / (2 * hstep)
            errs.append(abs(fd - g[ix]) / (abs(g[ix]) + scale))
    errs = np.array(errs)
    assert np.median(errs) < 1e-3 and errs.max() < 2e-2, errs


def test_batch_of_pairs_with_recomputation():
    import paper_2010_06931_gb300 as octmc
    from paper_2010_06931_gb300.autograd import batch_objective
    pairs = [make_pair(48, 40, 64, n_layers=6, n_slabs=2, n_saccades=2, max_saccade=4.0,
                       drift_sigma=0.03, seed=100 + b) for b in range(16)]
    probs = [octmc.Problem(q["sx"], q["sy"], q["tx"], q["ty"], q["ax"], q["ay"], q["vx"], q["vy"])
             for q in pairs]
    rng = np.random.default_rng(5)
    Ds = [torch.from_numpy(rng.normal(0.0, 0.5, (2, 3, 40, 48))).cuda().requires_grad_(True) for _ in pairs]
    total = batch_objective(probs, 0, Ds, mode="recompute")
    total.backward()
    ref = 0.0
    for b in (0, 7, 15):  # spot-check three members against the oracle
        q = pairs[b]
        C = O.OracleProblem(q["sx"], q["sy"], q["tx"], q["ty"], q["ax"], q["ay"], q["vx"], q["vy"])
        fc, gc, _ = C.eval(Ds[b].detach().cpu().numpy())
        gb = Ds[b].grad.cpu().numpy()
        assert np.linalg.norm(gb - gc) <= 1e-4 * np.linalg.norm(gc)
    fsum = sum(P.eval_objective_grad(0, D.detach()) for P, D in zip(probs, Ds))
    assert total.item() == pytest.approx(fsum, rel=1e-12)
    # the batched evaluation (one launch per kernel for all 16 pairs) gives each
    # member exactly its single evaluation, in both modes
    singles, sgrads = [], []
    for P, D in zip(probs, Ds):
        g = torch.empty_like(D)
        singles.append(P.eval_objective_grad(0, D.detach(), g))
        sgrads.append(g)
    bgrads = [torch.empty_like(D) for D in Ds]
    fb = octmc.eval_batch(probs, [0] * len(probs), [D.detach() for D in Ds], bgrads)
    assert fb == singles
    assert all(torch.equal(a, b) for a, b in zip(bgrads, sgrads))
    Es = [D.detach().clone().requires_grad_(True) for D in Ds]
    total_s = batch_objective(probs, 0, Es, mode="save")
    total_s.backward()
    assert total_s.item() == total.item()
    assert all(torch.equal(E.grad, D.grad) for E, D in zip(Es, Ds))
