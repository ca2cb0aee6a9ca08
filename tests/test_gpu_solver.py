"""Stopping paths of the device-resident level solve (GPU only), against the
FP64 oracle's minimiser with the same constants (Sec. 2.1, L-BFGS solve):
the iteration cap and the gradient test at the start point."""
import numpy as np
import pytest

import oracle as O
from octsynth import make_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problems(p, **kw):
    import paper_2010_06931_gb300 as octmc
    G = octmc.Problem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"], **kw)
    C = O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"])
    return G, C


def test_iteration_cap_stops_every_level_with_status_1():
    p, _ = make_config("c1")
    G, C = problems(p, levels=3, max_iter=7)
    D, st = G.solve_full()
    Dc, stc = C.solve_full(3, max_iter=7)
    assert [s["status"] for s in st] == [1, 1, 1], st
    assert [s["iters"] for s in st] == [7, 7, 7], st
    assert [s["status"] for s in stc] == [1, 1, 1], stc
    assert [s["iters"] for s in stc] == [7, 7, 7], stc
    # the start evaluation and at least one trial per iteration
    assert all(s["evals"] >= 8 for s in st), st
    assert torch.isfinite(D).all()


def test_gradient_test_stops_at_the_start_point():
    # gtol above max |grad| at the start: every level stops at its start
    # point (status 0, no iteration, one evaluation) and returns it; the
    # coarsest level starts from zero and the prolongation of zero is zero
    p, _ = make_config("c1")
    G, C = problems(p, levels=2, gtol=1e30)
    D, st = G.solve_full()
    Dc, stc = C.solve_full(2, gtol=1e30)
    assert [s["status"] for s in st] == [0, 0], st
    assert [s["iters"] for s in st] == [0, 0], st
    assert [s["evals"] for s in st] == [1, 1], st
    assert [s["status"] for s in stc] == [0, 0], stc
    assert [s["iters"] for s in stc] == [0, 0], stc
    assert float(D.abs().max()) == 0.0
    assert float(np.abs(Dc).max()) == 0.0


def clean_c1():
    return make_config("c1", speckle=False, angio_noise=False, n_saccades=0)


def test_persistent_level_kernel_converges_to_the_oracle_minimum():
    # every level solved by the persistent cooperative kernel (opt-in): the
    # same algorithm as the graph-driven loop, other reduction orders
    p, cfg = clean_c1()
    G, _ = problems(p, levels=3, loss=1, ftol=1e-6, persistent_ascans=1 << 20)
    D, st = G.solve_full()
    C = O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"], loss=1)
    Dc, stc = C.solve_full(3, ftol=1e-6)
    D = D.cpu().numpy()
    rms = float(np.sqrt(((D - Dc) ** 2).mean()))
    P0 = C.pyramid(1)[0]
    P0.eta = stc[-1]["eta"]
    f_g = P0.eval(D, grad=False)[0]
    print("persistent levels, clean c1 (SSD): GPU vs oracle %.4f px, FP64 objective %.9g / %.9g, iters %s / %s"
          % (rms, f_g, stc[-1]["f"], [s["iters"] for s in st], [s["iters"] for s in stc]))
    assert [s["status"] for s in st] == [0, 0, 0], st
    assert rms <= 0.05
    assert f_g <= stc[-1]["f"] * (1.0 + 1e-4)


def test_persistent_level_kernel_iteration_cap():
    p, _ = make_config("c1")
    G, _ = problems(p, levels=2, max_iter=7, persistent_ascans=1 << 20)
    D, st = G.solve_full()
    assert [s["status"] for s in st] == [1, 1], st
    assert [s["iters"] for s in st] == [7, 7], st
    assert torch.isfinite(D).all()


def test_bounded_grid_barrier_reports_timeout():
    # a barrier waiting for one block more than the grid has cannot complete:
    # every wait runs out (about 2 s), the call reports TIMEOUT, nothing
    # traps, and the device stays usable
    from paper_2010_06931_gb300 import _native as N
    L = N.lib()
    assert L.octmc_barrier_selftest(0) == 0
    assert L.octmc_barrier_selftest(1) == -5
    assert L.octmc_barrier_selftest(0) == 0
    p, _ = make_config("c1")
    G, C = problems(p)
    D = torch.zeros(G.disp_shape(0), dtype=torch.float64, device="cuda")
    assert np.isfinite(G.eval_objective_grad(0, D))
