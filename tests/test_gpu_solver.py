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
