"""octmc_data_term_static: the data-term entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (allocator callbacks,
frameworks owning all device memory), so it keeps its scratch in a fixed
device array inside the library.  This test calls it through the C ABI and
checks its sums and gradient against the regular entry point
(octmc_eval_terms with the regulariser and mean term switched off) on two
calls in a row, which share that array.  Kept in its own file, collected
last.
"""
import ctypes as C

import numpy as np
import pytest

from octsynth import make_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4


def test_static_entry_point_matches_the_problem_api():
    import paper_2010_06931_gb300 as octmc
    from paper_2010_06931_gb300 import _native as N

    p, cfg = make_config("c1")
    h, w, d = p["sx"].shape
    assert d % 4 == 0
    eta = 0.83
    # reference: the problem API with alpha = 0 and a negligible mean-term weight
    P = octmc.Problem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"],
                      alpha=0.0, mu=1e-300)
    P.set_eta(0, eta)
    dev = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("sx", "sy", "ax", "ay", "vx", "vy")}
    lib = N.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(21)
    for call in range(2):  # two calls in a row share the static scratch
        D = torch.from_numpy(rng.normal(0.0, 0.7 + call, (2, 3, h, w))).cuda()
        g_ref = torch.empty_like(D)
        t = P.eval_terms(0, D, g_ref)
        g = torch.full_like(D, float("nan"))
        sums = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        ptr = lambda x: C.c_void_p(x.data_ptr())
        rc = lib.octmc_data_term_static(ptr(dev["sx"]), ptr(dev["sy"]), ptr(dev["ax"]), ptr(dev["ay"]),
                                        ptr(dev["vx"]), ptr(dev["vy"]), w, h, d, ptr(D), eta, 0.5, 1e-3,
                                        0, ptr(g), ptr(sums), stream)
        assert rc == 0
        torch.cuda.synchronize()
        s = sums.cpu().numpy()
        assert abs(s[0] - t[0]) <= F_TOL * abs(t[0])
        assert abs(s[1] - t[1]) <= F_TOL * abs(t[1])
        gn, gr = g.cpu().numpy(), g_ref.cpu().numpy()
        assert np.linalg.norm(gn - gr) <= G_TOL * np.linalg.norm(gr)


def test_static_entry_point_rejects_oversized_grids():
    from paper_2010_06931_gb300 import _native as N
    lib = N.lib()
    dummy = torch.zeros(8, device="cuda")
    ptr = C.c_void_p(dummy.data_ptr())
    rc = lib.octmc_data_term_static(ptr, ptr, None, None, None, None, 1024, 1024, 8, ptr, 1.0, 0.5, 1e-3, 0,
                                    None, ptr, None)
    assert rc == -7
    rc = lib.octmc_data_term_static(ptr, ptr, None, None, None, None, 4, 4, 6, ptr, 1.0, 0.5, 1e-3, 0,
                                    None, ptr, None)
    assert rc == -1  # depth must be a multiple of 4
    # 512 x 512 A-scans of 65536 samples: 2^32 groups of 4 samples, beyond the
    # kernel's 32-bit addressing; rejected before any launch
    rc = lib.octmc_data_term_static(ptr, ptr, None, None, None, None, 512, 512, 65536, ptr, 1.0, 0.5, 1e-3, 0,
                                    None, ptr, None)
    assert rc == -1
    # non-finite scalars are rejected
    for eta, delta0, eps_h in ((float("inf"), 0.5, 1e-3), (1.0, float("nan"), 1e-3), (1.0, 0.5, float("inf"))):
        rc = lib.octmc_data_term_static(ptr, ptr, None, None, None, None, 4, 4, 8, ptr, eta, delta0, eps_h, 0,
                                        None, ptr, None)
        assert rc == -1
