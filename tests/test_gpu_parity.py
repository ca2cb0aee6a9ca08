"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Tolerances (float data term, float64 reductions): objective and each of its
terms 1e-5 relative, gradient 1e-4 relative L2 (over the whole field),
pyramid bit-exact, the L-BFGS direction 1e-10 relative L2 (float64 history
and products), converged solves 0.05 px RMS where the minimum is determined
(the noise-free c1 rendering); on the speckled pairs, whose minima move by
more than that under 1e-7 relative input perturbations, bars set from that
spread (median A-scan, field RMS, FP64 depth of the minimum).
"""
import numpy as np
import pytest

import oracle as O
from octsynth import make_config, make_pair, true_displacement

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4


def gpu_problem(p, **kw):
    import paper_2010_06931_gb300 as octmc
    return octmc.Problem(p["sx"], p["sy"], p["tx"], p["ty"], p.get("ax"), p.get("ay"), p.get("vx"),
                         p.get("vy"), **kw)


def cpu_problem(p, **kw):
    kw = {k: v for k, v in kw.items() if k in ("alpha", "delta0", "eps_h", "eps_r", "mu", "loss")}
    if kw.get("mu", 0.0) == 0.0:
        kw["mu"] = None
    return O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"], p.get("ax"), p.get("ay"), p.get("vx"),
                           p.get("vy"), **kw)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def compare_eval(p, D, eta=0.8, **kw):
    G = gpu_problem(p, **kw)
    C = cpu_problem(p, **kw)
    G.set_eta(0, eta)
    C.eta = eta
    g = torch.zeros(G.disp_shape(0), dtype=torch.float64, device="cuda")
    tg = G.eval_terms(0, cuda(D), g)
    fc, gc, tc = C.eval(D)
    assert abs(tg[4] - fc) <= F_TOL * abs(fc), (tg, tc)
    for t in range(4):
        tol = F_TOL * max(abs(tc[t]), 1e-12 * abs(fc))
        assert abs(tg[t] - tc[t]) <= tol, (t, tg, tc)
    err = rel_l2(g.cpu().numpy(), gc)
    assert err <= G_TOL, err
    return tg, g.cpu().numpy(), tc, gc


@pytest.fixture(scope="module")
def c1():
    return make_config("c1")


@pytest.mark.parametrize("loss", [0, 1])
def test_eval_c1_random_displacements(c1, loss):
    p, cfg = c1
    rng = np.random.default_rng(11)
    for scale in (0.0, 0.6, 3.0):
        D = rng.normal(0.0, scale, (2, 3, cfg["h"], cfg["w"]))
        compare_eval(p, D, loss=loss)


def test_eval_c1_at_truth_and_oct_only(c1):
    p, cfg = c1
    T, _ = true_displacement(p, cfg["w"], cfg["h"])
    compare_eval(p, T)
    q = dict(p)
    for k in ("ax", "ay", "vx", "vy"):
        q[k] = None
    compare_eval(q, T, delta0=0.0)


@pytest.mark.parametrize("shape", [(29, 37, 245), (5, 3, 1), (1, 7, 6), (8, 1, 117), (13, 11, 4),
                                   (6, 5, 52), (7, 9, 168), (9, 7, 169)])
def test_eval_ragged_shapes(shape):
    # depth not a multiple of 4 nor of the 116-sample blocks, odd grids, degenerate axes;
    # last blocks of 52 outputs (the most the split mapping takes: d = 52, 116 + 52) and
    # of 53 (the least a full block takes: d = 116 + 53)
    h, w, d = shape
    p = make_pair(w, h, d, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=3)
    rng = np.random.default_rng(5)
    D = rng.normal(0.0, 1.5, (2, 3, h, w))
    compare_eval(p, D)
    compare_eval(p, D, loss=1, alpha=0.3, eps_r=0.2, mu=0.05)


@pytest.mark.parametrize("shape", [(11, 13, 128), (6, 7, 256), (5, 9, 233), (4, 6, 117)])
def test_eval_depth_block_boundaries(shape):
    # depths just past and inside a block boundary of the depth mapping (blocks of 116
    # outputs): a last block of 1 output (117, 233), of 12 (128) and of 24 (256); the depth
    # shifts reach past both ends of the volume, so the edge groups take the edge rule
    h, w, d = shape
    p = make_pair(w, h, d, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=6)
    rng = np.random.default_rng(8)
    D = rng.normal(0.0, 1.5, (2, 3, h, w))
    compare_eval(p, D)
    compare_eval(p, D, loss=1, alpha=0.3, eps_r=0.2, mu=0.05)
    D[:, 2] = rng.uniform(-d - 12, d + 12, (2, h, w))
    compare_eval(p, D)


def test_eval_far_outside_the_grid():
    # displacements beyond every edge: all taps are edge samples (clamp-to-edge)
    h, w, d = 9, 10, 23
    p = make_pair(w, h, d, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=4)
    D = np.zeros((2, 3, h, w))
    D[0, 0] = 1e4
    D[1, 1] = -3e5
    D[0, 2] = -77.3
    D[1, 2] = 1e9
    compare_eval(p, D)


def test_identical_inputs_give_exact_zero(c1):
    p, cfg = c1
    q = dict(p)
    q["sy"], q["ay"] = p["sx"].copy(), p["ax"].copy()
    G = gpu_problem(q)
    g = torch.full(G.disp_shape(0), 7.0, dtype=torch.float64, device="cuda")
    t = G.eval_terms(0, G.zeros(0), g)
    assert np.all(t[:5] == 0.0)
    assert torch.count_nonzero(g).item() == 0


def test_nonfinite_displacement_is_reported(c1):
    import paper_2010_06931_gb300 as octmc
    p, cfg = c1
    G = gpu_problem(p)
    D = G.zeros(0)
    D[0, 0, 3, 4] = float("nan")
    with pytest.raises(octmc.OctmcError) as e:
        G.eval_terms(0, D)
    assert e.value.code == -4


def test_nonfinite_inputs_are_reported(c1):
    # a NaN voxel in a volume reaches the objective (non-finite f, -4); a non-finite
    # acquisition time is rejected when the problem is created (-1)
    import paper_2010_06931_gb300 as octmc
    p, cfg = c1
    q = dict(p, sx=p["sx"].copy())
    q["sx"][5, 7, 9] = np.nan
    G = gpu_problem(q)
    with pytest.raises(octmc.OctmcError) as e:
        G.eval_terms(0, G.zeros(0))
    assert e.value.code == -4
    q = dict(p, tx=p["tx"].copy())
    q["tx"][2, 3] = np.inf
    with pytest.raises(octmc.OctmcError) as e:
        gpu_problem(q)
    assert e.value.code == -1


def test_eval_is_deterministic(c1):
    p, cfg = c1
    G = gpu_problem(p)
    D = cuda(np.random.default_rng(1).normal(0, 1.0, G.disp_shape(0)))
    g1, g2 = torch.empty_like(D), torch.empty_like(D)
    t1 = G.eval_terms(0, D, g1)
    t2 = G.eval_terms(0, D, g2)
    assert np.array_equal(t1, t2) and torch.equal(g1, g2)


def test_eta_parity(c1):
    p, cfg = c1
    G, C = gpu_problem(p), cpu_problem(p)
    D = np.random.default_rng(2).normal(0, 0.5, G.disp_shape(0))
    assert G.compute_eta(0, cuda(D)) == pytest.approx(C.compute_eta(D), rel=F_TOL)
    q = dict(p)
    q["ax"] = q["ay"] = None
    assert gpu_problem(q).compute_eta(0, cuda(D)) == 1.0


def test_pyramid_bit_exact():
    p = make_pair(37, 29, 51, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=8)
    G = gpu_problem(p, levels=3)
    C = cpu_problem(p).pyramid(3)
    for l in range(3):
        got = {k: v.cpu().numpy() for k, v in G.level_data(l).items()}
        for k in ("sx", "sy", "ax", "ay", "vx", "vy"):
            ref = getattr(C[l], k)
            assert got[k].shape == ref.shape, (l, k)
            assert np.array_equal(got[k], ref), (l, k)


def test_prolong_parity():
    p = make_pair(37, 29, 8, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=8)
    G = gpu_problem(p, levels=2)
    w1, h1, _ = G.level_shape(1)
    c = np.random.default_rng(3).normal(size=(2, 3, h1, w1))
    fine = G.prolong(1, cuda(c)).cpu().numpy()
    ref = O.prolong(c, 29, 37)
    assert np.allclose(fine, ref, rtol=1e-14, atol=1e-14)


def test_lbfgs_direction_parity():
    import paper_2010_06931_gb300 as octmc
    rng = np.random.default_rng(6)
    n = 5000
    A = rng.uniform(0.5, 3.0, size=n)  # diagonal SPD curvature
    S = [rng.normal(size=n) for _ in range(11)]
    Y = [A * s + 0.01 * rng.normal(size=n) for s in S]
    g = rng.normal(size=n)
    H = octmc.Lbfgs(n, m=8)
    for s, y in zip(S, Y):
        assert H.push(cuda(s), cuda(y)) == 0
    d, gtd = H.direction(cuda(g))
    ref = O.lbfgs_direction(S[-8:], Y[-8:], g)  # the last 8 pairs are kept
    # The library keeps the pairs in float32 (relative rounding 2^-24; it moves this
    # direction by 3e-9) and takes their products with y and g as float32 FMAs over
    # <= 8 elements per thread and a 32-lane float32 butterfly before float64 sums:
    # up to ~1e-6 relative error on a product with heavy cancellation, entering
    # the direction only through the small history correction.
    # float64 pairs and products on both sides; the compact and the two-loop
    # forms agree in exact arithmetic, so only rounding separates them
    err = rel_l2(d.cpu().numpy(), ref)
    print("lbfgs direction rel L2 %.3e, g'dir rel %.3e" % (err, abs(gtd - g @ ref) / abs(g @ ref)))
    assert err < 1e-10
    assert gtd == pytest.approx(float(g @ ref), rel=1e-10)
    # a pair with negative curvature is rejected and changes nothing
    assert H.push(cuda(S[0]), cuda(-Y[0])) == 1
    d2, _ = H.direction(cuda(g))
    assert torch.equal(d, d2)
    H.reset()
    d3, gtd3 = H.direction(cuda(g))
    assert np.array_equal(d3.cpu().numpy(), -g) and gtd3 == pytest.approx(-(g @ g), rel=1e-12)


def test_lbfgs_direction_parity_longest_history():
    # m = 32 (the largest history a problem accepts): 66 history vectors, several
    # block rows of the dot-product kernel, a ragged length
    import paper_2010_06931_gb300 as octmc
    rng = np.random.default_rng(7)
    n = 3001
    A = rng.uniform(0.5, 3.0, size=n)
    S = [rng.normal(size=n) for _ in range(40)]
    Y = [A * s + 0.01 * rng.normal(size=n) for s in S]
    g = rng.normal(size=n)
    H = octmc.Lbfgs(n, m=32)
    for s, y in zip(S, Y):
        assert H.push(cuda(s), cuda(y)) == 0
    d, gtd = H.direction(cuda(g))
    ref = O.lbfgs_direction(S[-32:], Y[-32:], g)
    assert rel_l2(d.cpu().numpy(), ref) < 1e-10
    assert gtd == pytest.approx(float(g @ ref), rel=1e-10)


def test_solve_parity_longest_history():
    # the solver's speculative pair + gradient products with 2 (m + 1) = 66
    # history vectors, on the well-posed noise-free pair, both run to the
    # ftol stopping rule through the pyramid
    p, cfg = clean_c1()
    G = gpu_problem(p, levels=3, lbfgs_m=32, ftol=1e-6)
    C = cpu_problem(p)
    Dg, st = G.solve_full()
    Dc, stc = C.solve_full(3, m=32, ftol=1e-6)
    rms = float(np.sqrt(((Dg.cpu().numpy() - Dc) ** 2).mean()))
    print("clean c1 converged, m = 32: GPU vs oracle %.4f px" % rms)
    assert [s["status"] for s in st] == [0, 0, 0], st
    assert [s["status"] for s in stc] == [0, 0, 0], stc
    assert rms <= 0.05, (rms, st, stc)


def clean_c1():
    # the c1 scan pair rendered without noise and saccades: the objective has a
    # well-determined minimum (two float64 oracle runs whose inputs differ by
    # 1e-7 relative end 0.001 px apart), so converged solves can be compared tightly
    return make_config("c1", speckle=False, angio_noise=False, n_saccades=0)


@pytest.mark.parametrize("loss", [0, 1])
def test_solve_full_converged_parity_clean_c1(loss):
    # the coarse-to-fine solve run to convergence on both sides (status 0 on
    # every level), identical algorithm and constants; the converged minima
    # agree within the 0.05 px bar, and both recover the known motion.  At
    # this noise-free minimum the GPU's float-evaluated objective rounds at
    # about 4e-5 of f, far above ftol, so where the GPU's stopping rule fires
    # depends on rounding: changes of summation order alone moved its endpoint
    # between 0.0009 and 0.014 px from the oracle's
    p, cfg = clean_c1()
    T, mask = true_displacement(p, cfg["w"], cfg["h"])
    G = gpu_problem(p, levels=3, loss=loss, ftol=1e-6)
    C = cpu_problem(p, loss=loss)
    Dg, st = G.solve_full()
    Dc, stc = C.solve_full(3, ftol=1e-6)
    Dg = Dg.cpu().numpy()
    rms = float(np.sqrt(((Dg - Dc) ** 2).mean()))
    # the GPU's minimum is at least as deep as the oracle's, both measured by
    # the FP64 objective.  The GPU minimises its float-evaluated objective,
    # whose rounding at this noise-free minimum (residuals near zero, float
    # interpolants rounded at 2^-24 of values up to 1 on 2.6e5 voxel pairs) is
    # about 4e-5 of f, so its minimum may sit that much higher in FP64; it may
    # also sit lower, where the oracle's ftol stopped it earlier in the valley
    P0 = C.pyramid(1)[0]
    P0.eta = stc[-1]["eta"]
    f_g = P0.eval(Dg, grad=False)[0]
    print("clean c1 converged (loss %d): GPU vs oracle %.4f px, FP64 objective %.9g / %.9g, iters %s / %s" %
          (loss, rms, f_g, stc[-1]["f"], [s["iters"] for s in st], [s["iters"] for s in stc]))
    assert [s["status"] for s in st] == [0, 0, 0], st
    assert [s["status"] for s in stc] == [0, 0, 0], stc
    assert rms <= 0.05
    assert f_g <= stc[-1]["f"] * (1.0 + 1e-4)
    mask[:, :4] = mask[:, -4:] = False
    mask[:, :, :4] = mask[:, :, -4:] = False
    m6 = np.broadcast_to(mask[:, None], T.shape)
    assert np.sqrt(((Dg - T)[m6] ** 2).mean()) < 0.2


def test_solve_full_converged_parity_c1(c1):
    # the speckled c1 pair (drift, saccades, noise) at the library's default
    # stopping rule.  Its minimum is not determined to 0.05 px RMS: six float64
    # oracle solves whose inputs differ from the unperturbed ones by 1e-7
    # relative end 0.021-0.079 px RMS from the unperturbed solve (median A-scan
    # 0.001-0.008 px), and the FP64 objective at those minima lies within
    # -1.9e-3 .. +3.8e-4 relative of the unperturbed one.  Pinned: both
    # converge, the median A-scan agrees within 0.02 px, the field within twice
    # the oracle's own spread, and the GPU minimum is as deep as the oracle's to
    # 1e-3 relative (both evaluated by the FP64 oracle at the same eta)
    p, cfg = c1
    G = gpu_problem(p, levels=3)
    C = cpu_problem(p)
    Dg, st = G.solve_full()
    Dc, stc = C.solve_full(3)
    Dg = Dg.cpu().numpy()
    diff = Dg - Dc
    rms = float(np.sqrt((diff ** 2).mean()))
    med = float(np.median(np.sqrt((diff.reshape(6, -1) ** 2).mean(axis=0))))
    P0 = C.pyramid(1)[0]
    P0.eta = stc[-1]["eta"]
    f_g = P0.eval(Dg, grad=False)[0]
    f_c = stc[-1]["f"]
    print("c1 converged: GPU vs oracle %.4f px RMS, median A-scan %.4f px, FP64 objective %.6f (GPU) / "
          "%.6f (oracle), iters %s / %s" % (rms, med, f_g, f_c, [s["iters"] for s in st],
                                            [s["iters"] for s in stc]))
    assert [s["status"] for s in st] == [0, 0, 0], st
    assert [s["status"] for s in stc] == [0, 0, 0], stc
    assert med <= 0.02
    assert rms <= 0.16
    assert f_g <= f_c * (1.0 + 1e-3)


@pytest.fixture(scope="module")
def c2():
    return make_config("c2")


def test_eval_parity_clinical_size(c2):
    # the benchmark's workload (300 x 300 A-scans x 512, float32, level 0) through the
    # batched launch path the benchmark times: the true displacement (the benchmark's
    # input) and, with the SSD loss, the truth plus 0.5 px of noise
    p, cfg = c2
    T, _ = true_displacement(p, cfg["w"], cfg["h"])
    compare_eval(p, T)
    compare_eval(p, T + np.random.default_rng(4).normal(0.0, 0.5, T.shape), loss=1, alpha=0.1)


def test_solve_full_converged_minimum_clinical_size(c2):
    # the benchmark's converged solve (300 x 300 A-scans x 512, three levels,
    # library defaults) against the FP64 oracle's converged solve stored in
    # tests/golden/c2_oracle_solution.npz.  This objective is non-convex and its
    # minimum is not determined to 0.05 px: two GPU solves whose inputs differ
    # by 1e-7 relative end 0.24 px RMS apart (0.28 at ftol 1e-8 and 1e-9), and
    # a GPU solve started at the oracle's minimum moves 0.19 px.  Most A-scans
    # agree closely; patches of a tenth of them settle in neighbouring minima.
    # Pinned: both converge, the GPU's minimum is as deep as the oracle's in
    # the FP64 objective to 1e-3 relative (both evaluated here, same inputs,
    # same eta; minima reached under 1e-7 input perturbations differ in depth
    # by up to 1.9e-3 on the speckled c1 pair), the median A-scan agrees within
    # 0.05 px, and the whole field within twice the perturbation spread.  The stored solve may come from a platform
    # whose rendering of the inputs differs in the last bits (an input
    # perturbation of the size the control above uses), so its inputs are
    # matched by fingerprint
    import json
    import os
    from octsynth import fingerprint, fingerprints_match
    p, cfg = c2
    path = os.path.join(os.path.dirname(__file__), "golden", "c2_oracle_solution.npz")
    z = np.load(path)
    ref = z["disp"].astype(np.float64)
    meta = json.loads(str(z["meta"]))
    assert fingerprints_match(fingerprint(p), meta["inputs_fingerprint"]), "stored solve is of other inputs"
    assert [s["status"] for s in meta["stats"]] == [0, 0, 0]
    G = gpu_problem(p, levels=meta["levels"], lbfgs_m=meta["solver"]["m"],
                    ftol=meta["solver"]["ftol"])
    Dg, st = G.solve_full()
    Dg = Dg.cpu().numpy().astype(np.float64)
    assert [s["status"] for s in st] == [0, 0, 0], st
    diff = Dg - ref
    rms = float(np.sqrt((diff ** 2).mean()))
    per_ascan = np.sqrt((diff.reshape(6, -1) ** 2).mean(axis=0))
    med = float(np.median(per_ascan))
    C = cpu_problem(p)
    C.eta = meta["stats"][-1]["eta"]
    f_g = C.eval(Dg, grad=False)[0]
    f_o = C.eval(ref, grad=False)[0]
    print("c2 converged: GPU vs oracle %.4f px RMS, median A-scan %.4f px; FP64 objective "
          "%.3f (GPU) / %.3f (oracle); iters %s / %s" %
          (rms, med, f_g, f_o, [s["iters"] for s in st], [s["iters"] for s in meta["stats"]]))
    assert f_g <= f_o * (1.0 + 1e-3)
    assert med <= 0.05
    assert rms <= 0.5


def test_async_evaluation_equals_the_synchronous_one(c1):
    # the same evaluation enqueued without waiting, back to back on one
    # stream: bitwise the synchronous result, the terms left in device memory
    p, cfg = c1
    G = gpu_problem(p)
    G.set_eta(0, 0.8)
    rng = np.random.default_rng(11)
    Ds = [cuda(rng.normal(0.0, 0.7, G.disp_shape(0))) for _ in range(3)]
    ref = []
    for D in Ds:
        g = torch.zeros(G.disp_shape(0), dtype=torch.float64, device="cuda")
        t = G.eval_terms(0, D, g)
        ref.append((t, g))
    st = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(st):
        for D in Ds:
            g = torch.zeros(G.disp_shape(0), dtype=torch.float64, device="cuda")
            t = torch.zeros(6, dtype=torch.float64, device="cuda")
            G.eval_objective_grad_async(0, D, g, t, stream=st)
            outs.append((t, g))
    st.synchronize()
    for (t, g), (tr, gr) in zip(outs, ref):
        assert np.array_equal(t.cpu().numpy(), np.asarray(tr, dtype=np.float64))
        assert torch.equal(g, gr)
