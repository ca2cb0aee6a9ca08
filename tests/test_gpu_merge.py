"""Final resampling and merging on the GPU (Sec. 2.1, 2.5) against the oracle:
motion-corrected volumes, merge weights, merged volume and merged en-face
angiography, at zero motion, at the true motion of a synthetic pair, on a
ragged shape and with 16-bit storage; results are deterministic."""
import numpy as np
import pytest

import oracle as O
from octsynth import make_config, make_pair, true_displacement

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def round_bf16(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32)).view(np.float32)


ROUND = {1: round_bf16, 2: lambda a: np.asarray(a, np.float32).astype(np.float16).astype(np.float32)}

ALL = ("merged", "corrected_x", "corrected_y", "weights", "angio")


def inputs(p):
    return [p[k] for k in ("sx", "sy", "tx", "ty", "ax", "ay", "vx", "vy")]


def decided(ref, beta, tau, margin=1e-4):
    """A-scans whose clipping decisions (raw weight vs tau, and which scan is
    kept when both are clipped) are not within `margin` of a tie."""
    raw = np.exp(-beta * np.maximum(0.0, ref["density"] - 1.0))
    ok = np.all(np.abs(raw - tau) > margin, axis=0)
    both = np.all(raw < tau, axis=0)
    return ok & ~(both & (np.abs(raw[0] - raw[1]) <= margin))


def compare(G, C, D, beta=2.0, tau=0.05):
    got = {k: v.cpu().numpy() for k, v in G.merge(torch.from_numpy(D).cuda(), beta, tau, outputs=ALL).items()}
    ref = C.merge(D, beta, tau)
    scale = max(float(np.abs(C.sx).max()), float(np.abs(C.sy).max()))
    for k, r in (("corrected_x", "cx"), ("corrected_y", "cy")):
        err = np.abs(got[k] - ref[r]).max()
        assert err <= 2e-6 * scale, (k, err)
    m = decided(ref, beta, tau)
    assert m.mean() > 0.99
    werr = np.abs(got["weights"] - ref["weights"])[:, m].max()
    assert werr <= 2e-5, werr
    merr = np.abs(got["merged"] - ref["merged"])[m].max()
    assert merr <= 2e-6 * scale + 2e-5 * scale, merr
    if ref["angio"] is not None:
        ascale = max(float(np.abs(C.ax).max()), float(np.abs(C.ay).max()), 1e-30)
        aerr = np.abs(got["angio"] - ref["angio"])[m].max()
        assert aerr <= 1e-4 * ascale, aerr
    return got, ref, m


def test_zero_motion_gives_the_average_on_a_ragged_shape():
    import paper_2010_06931_gb300 as octmc
    p = make_pair(37, 29, 51, n_layers=4, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=8)
    G = octmc.Problem(*inputs(p), levels=1)
    C = O.OracleProblem(*inputs(p))
    D = np.zeros(C.shape_disp())
    got, ref, m = compare(G, C, D)
    assert m.all()
    assert np.all(got["weights"] == 0.5)
    assert np.array_equal(got["corrected_x"], p["sx"]) and np.array_equal(got["corrected_y"], p["sy"])


def test_true_motion_of_a_synthetic_pair():
    import paper_2010_06931_gb300 as octmc
    p, cfg = make_config("c1")
    T, _ = true_displacement(p, cfg["w"], cfg["h"])
    G = octmc.Problem(*inputs(p), levels=1)
    C = O.OracleProblem(*inputs(p))
    got, ref, m = compare(G, C, T)
    # the saccades leave gaps and duplicates: some weights move away from 1/2
    assert np.abs(ref["weights"] - 0.5).max() > 0.1


def test_ragged_shape_with_random_motion_and_both_clipped():
    import paper_2010_06931_gb300 as octmc
    p = make_pair(45, 33, 133, n_layers=5, n_slabs=2, n_saccades=2, max_saccade=4.0, drift_sigma=0.05, seed=12)
    G = octmc.Problem(*inputs(p), levels=1)
    C = O.OracleProblem(*inputs(p))
    rng = np.random.default_rng(3)
    D = rng.normal(0.0, 1.5, C.shape_disp())
    D[:, 0, 10:14, :] -= 3.0  # rows collapsing onto each other in both scans
    D[:, 1, :, 20:23] += 2.5
    D[:, :, 0, 0] = [[-40.0, 55.0, 200.0], [70.0, -90.0, -300.0]]  # far outside the volume
    got, ref, m = compare(G, C, D, beta=3.0, tau=0.2)
    raw = np.exp(-3.0 * np.maximum(0.0, ref["density"] - 1.0))
    assert np.any(np.all(raw < 0.2, axis=0) & m)  # the keep-the-larger rule is exercised


@pytest.mark.parametrize("storage", [1, 2])
def test_16bit_storage_matches_the_oracle_on_rounded_volumes(storage):
    import paper_2010_06931_gb300 as octmc
    p, cfg = make_config("c1")
    T, _ = true_displacement(p, cfg["w"], cfg["h"])
    G = octmc.Problem(*inputs(p), levels=1, storage=storage)
    q = dict(p, sx=ROUND[storage](p["sx"]), sy=ROUND[storage](p["sy"]))
    C = O.OracleProblem(*inputs(q))
    compare(G, C, T)


def test_deterministic_and_outputs_independent():
    import paper_2010_06931_gb300 as octmc
    p, cfg = make_config("c1")
    T, _ = true_displacement(p, cfg["w"], cfg["h"])
    G = octmc.Problem(*inputs(p), levels=1)
    Dd = torch.from_numpy(T).cuda()
    a = G.merge(Dd, outputs=ALL)
    b = G.merge(Dd, outputs=ALL)
    for k in ALL:
        assert torch.equal(a[k], b[k]), k
    # merged alone (weights kept internally) equals merged with weights requested
    c = G.merge(Dd, outputs=("merged",))
    assert torch.equal(c["merged"], a["merged"])
    e = G.merge(Dd, outputs=("corrected_y",))
    assert torch.equal(e["corrected_y"], a["corrected_y"])


def test_invalid_arguments_are_rejected():
    import paper_2010_06931_gb300 as octmc
    p = make_pair(16, 12, 20, n_layers=3, n_slabs=1, n_saccades=1, max_saccade=2.0, drift_sigma=0.05, seed=4)
    G = octmc.Problem(*inputs(p), levels=1)
    D = G.zeros(0)
    with pytest.raises(octmc.OctmcError):
        G.merge(D, tau=1.5)
    with pytest.raises(octmc.OctmcError):
        G.merge(D, beta=-1.0)
    with pytest.raises(ValueError):
        G.merge(D, outputs=("nope",))
