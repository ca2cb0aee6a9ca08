"""Saccade validity and en-face OCTA projection on the GPU (Sec. 2.2, 2.3)
against the oracle: the filtered volume and the quantiles bit-exact (order
statistics of the same float values), the mask counts equal, the en-face
image within float rounding of the depth means; both scan orientations,
ragged sizes, saturated B-scans, an explicit OCT threshold, no valid B-scan,
and repeatability."""
import numpy as np
import pytest

import oracle as O
from octsynth import make_octa_scan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(sc, v=None, **kw):
    import paper_2010_06931_gb300 as octmc
    A = torch.from_numpy(sc["A"]).cuda()
    S = torch.from_numpy(sc["S"]).cuda()
    if v is None:
        vg, mg = octmc.saccade_validity(A, sc["fast_axis"])
    else:
        vg, mg = torch.from_numpy(v).cuda(), None
    F = torch.empty_like(A)
    E, info = octmc.enface(A, S, sc["fast_axis"], vg, filtered=F, **kw)
    return vg.cpu().numpy(), (None if mg is None else mg.cpu().numpy()), E.cpu().numpy(), info, F.cpu().numpy()


def check(sc, v=None, **kw):
    vg, mg, E, info, F = run(sc, v, **kw)
    if v is None:
        vo, mo = O.saccade_validity(sc["A"], sc["fast_axis"])
        assert np.array_equal(vg, vo)
        assert np.allclose(mg, mo, rtol=1e-12, atol=0)
    else:
        vo = v
    t_oct = kw.get("t_oct")
    Eo, io, Fo = O.enface(sc["A"], sc["S"], sc["fast_axis"], vo, t_oct=t_oct, want_filtered=True,
                          **{k: kw[k] for k in ("q_lo", "q_hi", "thresh") if k in kw})
    assert np.array_equal(F, Fo)
    assert info["p_lo"] == io["p_lo"] and info["p_hi"] == io["p_hi"]
    assert info["t_oct"] == pytest.approx(io["t_oct"], rel=1e-12)
    assert info["kept"] == io["kept"]
    assert np.abs(E - Eo).max() <= 2e-6 * max(1.0, float(np.abs(Eo).max()))
    return vg, E, info


@pytest.mark.parametrize("fast_axis", [0, 1])
def test_validity_and_projection_match_the_oracle(fast_axis):
    sc = make_octa_scan(61, 47, 90, fast_axis=fast_axis, n_saturated=2, seed=11 + fast_axis)
    v, E, info = check(sc)
    # the saturated B-scans are found and replaced by valid neighbours
    for b in sc["saturated"]:
        assert v[b] == 0
    line = E if fast_axis == 0 else E.T
    bad = np.where(v == 0)[0]
    good = np.where(v != 0)[0]
    for b in bad:
        near = good[np.argmin(np.abs(good - b) * 2 + (good > b))]
        assert np.array_equal(line[b], line[near])
    assert 0 < info["kept"] < sc["A"].size


def test_explicit_oct_threshold_and_other_quantiles():
    sc = make_octa_scan(40, 36, 64, fast_axis=0, n_saturated=1, seed=5)
    check(sc, t_oct=0.2, q_lo=0.1, q_hi=0.9, thresh=0.2)


def test_no_valid_bscan_uses_every_voxel():
    sc = make_octa_scan(33, 29, 50, fast_axis=1, n_saturated=0, seed=6)
    check(sc, v=np.zeros(33, np.float32))


@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 1, 7), (1, 6, 3), (17, 13, 1)])
def test_degenerate_shapes(shape):
    h, w, d = shape
    rng = np.random.default_rng(h * 100 + w * 10 + d)
    sc = dict(A=rng.random((h, w, d)).astype(np.float32), S=rng.random((h, w, d)).astype(np.float32), fast_axis=0)
    check(sc)


def test_repeatable_and_validates_arguments():
    import paper_2010_06931_gb300 as octmc
    sc = make_octa_scan(48, 40, 64, fast_axis=0, seed=9)
    a = run(sc)
    b = run(sc)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    A = torch.from_numpy(sc["A"]).cuda()
    with pytest.raises(octmc.OctmcError):
        octmc.enface(A, A, 0, torch.ones(40, device="cuda"), q_lo=1.5)
    with pytest.raises(ValueError):
        octmc.enface(A, A, 0, torch.ones(41, device="cuda"))
