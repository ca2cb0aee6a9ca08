"""Input generator: stored results are matched to their inputs by
fingerprint, which must accept a rendering that differs in the last bits and
reject any other input."""
import json
import os

import numpy as np

from octsynth import fingerprint, fingerprints_match, make_config


def test_fingerprint_accepts_last_bit_differences_only():
    p, _ = make_config("c1")
    f = fingerprint(p)
    assert fingerprints_match(f, f)
    q = dict(p)
    rng = np.random.default_rng(0)
    sx = p["sx"].copy()
    # one ulp up or down on a tenth of the voxels: what another platform's
    # rounding of the rendering does
    flip = rng.random(sx.shape) < 0.1
    sx[flip] = np.nextafter(sx[flip], np.where(rng.random(flip.sum()) < 0.5, -np.inf, np.inf)).astype(sx.dtype)
    q["sx"] = sx
    assert fingerprints_match(f, fingerprint(q))
    # the worst case: every voxel one ulp up
    q["sx"] = np.nextafter(p["sx"], np.float32(np.inf))
    assert fingerprints_match(f, fingerprint(q))
    # one voxel moved by the value range, or another seed: other inputs
    sx2 = p["sx"].copy()
    sx2.flat[12345] += 1.0
    q["sx"] = sx2
    assert not fingerprints_match(f, fingerprint(q))
    p2, _ = make_config("c1", seed=7)
    assert not fingerprints_match(f, fingerprint(p2))
    assert not fingerprints_match(f, {k: v for k, v in f.items() if k != "ax"})


def test_stored_clinical_size_solve_describes_its_inputs():
    z = np.load(os.path.join(os.path.dirname(__file__), "golden", "c2_oracle_solution.npz"))
    meta = json.loads(str(z["meta"]))
    assert z["disp"].shape == (2, 3, 300, 300)
    assert set(meta["inputs_fingerprint"]) == {"sx", "sy", "ax", "ay", "vx", "vy", "tx", "ty"}
    assert [s["status"] for s in meta["stats"]] == [0, 0, 0]
