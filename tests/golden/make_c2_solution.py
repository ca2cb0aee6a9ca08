"""Writes c2_oracle_solution.npz: the FP64 oracle's converged coarse-to-fine
solve of the clinical-size synthetic pair (300 x 300 A-scans x 512 samples,
three levels, the library's default constants and stopping rule).

The solve takes the CPU oracle about an hour or more, so the benchmark and
the GPU tests compare against this stored result instead of recomputing it.
Only ``oracle`` and the input generator are used.  The inputs are identified
by the generator preset and seed, by a checksum of the rendered volumes and
by their fingerprint (float64 sums and sums of squares per array): another
platform's rendering may differ in the last bits of some voxels, so users of
the stored solve match the fingerprint to a relative tolerance.

Run: python tests/golden/make_c2_solution.py              (solve and store)
     python tests/golden/make_c2_solution.py --meta-only  (re-describe the inputs of the stored solve)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from octsynth import fingerprint, make_config  # noqa: E402

OUT = os.path.join(HERE, "c2_oracle_solution.npz")

# the library's defaults (octmc_desc_defaults): alpha 0.1, delta_0 0.5,
# eps_H 1e-3, eps_R 0.01, mu 1/(2 w h), pseudo-Huber loss, m 8, ftol 1e-7
SOLVER = dict(m=8, max_iter=5000, max_ls=20, gtol=1e-6, ftol=1e-7)


def inputs_checksum(p):
    h = hashlib.sha1()
    for k in ("sx", "sy", "ax", "ay", "vx", "vy", "tx", "ty"):
        h.update(np.ascontiguousarray(p[k]).tobytes())
    return h.hexdigest()


def main():
    p, cfg = make_config("c2")
    P = O.OracleProblem(p["sx"], p["sy"], p["tx"], p["ty"], p["ax"], p["ay"], p["vx"], p["vy"])
    t0 = time.time()
    D, stats = P.solve_full(cfg["levels"], **SOLVER)
    secs = time.time() - t0
    meta = dict(preset="c2", seed=cfg["seed"], levels=cfg["levels"], solver=SOLVER, stats=stats,
                seconds=secs, threads=O.num_threads(), inputs_sha1=inputs_checksum(p),
                inputs_fingerprint=fingerprint(p))
    np.savez_compressed(OUT, disp=D.astype(np.float32), meta=json.dumps(meta))
    print(json.dumps(meta))


def meta_only():
    # the stored field is kept as it is; only the description of its inputs
    # (rendered again by the same generator on this machine) is rewritten
    z = np.load(OUT)
    disp = z["disp"]
    meta = json.loads(str(z["meta"]))
    p, cfg = make_config(meta["preset"])
    sha = inputs_checksum(p)
    if sha != meta["inputs_sha1"]:
        raise SystemExit("inputs rendered here differ from the stored solve's (%s != %s)"
                         % (sha, meta["inputs_sha1"]))
    meta["inputs_fingerprint"] = fingerprint(p)
    np.savez_compressed(OUT, disp=disp, meta=json.dumps(meta))
    print(json.dumps(meta["inputs_fingerprint"]))


if __name__ == "__main__":
    if "--meta-only" in sys.argv[1:]:
        meta_only()
    else:
        main()
