"""Write the checker's load paths that the GPU path tests compare against.

Calls only the FP64 checker in ``oracle/`` (and the specimen generator for the inputs).
Each case runs the staggered iteration of Sec. 3.1 (ST) or the fixed-stress S-step of
Sec. 3.3-3.5 (S1/S2/S3) on the tensile notched square of Sec. 4.1 and stores, per load
step, the reaction force, the staggered pass count and the convergence flag, plus the
phase field at a few load steps.  The paths are long (the crack phase needs thousands of
passes at the finer grid), so they are stored rather than recomputed by the tests.

    python tests/golden/make_oracle_paths.py tensile128 0     # one scheme of one case
    python tests/golden/make_oracle_paths.py merge             # join the parts

Cases:
  tensile64   64 x 64, l = 0.03 mm, 20 steps to 6e-3 mm, ST, TOL_ST 1e-9 (the plain
              standard-scheme benchmark in FP64), phase field at every step.
  tensile128  128 x 128, l = 0.03 mm (l/h = 3.84, the l/h of the 512 x 512 workload with
              l = 0.0075 mm), 100 steps to 6e-3 mm, ST/S1/S2/S3, TOL_ST 1e-5, phase field
              at steps 40, 60, 80 and 100.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import model, q1, staggered as stg  # noqa: E402
from paper_2209_07969_gb300 import specimens as S  # noqa: E402

CASES = {
    "tensile64": dict(n=64, l=0.03, steps=20, schemes=(0,), tol=1e-9,
                      keep=tuple(range(1, 21))),
    "tensile128": dict(n=128, l=0.03, steps=100, schemes=(0, 1, 2, 3), tol=1e-5,
                       keep=(40, 60, 80, 100)),
}


def run(case, scheme):
    c = CASES[case]
    spec = S.tensile(c["n"], l=c["l"], steps=c["steps"], u_max=6e-3)
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    st = stg.State(g)
    opts = stg.Options(tol_st=c["tol"], max_stag=20000)
    F, it, conv, fields = [], [], [], []
    t0 = time.time()
    for k, du in enumerate(spec.increments):
        r = stg.load_step(g, m, st, du, scheme, opts, spec.reaction_dir)
        F.append(r.reaction)
        it.append(r.stag_iters)
        conv.append(bool(r.converged))
        if k + 1 in c["keep"]:
            fields.append(st.d.copy())
        print(case, scheme, k + 1, f"{r.reaction:.8e}", r.stag_iters, r.converged,
              f"{time.time() - t0:.0f}s", flush=True)
    out = os.path.join(HERE, f".part_{case}_s{scheme}.npz")
    np.savez_compressed(out, reaction=np.array(F), stag_iters=np.array(it),
                        converged=np.array(conv), d=np.array(fields),
                        keep=np.array(c["keep"]))


def merge():
    for case, c in CASES.items():
        arrs = {}
        for s in c["schemes"]:
            part = os.path.join(HERE, f".part_{case}_s{s}.npz")
            if not os.path.exists(part):
                print(f"{case}: scheme {s} not written yet")
                continue
            z = np.load(part)
            for k in ("reaction", "stag_iters", "converged"):
                arrs[f"s{s}_{k}"] = z[k]
            # the phase field is compared to 1e-5 at most: single precision holds it
            arrs[f"s{s}_d"] = z["d"].astype(np.float32)
            arrs["keep"] = z["keep"]
        arrs["tol"] = np.array(c["tol"])
        np.savez_compressed(os.path.join(HERE, f"oracle_{case}.npz"), **arrs)


if __name__ == "__main__":
    if sys.argv[1] == "merge":
        merge()
    else:
        run(sys.argv[1], int(sys.argv[2]))
