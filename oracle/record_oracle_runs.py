"""Records how much work the FP64 oracle needs to solve a workload to its
tolerance, so that a bounded timing sample of the oracle can be scaled to
whole solves.

TEST INFRASTRUCTURE ONLY (as the rest of oracle/): calls nothing but the
oracle and the seeded input generators.  Usage:

    python oracle/record_oracle_runs.py steady3d 150 [threads]

solves the steady 3D workload (n^3 hexahedra x 6 tetrahedra, dispersion
field rotated per 10^3 block) with MPRGP + active-set polish (the oracle's
solve_qp) and writes oracle/runs/steady3d_n<n>.json with the MPRGP
iteration count, the polish rounds, the KKT residual of the result and the
wall time, plus oracle/runs/steady3d_n<n>_x.npy (the oracle solution at the
free unknowns, float64) when --keep-x is given.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import nn_inputs as I  # noqa: E402
from oracle import oracle as O  # noqa: E402


def steady3d(n, threads, keep_x=False):
    spec = I.config3_steady_3d(n=n)
    t0 = time.time()
    coords, conn = O.mesh_structured(3, spec.nx)
    asm = O.assemble(coords, conn, spec.coef_kind, spec.coef, spec.aL, spec.aT, spec.DM, spec.f_elem)
    red = O.Reduced(asm, spec.dmask, spec.dval)
    b = red.rhs()
    t1 = time.time()
    x, info = O.solve_qp(red.A, b, spec.lo, spec.hi, threads=threads)
    t2 = time.time()
    k = O.kkt(red.A, b, spec.lo, spec.hi, x)
    out = dict(workload="steady3d_n%d" % n, n_free=int(red.nF), nnz_free=int(red.A.nnz),
               mprgp_iters=int(info["mprgp_iters"]), polish_rounds=int(info["polish_rounds"]),
               polished=bool(info["polished"]), kkt_rel=float(k["kkt_rel"]), bounds_ok=bool(k["bounds_ok"]),
               assemble_s=t1 - t0, solve_s=t2 - t1, threads=threads,
               how="oracle.solve_qp (MPRGP to ||gP|| <= 1e-12 ||b||, then active-set polish)")
    os.makedirs(os.path.join(HERE, "runs"), exist_ok=True)
    with open(os.path.join(HERE, "runs", "steady3d_n%d.json" % n), "w") as f:
        json.dump(out, f, indent=1)
    if keep_x:
        np.save(os.path.join(HERE, "runs", "steady3d_n%d_x.npy" % n), x)
    return out


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    if not args or args[0] != "steady3d":
        sys.exit(__doc__)
    n = int(args[1]) if len(args) > 1 else 150
    threads = int(args[2]) if len(args) > 2 else (os.cpu_count() or 1)
    print(json.dumps(steady3d(n, threads, keep_x="--keep-x" in sys.argv)))
