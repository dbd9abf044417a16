"""Run the oracle's full FGMRES(50) solve of a named workload and record its
iteration count (used to scale the oracle's per-iteration time into a
per-solve time in the benchmark's CPU baseline). Writes
oracle/iteration_counts.json. Test infrastructure only.

usage: python -m oracle.solve_workload cube64 [cube8 ...]
"""
import json
import os
import sys
import time

import numpy as np

import sinker_inputs as si

from . import gmg, krylov, mesh, operators, sinker

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "iteration_counts.json")


def solve(name, rtol=1e-8):
    p = si.workload(name)
    m = mesh.Mesh(p.n)
    mus = sinker.level_viscosities(m, p, p.n_levels)
    G = gmg.GMG(p.n, p.n_levels, mus)
    ops = G.levels[-1].ops
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    b = np.concatenate([F, np.zeros(m.n_p)])
    Pc = krylov.StokesPreconditioner(ops, G)
    t = time.time()
    x, its, hist = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=rtol)
    secs = time.time() - t
    true = float(np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b))
    return {"iterations": int(its), "rtol": rtol, "true_rel_residual": true, "seconds": secs,
            "n_u": int(m.n_u), "n_p": int(m.n_p)}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        data[name] = solve(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["cube8"])
