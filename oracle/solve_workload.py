"""Run the oracle's full FGMRES(50) solve of a named workload and record its
iteration count (used to scale the oracle's per-iteration time into a
per-solve time in the benchmark's CPU baseline). Writes
oracle/iteration_counts.json. Test infrastructure only.

With --solutions it also solves the workload to a relative residual of 1e-12
and stores that solution (zero-mean pressure) as
oracle/solutions/<name>.npy: the reference the benchmark measures each GPU
solve's error against (small workloads only).

usage: python -m oracle.solve_workload [--solutions] cube64 [cube8 ...]
"""
import json
import os
import sys
import time

import numpy as np

import sinker_inputs as si

from . import gmg, krylov, mesh, operators, sinker

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "iteration_counts.json")
SOL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "solutions")


def solve(name, rtol=1e-8, keep=None):
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
    if keep is not None:
        keep.append(krylov.zero_mean_pressure(ops, x))
    return {"iterations": int(its), "rtol": rtol, "true_rel_residual": true, "seconds": secs,
            "n_u": int(m.n_u), "n_p": int(m.n_p)}


def main(names, solutions=False):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        data[name] = solve(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        if solutions:
            keep = []
            info = solve(name, rtol=1e-12, keep=keep)
            os.makedirs(SOL, exist_ok=True)
            np.save(os.path.join(SOL, name + ".npy"), keep[0])
            print(name, "solution to 1e-12:", info, flush=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    sol = "--solutions" in args
    args = [a for a in args if a != "--solutions"]
    main(args or ["cube8"], solutions=sol)
