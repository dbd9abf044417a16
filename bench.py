#!/usr/bin/env python
"""Benchmark of the matrix-free GMG Stokes hot path on GB300.

One step = one whole solve of the Stokes system of the 64^3 sinker workload
(8 sinkers, viscosity ratio 1e4, 7 GMG levels, Chebyshev degree 4) to a
relative residual of 1e-8: FP64 FGMRES(50) preconditioned by the block-
triangular P^-1 with the GMG V-cycle in FP32 and the Schur approximation,
outer operator and coarse solve in FP64. Inputs (viscosity, right-hand side,
level tables) are resident in HBM; each step starts from a zero guess.

value = whole-job solve throughput: (N_u + N_p) * n_gpus / (seconds per solve)
in GDoF/s. Extra keys report the pieces of the metric: the solve time with the
FP32 and the FP64 V-cycle, iterations, the standalone vmult rate (GDoF/s and
fraction of HBM peak), the roofline of the dominant kernel, the end-to-end
time through the host-buffer entry point, and the CPU oracle as a baseline.

usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload cube64]
Multi-GPU (torchrun): each rank solves its own replica (no collective on the
data path; the path shards into independent problems), time = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vmult GDoF/s & %HBM peak; Stokes solve s to 1e-8 rel (FP32 vs FP64 GMG)"
RTOL = 1e-8
# Algorithmic flops per cell of the velocity operator A by sum factorisation as implemented
# (multiply-add = 2 flops): 36 sweeps of 9 lines. Interpolations and their transposes (18
# sweeps): 3 outputs x 3 MACs per line. Derivatives (9 sweeps): the outer outputs 3 MACs, the
# middle one a difference times a constant (the derivative matrix at symmetric Gauss points is
# antisymmetric, its centre 0), 2 flops. Transposed derivatives (9): 3 MACs, and a difference
# and one MAC, 3 flops.
A_FLOP_PER_CELL = 18 * 9 * 18 + 9 * 9 * (12 + 2) + 9 * 9 * (12 + 3)
# Outer operator [A B^T; B 0]: B^T and B as tensor products of 3x2 moment matrices, 3
# components x 114 MACs each.
STOKES_FLOP_PER_CELL = A_FLOP_PER_CELL + 2 * (342 + 342)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube64")
    ap.add_argument("--no-extras", action="store_true", help="skip the sweep/profile/e2e/cpu legs")
    ap.add_argument("--no-large", action="store_true", help="skip the 128^3 vmult and solve leg")
    ap.add_argument("--vmult-sweep", action="store_true",
                    help="finest-level velocity operator A, FP32 and FP64, on uniform meshes of 16..128 cells per "
                         "axis (8 sinkers, viscosity ratio 1e4); one JSON line per size")
    ap.add_argument("--solve-report", action="store_true",
                    help="one FP32-V-cycle and one FP64-V-cycle solve of the workload: iterations, times, "
                         "true FP64 residuals and the difference of the two solutions (any size)")
    ap.add_argument("--outer", default="fgmres", choices=["fgmres", "idr", "gmres", "both", "all"],
                    help="with --solve-report: outer solver(s) of the FP32/FP64 V-cycle solves (idr = IDR(2), "
                         "gmres = GMRES(50) with the fixed preconditioner; both = idr + fgmres; all = the three). "
                         "--precond both adds MINRES with P_D next to FGMRES with P_D")
    ap.add_argument("--fp32-only", action="store_true",
                    help="with --solve-report: skip the FP64-V-cycle legs (largest problems)")
    ap.add_argument("--schur-degree", type=int, default=None,
                    help="with --solve-report: S_hat^-1 Chebyshev degree of the main solver (0 = diag(M_p))")
    ap.add_argument("--precond", default="triangular", choices=["triangular", "both"],
                    help="with --solve-report: 'both' adds FP32-V-cycle solves with the block-diagonal P_D "
                         "(Table 1 comparison)")
    ap.add_argument("--kernels", action="store_true",
                    help="profiling case: set up the workload, run 3 FP32 vmults, 2 FP64 Stokes applies, "
                         "1 FP32 V-cycle and 1 preconditioner application, print one line and exit (for ncu); "
                         "no Krylov basis is allocated")
    ap.add_argument("--kernels-gs", action="store_true",
                    help="with --kernels: also 40 FGMRES iterations (Gram-Schmidt passes up to a 40-vector basis)")
    ap.add_argument("--vmult-kernel", type=int, default=None,
                    help="with --kernels: level operator (0 cell kernel, 1 brick, 2 tensor cores)")
    ap.add_argument("--outer-arith", type=int, default=None,
                    help="with --kernels: outer operator (0 native FP64, 1 double-float, 2 tensor-core digit slices)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest `value` over all ranks (every rank gets it); `value` itself without a process
    group. The replicas' step time is the slowest rank's."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, n_dofs, ms):
    """Whole-job GDoF/s of `world` replicas that each solve n_dofs in `ms` (the slowest rank's time)."""
    return world * n_dofs / (ms / 1e3) / 1e9


# ----------------------------------------------------------------- clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(index):
    path = tempfile.mktemp(suffix=".csv")
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + CLOCK_Q, "--format=csv,noheader,nounits",
                              "-lms", "200"], stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except (FileNotFoundError, OSError):
        return None, path
    return p, path


def clocks_stop(p, path):
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    time.sleep(0.25)
    p.terminate()
    p.wait()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for name, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(name)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# Sources that define each profiled kernel class (a recorded ncu traffic figure is used only
# while these files are unchanged).
KERNEL_SOURCES = {
    "stokes_df64": ("q2_basis.cuh", "df64.cuh", "outer.cuh", "outer.cu"),
    "stokes_df64_inst": ("q2_basis.cuh", "df64.cuh", "outer.cuh", "outer.cu"),
    "stokes_fp64": ("q2_basis.cuh", "ops.cu"),
    "vmult_A_fp32": ("q2_basis.cuh", "brick.cuh", "brick.cu"),
    "krylov_vec": ("krylov.cu", "vec.cu"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_1907_06696_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel source."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    e = rec.get(kernel, {}).get(workload)
    if not e or kernel not in KERNEL_SOURCES or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e.get("bytes_per_launch")


def krylov_alg_bytes(N, its, m, delayed=True):
    """Algorithmic HBM bytes of the FGMRES vector kernels over a solve of `its` iterations with
    restart m: per cycle the residual (w = b - K x: 3 vectors, |w|: 1) and V_0 = w / beta (2);
    per iteration with k = j + 1 basis vectors the FP64 copy of row j for the preconditioner (2)
    and the Gram-Schmidt passes: delayed re-orthogonalisation (option gram_schmidt 1) reads the
    k rows and w twice and writes rows j and j + 1, (k + 1) + (k + 3); three passes read them
    three times, (k + 1) + (k + 2) and (k + 2) more when V_k is formed (k < m); x += Z y, k + 2;
    and the final residual."""
    vecs, left = N, its   # |b|
    while left > 0:
        kc = min(m, left)
        vecs += 6 * N
        for k in range(1, kc + 1):
            if delayed:
                vecs += (2 * k + 6) * N
            else:
                vecs += (2 * k + 5) * N + ((k + 2) * N if k < m else 0)
        vecs += (kc + 2) * N
        left -= kc
    vecs += 4 * N
    return 8 * vecs


# ----------------------------------------------------------------- CPU oracle legs
def oracle_iterations(name):
    try:
        return json.load(open(os.path.join(ROOT, "oracle", "iteration_counts.json")))[name]["iterations"]
    except (OSError, ValueError, KeyError):
        return None


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


# ----------------------------------------------------------------- reference arm
def workload_config(prob, n_u, n_p):
    """The workload and method, shared by both arms' `config` (implementation details of our arm
    go to its `impl_config`)."""
    return {"workload": prob.name, "n": prob.n, "levels": prob.n_levels, "sinkers": prob.n_sinkers,
            "dr": prob.mu_max / prob.mu_min, "n_u": int(n_u), "n_p": int(n_p), "rtol": RTOL,
            "vcycle": "fp32", "outer": "fp64 FGMRES(50)", "cheb_degree": 4, "schur": "Chebyshev degree 5 on M_p"}


# basis rows the Gram-Schmidt step of the timed oracle iteration runs against: the mean over a
# restart cycle of FGMRES(50) (iteration j projects against j + 1 rows)
ORACLE_GS_ROWS = 25


def _oracle_setup(prob):
    import numpy as np
    from oracle import gmg, krylov, mesh, operators, sinker
    m = mesh.Mesh(prob.n)
    mus = sinker.level_viscosities(m, prob, prob.n_levels)
    G = gmg.GMG(prob.n, prob.n_levels, mus)
    ops = G.levels[-1].ops
    Pc = krylov.StokesPreconditioner(ops, G)
    N = m.n_u + m.n_p
    V = np.empty((ORACLE_GS_ROWS, N))
    for i in range(ORACLE_GS_ROWS):
        V[i] = np.sin(np.arange(N) * (0.37 + 0.11 * i))
        V[i] /= np.linalg.norm(V[i])
    return ops, Pc, V, N


def _oracle_iteration(ops, Pc, V, v):
    """One iteration of the oracle's FGMRES (krylov.fgmres): z = P^-1 v (V-cycle, S_hat^-1,
    B^T), w = K z, modified Gram-Schmidt of w against the basis rows, its norm."""
    import numpy as np
    z = Pc.apply(v)
    w = ops.apply_stokes(z)
    for i in range(V.shape[0]):
        w = w - (w @ V[i]) * V[i]
    return np.linalg.norm(w)


def _oracle_steps(prob, warmup, steps):
    """Mean seconds of one oracle FGMRES iteration on the full workload (set-up untimed)."""
    ops, Pc, V, N = _oracle_setup(prob)
    v = V[0].copy()
    ts = []
    for i in range(warmup + steps):
        t = time.perf_counter()
        _oracle_iteration(ops, Pc, V, v)
        if i >= warmup:
            ts.append(time.perf_counter() - t)
    return ts, N


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import sinker_inputs as si
    prob = si.workload(args.workload)
    its = oracle_iterations(args.workload)
    if its is None:
        print(json.dumps({"impl": "reference", "unavailable": "no recorded oracle iteration count for %s "
                          "(run python -m oracle.solve_workload %s)" % (args.workload, args.workload)}))
        return
    # each step: one FGMRES iteration of the oracle on the full workload (one shared set-up); the
    # solve throughput scales the measured mean by the oracle's recorded iteration count
    ts, ndof = _oracle_steps(prob, args.warmup, args.steps)
    t_it = statistics.mean(ts)
    value = ndof / (t_it * its) / 1e9
    sample = ("1 FGMRES iteration of the numpy/scipy FP64 oracle per step on the full %s workload: "
              "P^-1 (V-cycle, S_hat^-1, B^T), K z, modified Gram-Schmidt against %d basis rows; "
              "value = N / (mean step time x the oracle's recorded %d iterations)"
              % (args.workload, ORACLE_GS_ROWS, its))
    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_it * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(prob, si.n_velocity(prob.n), si.n_pressure(prob.n)),
            "extrapolation": {"iterations_per_solve": its, "solve_s": t_it * its,
                              "step_ms": [round(t * 1e3, 1) for t in ts]},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        dist = None
        torch.cuda.set_device(0)
    from paper_1907_06696_gb300 import build as B
    if local_rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    from paper_1907_06696_gb300 import capi
    capi.load()
    import sinker_inputs as si

    prob = si.workload(args.workload)
    stream = torch.cuda.current_stream()
    ctx = capi.stokes_setup_problem(prob, stream=stream)
    # autotune the launch shape of the level operator only (the method, incl. degree 4, is unchanged)
    tuned_block, _ = capi.stokes_autotune(ctx, 1, stream=stream)
    n_u, n_p = ctx.n_u, ctx.n_p
    N = n_u + n_p
    up = torch.zeros(N, dtype=torch.float64, device="cuda")
    FP32, FP64 = capi.STOKES_FP32, capi.STOKES_FP64

    def solve(prec):
        up.zero_()
        return capi.stokes_solve(ctx, prec, None, up, rtol=RTOL, max_it=2000, stream=stream)

    for _ in range(args.warmup):
        info = solve(FP32)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk, clk_path = clocks_start(torch.cuda.current_device())
    time.sleep(0.3)
    l0 = capi.stokes_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    its = []
    for _ in range(args.steps):
        info = solve(FP32)
        its.append(info.iterations)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = capi.stokes_launch_count() - l0
    clocks = clocks_stop(clk, clk_path)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    if dist is not None:
        dist.barrier()
    value = replica_throughput(world, N, ms)
    true_res32 = info.rel_residual_true
    if rank != 0:
        return
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    hbm_src = "of measured" if "hbm_gbs" in pk else "of fallback"
    dopt = capi.stokes_default_options()
    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "df64 outer (FP64 true residual) + f32 V-cycle", "data": "synthetic",
            "config": workload_config(prob, n_u, n_p),
            "impl_config": {"parallelism": "replicas" if world > 1 else "1 GPU", "cell_block": tuned_block,
                            "vmult_kernel": VMULT_KERNELS.get(dopt.vmult_kernel, dopt.vmult_kernel),
                            "outer_arith": "double-float on FP32 pipes (~47-bit significand), restart and final "
                                           "residuals native FP64" if dopt.outer_arith == 1 else "native FP64",
                            "l2": "working set %.1f GB > L2 (no flush needed)" % (N * 8 * 103 / 1e9)},
            "solve": {"fp32_vcycle_s": ms / 1e3, "fp32_vcycle_iterations": its,
                      "fp32_true_rel_residual": true_res32},
            "gpu_launches": int(launches), "clocks": clocks}
    if args.no_extras:
        print(json.dumps(line))
        return

    # --- FP64 V-cycle solve (same FGMRES), one timed solve; the two solutions' difference
    sol32 = up.clone()
    e0.record(stream)
    info64 = solve(FP64)
    e1.record(stream)
    torch.cuda.synchronize()
    line["solve"].update({"fp64_vcycle_s": e0.elapsed_time(e1) / 1e3, "fp64_vcycle_iterations": info64.iterations,
                          "fp64_true_rel_residual": info64.rel_residual_true})
    line["solve"]["fp32_speedup_vs_fp64_gmg"] = line["solve"]["fp64_vcycle_s"] / line["solve"]["fp32_vcycle_s"]
    line["accuracy"] = {args.workload + "_fp32_vs_fp64_vcycle": solution_difference(sol32, up, n_u)}
    del sol32

    # --- standalone vmult (finest level) at the bench workload: vectors of 64^3 fit in L2
    vm64 = time_vmult(capi, ctx, prob.n, n_u, stream, hbm)
    line["vmult_l2_resident"] = dict(vm64, workload=args.workload,
                                     note="src + dst fit in the 126 MB L2: an L2 figure, not an HBM one")

    # --- profiled solve: time share per kernel class inside the step
    cells = prob.n ** 3
    capi.stokes_profile(1)
    capi.stokes_profile_read(reset=True)
    solve(FP32)
    torch.cuda.synchronize()
    prof = capi.stokes_profile_read(reset=True)
    capi.stokes_profile(0)
    tot = sum(v[0] for v in prof.values())
    line["kernel_share"] = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / tot, 4)}
                            for k, v in prof.items() if v[1]}
    # live FMA peaks of this GPU (FMA-chain probe), for the ALU side of the roofline
    f32_peak, f64_peak = capi.stokes_probe_fma()
    line["alu_peaks_tflops"] = {"fp32": f32_peak, "fp64": f64_peak, "how": "stokes_probe_fma: 8 FMA chains/thread"}
    line["roofline"] = dominant_roofline(prof, dopt, cells, n_u, N, hbm, hbm_src, f32_peak, f64_peak, args.workload)

    # class-level roofline of the FGMRES vector kernels: algorithmic bytes of their passes over
    # the profiled solve / their summed time
    kb = krylov_alg_bytes(N, its[-1], dopt.restart,
                          dopt.gram_schmidt == 1 and dopt.outer_arith == 1 and dopt.restart <= 64)
    kt = prof["krylov_vec"][0] / 1e3
    line["roofline_krylov"] = {"kernels": "k_gs_df (Gram-Schmidt passes), k_gs_final, k_df_*, k_axpby, norms",
                               "bound": "hbm", "achieved": kb / kt / 1e9, "peak": hbm, "unit": "GB/s",
                               "frac": kb / kt / 1e9 / hbm, "peak_note": hbm_src,
                               "bytes": "%.1f GB algorithmic over %d launches" % (kb / 1e9, prof["krylov_vec"][1])}

    # --- autotuned Chebyshev degree (a different smoother than the paper's degree 4), one solve
    dctx = capi.stokes_setup_problem(prob, stream=stream)
    tb, tdeg = capi.stokes_autotune(dctx, 3, stream=stream)
    up.zero_()
    capi.stokes_solve(dctx, FP32, None, up, rtol=RTOL, max_it=2000, stream=stream)   # graph capture
    up.zero_()
    e0.record(stream)
    tinfo = capi.stokes_solve(dctx, FP32, None, up, rtol=RTOL, max_it=2000, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    line["autotuned"] = {"cheb_degree": tdeg, "cell_block": tb, "solve_s": e0.elapsed_time(e1) / 1e3,
                         "iterations": tinfo.iterations, "true_rel_residual": tinfo.rel_residual_true}
    dctx.close()

    # --- end to end through the host-buffer entry point (pinned host memory)
    rhs_h = torch.zeros(N, dtype=torch.float64, pin_memory=True)
    Fd = torch.empty(n_u, dtype=torch.float64, device="cuda")
    capi.stokes_get_rhs(ctx, Fd, stream=stream)
    torch.cuda.synchronize()
    rhs_h[:n_u].copy_(Fd.cpu())
    out_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
    capi.stokes_solve_host(ctx, FP32, rhs_h.numpy(), out_h.numpy(), rtol=RTOL, max_it=2000, stream=stream)
    e0.record(stream)
    for _ in range(args.steps):
        capi.stokes_solve_host(ctx, FP32, rhs_h.numpy(), out_h.numpy(), rtol=RTOL, max_it=2000, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ems = e0.elapsed_time(e1) / args.steps
    line["e2e"] = {"value": N / (ems / 1e3) / 1e9, "unit": "GDoF/s", "ms_per_step": ems,
                   "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8}
    ctx.close()
    del up
    torch.cuda.empty_cache()

    # --- each result's error against the FP64 oracle's solution where the oracle can solve
    for name in ("cube8", "cube16"):
        ref = stored_oracle_solution(name)
        if ref is None:
            continue
        sp = si.workload(name)
        sctx = capi.stokes_setup_problem(sp, stream=stream)
        acc = {}
        for tag, prec in (("fp32_vcycle", FP32), ("fp64_vcycle", FP64)):
            x = torch.zeros(sctx.n_u + sctx.n_p, dtype=torch.float64, device="cuda")
            inf = capi.stokes_solve(sctx, prec, None, x, rtol=RTOL, max_it=2000, stream=stream)
            acc[tag] = dict(solution_difference(x, torch.from_numpy(ref).cuda(), sctx.n_u),
                            iterations=inf.iterations, true_rel_residual=inf.rel_residual_true)
        line["accuracy"][name + "_vs_oracle_solution"] = acc
        sctx.close()
    line["accuracy"]["note"] = ("relative 2-norm differences of velocity and pressure; the oracle's FGMRES "
                                "solution to 1e-12 (oracle/solutions/, written by oracle/solve_workload.py)")

    # --- the 128^3 configuration: above-L2 vmult (the HBM figure) and one FP32-V-cycle solve
    if not args.no_large:
        line.update(run_large(capi, si, torch, stream, hbm, hbm_src))
        line["refinement"] = run_refinement(capi, si, torch, stream)

    # --- CPU oracle baseline: bounded sample, scaled to a solve
    its_ref = oracle_iterations(args.workload)
    try:
        ts, ndof = _oracle_steps(prob, 0, 3)
        t_it = statistics.mean(ts)
        n_it = its_ref if its_ref else its[-1]
        line["cpu_baseline"] = {"value": ndof / (t_it * n_it) / 1e9, "unit": "GDoF/s", "cores": cpu_threads(),
                                "kind": "oracle",
                                "sample": "3 FGMRES iterations of the numpy/scipy FP64 oracle on the full %s "
                                          "workload (set-up untimed; P^-1, K z, modified Gram-Schmidt against %d "
                                          "basis rows), %.2f s each, scaled by %d iterations%s"
                                          % (args.workload, ORACLE_GS_ROWS, t_it, n_it,
                                             " (oracle's recorded count)" if its_ref else " (GPU FP32 count)")}
    except MemoryError as e:
        line["cpu_baseline"] = {"value": None, "unit": "GDoF/s", "cores": cpu_threads(), "kind": "oracle",
                                "sample": "failed: %s" % e}
    print(json.dumps(line))


VMULT_KERNELS = {0: "k_cell_atomic (one thread per cell, FP32 pipes, atomic scatter)",
                 1: "k_brick + k_planes (brick-tiled, deterministic)",
                 2: "k_cell_tc (cell products on the tensor cores, tcgen05 kind::f16, shared-memory node tile)"}


def solution_difference(x, ref, n_u):
    """Relative 2-norm differences of the velocity and pressure parts of two solutions."""
    import torch
    du = torch.linalg.vector_norm(x[:n_u] - ref[:n_u]) / torch.linalg.vector_norm(ref[:n_u])
    dp = torch.linalg.vector_norm(x[n_u:] - ref[n_u:]) / torch.linalg.vector_norm(ref[n_u:])
    return {"u_rel": float(du), "p_rel": float(dp)}


def stored_oracle_solution(name):
    import numpy as np
    path = os.path.join(ROOT, "oracle", "solutions", name + ".npy")
    return np.load(path) if os.path.exists(path) else None


def time_vmult(capi, ctx, n, n_u, stream, hbm, reps=(20, 5)):
    """Finest-level dst = A src, FP32 and FP64: CUDA-event time of the whole call (zeroing the
    output, the operator kernel, the identity rows) and of the operator kernel alone (profiled
    class), algorithmic bytes (2 N_u + cells) x size / kernel time against the HBM peak."""
    import torch
    cells = n ** 3
    x32 = torch.rand(n_u, device="cuda", dtype=torch.float32)
    y32 = torch.empty_like(x32)
    x64 = x32.double()
    y64 = torch.empty_like(x64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for tag, prec, x, y, sz, r in (("fp32", capi.STOKES_FP32, x32, y32, 4, reps[0]),
                                   ("fp64", capi.STOKES_FP64, x64, y64, 8, reps[1])):
        for _ in range(3):
            capi.stokes_vmult(ctx, -1, capi.BLOCK_A, prec, x, y, stream=stream)
        capi.stokes_profile(1)
        capi.stokes_profile_read(reset=True)
        e0.record(stream)
        for _ in range(r):
            capi.stokes_vmult(ctx, -1, capi.BLOCK_A, prec, x, y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = capi.stokes_profile_read(reset=True)
        capi.stokes_profile(0)
        t_call = e0.elapsed_time(e1) / r / 1e3
        kname = "vmult_A_" + tag
        # one operator application = the cell kernel (+ the brick-plane kernel of the brick variant)
        t_kern = (prof[kname][0] + prof["smoother_vec"][0]) / max(prof[kname][1], 1) / 1e3
        bytes_alg = (2 * n_u + cells) * sz
        out[tag] = {"gdofs": n_u / t_call / 1e9, "call_ms": t_call * 1e3, "kernel_ms": t_kern * 1e3,
                    "kernel_gdofs": n_u / t_kern / 1e9, "algorithmic_bytes": bytes_alg,
                    "achieved_gbs": bytes_alg / t_kern / 1e9, "hbm_frac": bytes_alg / t_kern / 1e9 / hbm,
                    "call_hbm_frac": bytes_alg / t_call / 1e9 / hbm,
                    "gflops": cells * A_FLOP_PER_CELL / t_kern / 1e9}
    out["peak_gbs"] = hbm
    return out


def dominant_roofline(prof, dopt, cells, n_u, N, hbm, hbm_src, f32_peak, f64_peak, workload):
    """Roofline of the single kernel with the largest time in the profiled solve. achieved =
    algorithmic bytes per launch / its mean launch time, against the measured HBM peak; the ALU
    side (method flops against the FMA probe) beside it."""
    single = ("stokes_fp64", "vmult_A_fp32")
    dom = max(single, key=lambda k: prof.get(k, (0.0, 0))[0])
    dms = prof[dom][0] / max(prof[dom][1], 1)
    if dom == "stokes_fp64":
        bytes_alg = (2 * N + cells) * 8
        fl = cells * STOKES_FLOP_PER_CELL
        df = dopt.outer_arith == 1
        r = {"kernel": "k_outer_df64<1,1,1> (outer [A B^T; B 0], double-float)" if df else
                       "k_stokes_blocks<double,1,1,1> (outer [A B^T; B 0], FP64)",
             "bound": "hbm", "achieved": bytes_alg / (dms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
             "frac": bytes_alg / (dms / 1e3) / 1e9 / hbm,
             "traffic": recorded_traffic("stokes_df64" if df else "stokes_fp64", workload),
             "peak_note": hbm_src, "launch_ms": dms,
             "per_launch": "(2 (N_u + N_p) + cells) x 8 B = %d B (u, p read and written in FP64, cell viscosity)"
                           % bytes_alg}
        alu_peak = f32_peak if df else f64_peak
        r["alu"] = {"method_flop_per_cell": STOKES_FLOP_PER_CELL, "achieved_gflops": fl / (dms / 1e3) / 1e9,
                    "peak_gflops": alu_peak * 1e3, "frac": fl / (dms / 1e3) / 1e9 / (alu_peak * 1e3),
                    "peak_note": "of measured (%s probe, this run); the FP64 method flops %s"
                                 % ("FFMA" if df else "DFMA",
                                    "run as double-float on the FP32 pipes, several FP32 instructions each"
                                    if df else "on the FP64 pipe")}
        inst = recorded_traffic("stokes_df64_inst" if df else "stokes_fp64_inst", workload)
        if inst:
            ips = inst / (dms / 1e3)
            r["issue"] = {"thread_inst_per_launch": inst, "frac": ips / (f32_peak / 2 * 1e12),
                          "note": "instructions per launch (ncu smsp__inst_executed.sum x 32) against the "
                                  "FFMA probe's instruction rate (FMA = 1 instruction): the issue efficiency "
                                  "of the double-float code"}
        return r
    bytes_alg = (2 * n_u + cells) * 4
    return {"kernel": dom, "bound": "hbm", "achieved": bytes_alg / (dms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": bytes_alg / (dms / 1e3) / 1e9 / hbm, "traffic": recorded_traffic(dom, workload),
            "peak_note": hbm_src, "launch_ms": dms,
            "per_launch": "finest-level (2 N_u + cells) x 4 B = %d B (mean over the solve's levels is lower)"
                          % bytes_alg}


def run_refinement(capi, si, torch, stream):
    """One problem (16 sinkers, viscosity ratio 1e6, 3^3 coarsest mesh) on 24^3, 48^3, 96^3 cells:
    FP32-V-cycle FGMRES(50) iterations, time and true residual per mesh (Section 3.5: iteration
    counts stay constant under refinement)."""
    rows = []
    for name in ("seq24", "seq48", "seq96"):
        p = si.workload(name)
        ctx = capi.stokes_setup_problem(p, stream=stream)
        up = torch.zeros(ctx.n_u + ctx.n_p, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=3000, stream=stream, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        rows.append({"workload": name, "n": p.n, "dofs": ctx.n_u + ctx.n_p, "iterations": info.iterations,
                     "s": e0.elapsed_time(e1) / 1e3, "status": info.status,
                     "true_rel_residual": info.rel_residual_true})
        ctx.close()
        del up
        torch.cuda.empty_cache()
    return {"meshes": rows, "note": "first solve on each context (includes the V-cycle graph capture)"}


def run_large(capi, si, torch, stream, hbm, hbm_src, name="cube128"):
    """The 128^3 configuration (16 sinkers, viscosity ratio 1e6, 8 levels): the standalone vmult with
    vectors far above L2 (the HBM figure) and one FP32-V-cycle FGMRES solve to 1e-8 with its true
    residual from the native FP64 operator."""
    prob = si.workload(name)
    t0 = time.perf_counter()
    ctx = capi.stokes_setup_problem(prob, stream=stream)
    setup_s = time.perf_counter() - t0
    n_u, n_p = ctx.n_u, ctx.n_p
    vm = time_vmult(capi, ctx, prob.n, n_u, stream, hbm)
    vm.update({"workload": name, "peak_note": hbm_src,
               "note": "src + dst = %.0f MB FP32, above the 126 MB L2" % (2 * n_u * 4 / 1e6)})
    up = torch.zeros(n_u + n_p, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=3000, stream=stream, check=False)
    e1.record(stream)
    torch.cuda.synchronize()
    solve = {"workload": name, "n_u": n_u, "n_p": n_p, "levels": prob.n_levels, "dr": prob.mu_max / prob.mu_min,
             "sinkers": prob.n_sinkers, "setup_s": setup_s, "fp32_vcycle_s": e0.elapsed_time(e1) / 1e3,
             "iterations": info.iterations, "status": info.status,
             "true_rel_residual": info.rel_residual_true,
             "note": "first solve on the context (includes the V-cycle graph capture); true residual from the "
                     "library's native FP64 operator"}
    ctx.close()
    del up
    torch.cuda.empty_cache()
    return {"vmult": vm, "solve_" + name: solve}


def run_kernels(args):
    import torch
    from paper_1907_06696_gb300 import build as B
    B.build()
    from paper_1907_06696_gb300 import capi
    capi.load()
    import sinker_inputs as si
    if args.workload.startswith("oct"):
        # adaptive case: 2 outer applies (constrained FP64 blocks), 3 finest-level FP32 products, 1 V-cycle
        prob = si.octree_workload(args.workload)
        ctx = capi.stokes_setup_octree_problem(prob)
        N = ctx.n_u + ctx.n_p
        up = torch.rand(N, device="cuda", dtype=torch.float64)
        out = torch.empty_like(up)
        for _ in range(2):
            capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, up, out)
        NL = ctx.size(-1, 4)
        xf = torch.rand(ctx.size(NL - 1, 0), device="cuda", dtype=torch.float32)
        yf = torch.empty_like(xf)
        for _ in range(3):
            capi.stokes_vmult(ctx, NL - 1, capi.BLOCK_A, capi.STOKES_FP32, xf, yf)
        xu = torch.empty(ctx.n_u, device="cuda", dtype=torch.float64)
        capi.gmg_vcycle(ctx, capi.STOKES_FP32, up[:ctx.n_u], xu)
        torch.cuda.synchronize()
        print(json.dumps({"kernels": args.workload, "n_u": ctx.n_u, "n_p": ctx.n_p, "leaves": ctx.size(-1, 2)}))
        return
    prob = si.workload(args.workload)
    opt = capi.stokes_default_options()
    if args.vmult_kernel is not None:
        opt.vmult_kernel = args.vmult_kernel
    if args.outer_arith is not None:
        opt.outer_arith = args.outer_arith
    ctx = capi.stokes_setup_problem(prob, options=opt)
    n_u, n_p = ctx.n_u, ctx.n_p
    x = torch.rand(n_u, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    for _ in range(3):
        capi.stokes_vmult(ctx, -1, capi.BLOCK_A, capi.STOKES_FP32, x, y)
    up = torch.rand(n_u + n_p, device="cuda", dtype=torch.float64)
    out = torch.empty_like(up)
    for _ in range(2):
        capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, up, out)
    capi.gmg_vcycle(ctx, capi.STOKES_FP32, x, y)
    # one preconditioner application: S_hat^-1 steps, B^T, the FP32 V-cycle
    z = torch.empty_like(up)
    capi.stokes_precondition(ctx, capi.STOKES_FP32, up, z)
    if args.kernels_gs:
        # 40 FGMRES iterations: Gram-Schmidt passes up to a 40-vector basis
        up.zero_()
        try:
            capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-14, max_it=40)
        except capi.StokesError as e:
            if e.status != capi.STOKES_NOT_CONVERGED:
                raise
    capi.stokes_device_status(ctx)
    torch.cuda.synchronize()
    print(json.dumps({"kernels": args.workload, "n_u": n_u, "n_p": n_p}))


def run_batch(args):
    """Batched workload: many independent sinker problems of uneven sizes solved together with the
    FP32 V-cycle (stokes_batch_solve) -- one captured V-cycle graph per problem (batch_vcycle 0, the
    default, timed over the steps) and the V-cycles as one persistent launch per round
    (batch_vcycle 1) -- against the same problems solved one after the other with the FP32 and with
    the FP64 V-cycle. batch64s draws the sizes 16^3..24^3 only."""
    import torch
    from paper_1907_06696_gb300 import build as B
    B.build()
    from paper_1907_06696_gb300 import capi
    capi.load()
    import sinker_inputs as si
    small = args.workload.endswith("s")
    count = int(args.workload[len("batch"):].rstrip("s") or 64)
    probs = si.batch_workload(count, sizes=si.BATCH_SIZES_SMALL if small else si.BATCH_SIZES)
    ctxs = [capi.stokes_setup_problem(p) for p in probs]
    ups = [torch.zeros(c.n_u + c.n_p, dtype=torch.float64, device="cuda") for c in ctxs]
    ndof = sum(c.n_u + c.n_p for c in ctxs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def batch(mode):
        for c in ctxs:
            capi.stokes_set_batch_vcycle(c, mode)
        for u in ups:
            u.zero_()
        return capi.stokes_batch_solve(ctxs, capi.STOKES_FP32, ups, rtol=RTOL, max_it=3000)

    # the default: one captured V-cycle graph per problem on its own stream
    for _ in range(max(args.warmup, 1)):
        batch(0)
    torch.cuda.synchronize()
    clk, clk_path = clocks_start(torch.cuda.current_device())
    l0 = capi.stokes_launch_count()
    e0.record()
    for _ in range(args.steps):
        infos = batch(0)
    e1.record()
    torch.cuda.synchronize()
    launches = capi.stokes_launch_count() - l0
    clocks = clocks_stop(clk, clk_path)
    ms = e0.elapsed_time(e1) / args.steps
    # the same batch with the persistent batched V-cycle kernel (batch_vcycle 1)
    batch(1)
    torch.cuda.synchronize()
    e0.record()
    kinfos = batch(1)
    e1.record()
    torch.cuda.synchronize()
    kernel_ms = e0.elapsed_time(e1)
    # the same problems one after the other, FP32 and FP64 V-cycle
    seq = {}
    for tag, prec in (("fp32", capi.STOKES_FP32), ("fp64", capi.STOKES_FP64)):
        its = []
        e0.record()
        for c, u in zip(ctxs, ups):
            u.zero_()
            its.append(capi.stokes_solve(c, prec, None, u, rtol=RTOL, max_it=3000).iterations)
        e1.record()
        torch.cuda.synchronize()
        seq[tag] = (e0.elapsed_time(e1), its)
    line = {"metric": METRIC, "value": ndof / (ms / 1e3) / 1e9, "unit": "GDoF/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "df64 outer (FP64 true residual) + f32 V-cycle", "data": "synthetic",
            "config": {"workload": args.workload, "problems": count,
                       "sizes": sorted(set(p.n for p in probs)), "total_dofs": ndof, "rtol": RTOL},
            "batch": {"fp32_batch_graphs_s": ms / 1e3, "iterations": [i.iterations for i in infos],
                      "max_true_rel_residual": max(i.rel_residual_true for i in infos),
                      "fp32_batch_kernel_s": kernel_ms / 1e3, "kernel_iterations": [i.iterations for i in kinfos],
                      "fp32_sequential_s": seq["fp32"][0] / 1e3, "fp32_sequential_iterations": seq["fp32"][1],
                      "fp64_sequential_s": seq["fp64"][0] / 1e3, "fp64_sequential_iterations": seq["fp64"][1],
                      "batching_gain_vs_sequential_fp32": seq["fp32"][0] / ms,
                      "kernel_gain_vs_graphs": ms / kernel_ms,
                      "speedup_vs_sequential_fp64": seq["fp64"][0] / ms},
            "gpu_launches": int(launches), "clocks": clocks}
    for c in ctxs:
        c.close()
    print(json.dumps(line))


def run_report(args):
    import torch
    from paper_1907_06696_gb300 import build as B
    B.build()
    from paper_1907_06696_gb300 import capi
    capi.load()
    import sinker_inputs as si
    prob = si.workload(args.workload)
    t0 = time.perf_counter()
    opts = capi.stokes_default_options()
    solver_id = {"fgmres": 0, "idr": 1, "gmres": 2}
    names = {0: "FGMRES(50)", 1: "IDR(2)", 2: "GMRES(50)"}
    opts.outer_solver = solver_id.get(args.outer, 0)
    if args.schur_degree is not None:
        opts.schur_degree = args.schur_degree
    ctx = capi.stokes_setup_problem(prob, options=opts)
    setup_s = time.perf_counter() - t0
    N = ctx.n_u + ctx.n_p
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"outer": names[opts.outer_solver], "schur_degree": opts.schur_degree}
    sols = {}
    extra = {"both": ("idr",), "all": ("idr", "gmres")}.get(args.outer, ())
    for other in extra:   # other solvers first, each on a context of its own (main basis not allocated yet)
        oi = capi.stokes_default_options()
        oi.outer_solver = solver_id[other]
        ci = capi.stokes_setup_problem(prob, options=oi)
        legs = ((other + "_fp32_vcycle", capi.STOKES_FP32),) if args.fp32_only else \
            ((other + "_fp32_vcycle", capi.STOKES_FP32), (other + "_fp64_vcycle", capi.STOKES_FP64))
        for tag, prec in legs:
            up = torch.zeros(N, dtype=torch.float64, device="cuda")
            for _ in range(min(args.warmup, 1)):
                capi.stokes_solve(ci, prec, None, up, rtol=RTOL, max_it=5000, check=False)
                up.zero_()
            e0.record()
            info = capi.stokes_solve(ci, prec, None, up, rtol=RTOL, max_it=5000, check=False)
            e1.record()
            torch.cuda.synchronize()
            out[tag] = {"s": e0.elapsed_time(e1) / 1e3, "iterations": info.iterations, "status": info.status,
                        "true_rel_residual": info.rel_residual_true}
            del up
        ci.close()
        torch.cuda.empty_cache()
    legs = (("fp32_vcycle", capi.STOKES_FP32),) if args.fp32_only else \
        (("fp32_vcycle", capi.STOKES_FP32), ("fp64_vcycle", capi.STOKES_FP64))
    for tag, prec in legs:
        up = torch.zeros(N, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            up.zero_()
            capi.stokes_solve(ctx, prec, None, up, rtol=RTOL, max_it=5000)
        up.zero_()
        e0.record()
        info = capi.stokes_solve(ctx, prec, None, up, rtol=RTOL, max_it=5000, check=False)
        e1.record()
        torch.cuda.synchronize()
        out[tag] = {"s": e0.elapsed_time(e1) / 1e3, "iterations": info.iterations, "status": info.status,
                    "true_rel_residual": info.rel_residual_true}
        sols[tag] = up
    if not args.fp32_only:
        u32, u64 = sols["fp32_vcycle"][:ctx.n_u], sols["fp64_vcycle"][:ctx.n_u]
        p32, p64 = sols["fp32_vcycle"][ctx.n_u:], sols["fp64_vcycle"][ctx.n_u:]
        if args.precond == "both":
            o = capi.stokes_default_options()
            o.precond_kind = 1
            cd = capi.stokes_setup_problem(prob, options=o)
            up = torch.zeros(N, dtype=torch.float64, device="cuda")
            capi.stokes_solve(cd, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=5000, check=False)
            up.zero_()
            e0.record()
            info = capi.stokes_solve(cd, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=5000, check=False)
            e1.record()
            torch.cuda.synchronize()
            out["block_diagonal_fp32_vcycle"] = {"s": e0.elapsed_time(e1) / 1e3, "iterations": info.iterations,
                                                 "status": info.status, "true_rel_residual": info.rel_residual_true}
            cd.close()
            o.outer_solver = 3   # MINRES with the same P_D
            cd = capi.stokes_setup_problem(prob, options=o)
            up.zero_()
            capi.stokes_solve(cd, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=5000, check=False)
            up.zero_()
            e0.record()
            info = capi.stokes_solve(cd, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=5000, check=False)
            e1.record()
            torch.cuda.synchronize()
            out["minres_block_diagonal_fp32_vcycle"] = {"s": e0.elapsed_time(e1) / 1e3, "iterations": info.iterations,
                                                        "status": info.status,
                                                        "true_rel_residual": info.rel_residual_true}
            cd.close()
        out["rel_diff_u"] = float((u32 - u64).norm() / u64.norm())
        out["rel_diff_p"] = float((p32 - p64).norm() / p64.norm())
        out["speedup"] = out["fp64_vcycle"]["s"] / out["fp32_vcycle"]["s"]
    print(json.dumps({"report": args.workload, "n_u": ctx.n_u, "n_p": ctx.n_p, "setup_s": setup_s,
                      "sinkers": prob.n_sinkers, "dr": prob.mu_max / prob.mu_min, "rtol": RTOL, **out}))
    ctx.close()


def run_adapt(args):
    """Solve-estimate-refine loop (Section 3.3: from 4 global refinements, each cycle refines about
    1/7 of the cells by a gradient-based estimator): per cycle the host-side set-up time, the FP32-
    V-cycle FGMRES solve to 1e-8 on the GPU (CUDA events, after one warm-up solve), its iterations
    and true residual, and the host refinement time (stokes_octree_refine_gradient on the solved
    velocity). One JSON line per cycle, then a summary line."""
    import torch
    from paper_1907_06696_gb300 import build as B
    B.build()
    from paper_1907_06696_gb300 import capi
    capi.load()
    import sinker_inputs as si
    prob, cycles = si.adaptive_loop_workload(args.workload)
    keys = capi.stokes_octree_sinker_mesh(prob.base_level, prob.centres, prob.max_levels, prob.shell_radius,
                                          prob.shell_half_width)
    stream = torch.cuda.current_stream()
    rows = []
    for cycle in range(cycles + 1):
        t0 = time.perf_counter()
        ctx = capi.stokes_setup_octree(keys, prob.coarsest_level, prob.centres, prob.mu_min, prob.mu_max,
                                       prob.delta, prob.omega, prob.beta, stream=stream)
        setup_s = time.perf_counter() - t0
        n_u, n_p = ctx.n_u, ctx.n_p
        up = torch.zeros(n_u + n_p, dtype=torch.float64, device="cuda")
        capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=5000, stream=stream, check=False)
        up.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=RTOL, max_it=5000, stream=stream,
                                 check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        row = {"adapt": args.workload, "cycle": cycle, "leaves": int(keys.size), "n_u": n_u, "n_p": n_p,
               "setup_s": setup_s, "solve_s": e0.elapsed_time(e1) / 1e3, "iterations": info.iterations,
               "status": info.status, "true_rel_residual": info.rel_residual_true}
        if cycle < cycles:
            u = up[:n_u].cpu().numpy()
            t0 = time.perf_counter()
            keys, _ = capi.stokes_octree_refine_gradient(keys, prob.coarsest_level, u)
            row["refine_s"] = time.perf_counter() - t0
        ctx.close()
        del up
        torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"adapt": args.workload, "cycles": cycles, "sinkers": prob.n_sinkers,
                      "dr": prob.mu_max / prob.mu_min, "leaves": [r["leaves"] for r in rows],
                      "dofs": [r["n_u"] + r["n_p"] for r in rows], "iterations": [r["iterations"] for r in rows],
                      "solve_s": [r["solve_s"] for r in rows]}))


def run_octree(args):
    """Adaptive workload (octree mesh refined in shells around the sinkers, hanging nodes,
    local-smoothing GMG): host mesh and set-up times, FP32- and FP64-V-cycle solves to 1e-8,
    per-class kernel time of one solve, and the throughput of the active outer operator (FP64,
    constrained) and of the finest level operator (FP32)."""
    import torch
    from paper_1907_06696_gb300 import build as B
    B.build()
    from paper_1907_06696_gb300 import capi
    capi.load()
    import sinker_inputs as si
    prob = si.octree_workload(args.workload)
    t0 = time.perf_counter()
    keys = capi.stokes_octree_sinker_mesh(prob.base_level, prob.centres, prob.max_levels, prob.shell_radius,
                                          prob.shell_half_width)
    mesh_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx = capi.stokes_setup_octree(keys, prob.coarsest_level, prob.centres, prob.mu_min, prob.mu_max, prob.delta,
                                   prob.omega, prob.beta)
    setup_s = time.perf_counter() - t0
    n_u, n_p = ctx.n_u, ctx.n_p
    N = n_u + n_p
    NL = ctx.size(-1, 4)
    stream = torch.cuda.current_stream()
    up = torch.zeros(N, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def solve(prec):
        up.zero_()
        return capi.stokes_solve(ctx, prec, None, up, rtol=RTOL, max_it=5000, stream=stream, check=False)

    for _ in range(max(1, min(args.warmup, 3))):
        solve(capi.STOKES_FP32)
    torch.cuda.synchronize()
    clk, clk_path = clocks_start(torch.cuda.current_device())
    time.sleep(0.3)
    l0 = capi.stokes_launch_count()
    e0.record(stream)
    its = []
    for _ in range(args.steps):
        info = solve(capi.STOKES_FP32)
        its.append(info.iterations)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = capi.stokes_launch_count() - l0
    clocks = clocks_stop(clk, clk_path)
    ms = e0.elapsed_time(e1) / args.steps
    res32 = info.rel_residual_true
    st32 = info.status
    e0.record(stream)
    info64 = solve(capi.STOKES_FP64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    # one profiled FP32 solve: time per kernel class
    capi.stokes_profile(1)
    capi.stokes_profile_read(reset=True)
    solve(capi.STOKES_FP32)
    torch.cuda.synchronize()
    prof = capi.stokes_profile_read(reset=True)
    capi.stokes_profile(0)
    tot = sum(v[0] for v in prof.values())
    shares = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / tot, 4)} for k, v in prof.items() if v[1]}
    # operator throughput
    reps = 10
    x = torch.rand(N, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, x, y, stream=stream)
    e0.record(stream)
    for _ in range(reps):
        capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, x, y, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    outer_ms = e0.elapsed_time(e1) / reps
    nf = ctx.size(NL - 1, 0)
    xf = torch.rand(nf, dtype=torch.float32, device="cuda")
    yf = torch.empty_like(xf)
    capi.stokes_vmult(ctx, NL - 1, capi.BLOCK_A, capi.STOKES_FP32, xf, yf, stream=stream)
    e0.record(stream)
    for _ in range(reps):
        capi.stokes_vmult(ctx, NL - 1, capi.BLOCK_A, capi.STOKES_FP32, xf, yf, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    level_ms = e0.elapsed_time(e1) / reps
    leaves = ctx.size(-1, 2)
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    level_cells = ctx.size(NL - 1, 2)
    # algorithmic bytes of the finest level operator: src + dst (FP32) + the 27 node indices and mu per cell
    lvl_bytes = 2 * 4 * nf + level_cells * (27 * 4 + 4)
    line = {"metric": "Stokes solve s to 1e-8 rel (FP32 vs FP64 GMG), adaptive octree", "value": N / (ms / 1e3) / 1e9,
            "unit": "GDoF/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer + f32 V-cycle",
            "data": "synthetic",
            "config": {"workload": args.workload, "base_level": prob.base_level, "max_levels": [int(v) for v in prob.max_levels],
                       "sinkers": prob.n_sinkers, "dr": prob.mu_max / prob.mu_min, "leaves": leaves, "n_u": n_u,
                       "n_p": n_p, "levels": NL, "hanging_u": capi.stokes_octree_table(ctx, 6),
                       "hanging_p": capi.stokes_octree_table(ctx, 7), "rtol": RTOL,
                       "mesh_s": mesh_s, "setup_s": setup_s, "parallelism": "1 GPU",
                       "l2": "working set > L2 (no flush needed)"},
            "solve": {"fp32_vcycle_s": ms / 1e3, "fp32_vcycle_iterations": its, "fp32_true_rel_residual": res32,
                      "fp32_status": st32, "fp64_vcycle_s": ms64 / 1e3, "fp64_vcycle_iterations": info64.iterations,
                      "fp64_true_rel_residual": info64.rel_residual_true, "fp64_status": info64.status,
                      "fp32_speedup_vs_fp64_gmg": ms64 / ms},
            "operators": {"outer_fp64_ms": outer_ms, "outer_gdofs": N / (outer_ms / 1e3) / 1e9,
                          "finest_level_fp32_ms": level_ms, "finest_level_dofs": nf,
                          "finest_level_gdofs": nf / (level_ms / 1e3) / 1e9,
                          "finest_level_alg_gbs": lvl_bytes / (level_ms / 1e3) / 1e9, "peak_gbs": hbm},
            "kernel_share": shares, "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line))
    ctx.close()


SWEEP_SIZES = ((16, 5), (32, 6), (48, 5), (64, 7), (96, 6), (128, 8))   # (n, multigrid levels), n = c 2^(L-1)


def run_vmult_sweep(args):
    """Standalone velocity operator A on the finest level across mesh sizes: CUDA-event time per
    call (median of 20 after 3 warm-ups), the kernel's own time from the class profile, GDoF/s,
    algorithmic GB/s ((2 N_u + cells) x word size) and its fraction of the measured HBM peak (only
    meaningful where the vectors exceed L2, flagged), and GFLOP/s. Sources are U(0, 1)."""
    import statistics
    import torch
    from paper_1907_06696_gb300 import build as B
    B.build()
    from paper_1907_06696_gb300 import capi
    capi.load()
    import sinker_inputs as si
    torch.cuda.set_device(0)
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    l2 = getattr(torch.cuda.get_device_properties(0), "L2_cache_size", 129 * 2 ** 20)
    stream = torch.cuda.current_stream()
    for n, levels in SWEEP_SIZES:
        prob = si.dr_problem(n, levels, 8, 1e4, 1930 + n, "sweep%d" % n)
        ctx = capi.stokes_setup_problem(prob, stream=stream)
        n_u, cells = ctx.n_u, n ** 3
        out = {"sweep": "vmult_A", "n": n, "n_u": n_u, "peak_gbs": hbm,
               "peak_note": "of measured" if "hbm_gbs" in pk else "of fallback"}
        for tag, dtype, word in (("fp32", torch.float32, 4), ("fp64", torch.float64, 8)):
            prec = capi.STOKES_FP32 if tag == "fp32" else capi.STOKES_FP64
            x = torch.rand(n_u, device="cuda", dtype=dtype)
            y = torch.empty_like(x)
            for _ in range(3):
                capi.stokes_vmult(ctx, -1, capi.BLOCK_A, prec, x, y, stream=stream)
            ts = []
            for _ in range(20):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                capi.stokes_vmult(ctx, -1, capi.BLOCK_A, prec, x, y, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            capi.stokes_profile(1)
            capi.stokes_profile_read(reset=True)
            for _ in range(5):
                capi.stokes_vmult(ctx, -1, capi.BLOCK_A, prec, x, y, stream=stream)
            torch.cuda.synchronize()
            prof = capi.stokes_profile_read(reset=True)
            capi.stokes_profile(0)
            kname = "vmult_A_" + tag
            t_call = statistics.median(ts)
            t_kern = (prof[kname][0] + prof["smoother_vec"][0]) / max(prof[kname][1], 1) / 1e3
            bytes_alg = (2 * n_u + cells) * word
            out[tag] = {"call_ms": t_call * 1e3, "gdofs": n_u / t_call / 1e9, "kernel_ms": t_kern * 1e3,
                        "kernel_gdofs": n_u / t_kern / 1e9, "achieved_gbs": bytes_alg / t_kern / 1e9,
                        "hbm_frac": bytes_alg / t_kern / 1e9 / hbm, "exceeds_l2": 2 * n_u * word > l2,
                        "gflops": cells * A_FLOP_PER_CELL / t_kern / 1e9}
            del x, y
        ctx.close()
        torch.cuda.empty_cache()
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.vmult_sweep:
        run_vmult_sweep(args)
        return
    if args.solve_report:
        run_report(args)
        return
    if args.kernels:
        run_kernels(args)
    elif args.workload.startswith("oct") and args.impl != "reference":
        run_octree(args)
    elif args.workload.startswith("adapt") and args.impl != "reference":
        run_adapt(args)
    elif args.workload.startswith("batch") and args.impl != "reference":
        run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
