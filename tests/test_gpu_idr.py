"""GPU parity of the IDR(s) outer solver (option outer_solver = 1, Section 3.4) through the C ABI
against the oracle's idr_s on the same problems (same shadow space definition): FP64-V-cycle
iteration counts within 10% of the oracle's (at least 3). IDR(s) is not a minimal-residual method,
and its count moves with rounding-level changes of the operators, which differ from the oracle's
in summation order and, through the FP64 atomic scatters of the outer operator and the pressure
mass matrix, from one run to the next (with either level operator). Measured over 8 runs each
with the atomic (vmult_kernel 0) and the deterministic brick (1) level operators, oracle count in
brackets: cube8 s = 1: 33-35 [35]; s = 2: 33-35 [34]; s = 4: 31-32 [31]; cube16 s = 2: 102-106
[104].
true residuals recomputed by the oracle's operator, solutions equal to the oracle's FGMRES
solution to the accuracy the tolerance allows."""
import functools

import numpy as np
import pytest

import sinker_inputs as si
from oracle import adaptive, gmg, krylov, mesh, operators, octree, sinker

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06696_gb300 import build as B
    from paper_1907_06696_gb300 import capi as api
    B.build()
    api.load()
    return api


@functools.lru_cache(maxsize=None)
def uniform_oracle(name):
    p = si.workload(name)
    m = mesh.Mesh(p.n)
    mus = sinker.level_viscosities(m, p, p.n_levels)
    G = gmg.GMG(p.n, p.n_levels, mus)
    ops = G.levels[-1].ops
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    return p, m, G, ops, F


def idr_options(capi, sdim):
    o = capi.stokes_default_options()
    o.outer_solver = 1
    o.idr_s = sdim
    return o


@pytest.mark.parametrize("name,sdim", [("cube8", 1), ("cube8", 2), ("cube8", 4), ("cube16", 2)])
def test_idr_solve(capi, name, sdim):
    p, m, G, ops, F = uniform_oracle(name)
    b = np.concatenate([F, np.zeros(m.n_p)])
    Pc = krylov.StokesPreconditioner(ops, G)
    _, its_o, _ = krylov.idr_s(ops.apply_stokes, Pc.apply, b, s=sdim, rtol=1e-8, max_it=5000)
    xf, _, _ = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-10)
    xf = krylov.zero_mean_pressure(ops, xf)
    ctx = capi.stokes_setup_problem(p, options=idr_options(capi, sdim))
    for prec in (capi.STOKES_FP64, capi.STOKES_FP32):
        for _ in range(2):      # the workspace is reused by the second solve
            up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
            info = capi.stokes_solve(ctx, prec, None, up, rtol=1e-8, max_it=5000)
            x = up.cpu().numpy()
            true = np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b)
            assert info.status == capi.STOKES_OK
            assert true <= 1e-8 * 1.001, (prec, true)
            assert abs(info.rel_residual_true - true) <= 1e-3 * true + 1e-14
            # a relative residual of 1e-8 bounds the error only through the condition number of K:
            # IDR(s) iterates at that residual differ from the 1e-10 FGMRES solution by up to ~1e-5
            # of its largest entry (measured 1.03e-5 on cube8, s = 2), FGMRES iterates by ~4e-6
            assert np.abs(x - xf).max() <= 2e-5 * np.abs(xf).max()
            if prec == capi.STOKES_FP64:
                assert abs(info.iterations - its_o) <= max(3, 0.1 * its_o), (info.iterations, its_o)
    ctx.close()


def test_idr_octree(capi):
    p = si.octree_workload("oct_s")
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    S = adaptive.AdaptiveStokes(octree.Octree(lv, p.coarsest_level), p)
    ctx = capi.stokes_setup_octree_problem(p, options=idr_options(capi, 2))
    up = torch.zeros(S.n_u + S.n_p, dtype=torch.float64, device="cuda")
    info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=5000)
    b = np.concatenate([S.F, np.zeros(S.n_p)])
    assert info.status == capi.STOKES_OK
    assert np.linalg.norm(b - S.apply_stokes(up.cpu().numpy())) / np.linalg.norm(b) <= 1e-8 * 1.001
    ctx.close()


def test_idr_rejected_by_batch(capi):
    p, m, G, ops, F = uniform_oracle("cube8")
    ctx = capi.stokes_setup_problem(p, options=idr_options(capi, 2))
    up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.StokesError):
        capi.stokes_batch_solve([ctx], capi.STOKES_FP32, [up])
    ctx.close()
