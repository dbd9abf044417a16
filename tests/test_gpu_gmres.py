"""GPU parity of GMRES with a fixed preconditioner (option outer_solver = 2, Section 3.4) through
the C ABI against the oracle's gmres on the same problems: iteration counts (FP64 V-cycle) within
one of the oracle's, true residuals recomputed by the oracle's operator, solutions equal to the
oracle's FGMRES solution to the accuracy the tolerance allows; short restarts exercise the
cycle-end update x += P^-1 (V y) many times, in double-float and in native FP64 arithmetic."""
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


def gmres_options(capi, restart=50, outer_arith=1):
    o = capi.stokes_default_options()
    o.outer_solver = 2
    o.restart = restart
    o.outer_arith = outer_arith
    return o


@pytest.mark.parametrize("name,restart,arith", [("cube8", 50, 1), ("cube8", 7, 1), ("cube8", 7, 0),
                                                ("cube16", 50, 1), ("cube16", 10, 1)])
def test_gmres_solve(capi, name, restart, arith):
    p, m, G, ops, F = uniform_oracle(name)
    b = np.concatenate([F, np.zeros(m.n_p)])
    Pc = krylov.StokesPreconditioner(ops, G)
    _, its_o, _ = krylov.gmres(ops.apply_stokes, Pc.apply, b, rtol=1e-8, restart=restart, max_it=5000)
    xf, _, _ = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-10)
    xf = krylov.zero_mean_pressure(ops, xf)
    ctx = capi.stokes_setup_problem(p, options=gmres_options(capi, restart, arith))
    for prec in (capi.STOKES_FP64, capi.STOKES_FP32):
        for _ in range(2):      # the workspace is reused by the second solve
            up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
            info = capi.stokes_solve(ctx, prec, None, up, rtol=1e-8, max_it=5000)
            x = up.cpu().numpy()
            true = np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b)
            assert true <= 1e-8, (prec, true)
            assert abs(info.rel_residual_true - true) <= 1e-3 * true + 1e-14
            assert np.abs(x - xf).max() <= 1e-5 * np.abs(xf).max()
            if prec == capi.STOKES_FP64:
                assert abs(info.iterations - its_o) <= 1, (info.iterations, its_o)
    ctx.close()


def test_gmres_octree(capi):
    p = si.octree_workload("oct_s")
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    S = adaptive.AdaptiveStokes(octree.Octree(lv, p.coarsest_level), p)
    ctx = capi.stokes_setup_octree_problem(p, options=gmres_options(capi))
    up = torch.zeros(S.n_u + S.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=5000)
    b = np.concatenate([S.F, np.zeros(S.n_p)])
    assert np.linalg.norm(b - S.apply_stokes(up.cpu().numpy())) / np.linalg.norm(b) <= 1e-8
    ctx.close()


def test_gmres_batch(capi):
    """Batched solves run the same non-flexible cycles per problem."""
    p, m, G, ops, F = uniform_oracle("cube8")
    ctxs = [capi.stokes_setup_problem(p, options=gmres_options(capi)) for _ in range(2)]
    ups = [torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda") for _ in ctxs]
    capi.stokes_batch_solve(ctxs, capi.STOKES_FP32, ups)
    b = np.concatenate([F, np.zeros(m.n_p)])
    for up in ups:
        assert np.linalg.norm(b - ops.apply_stokes(up.cpu().numpy())) / np.linalg.norm(b) <= 1e-8
    for c in ctxs:
        c.close()


def test_gmres_diagonal_schur(capi):
    """S_hat = diag(M_p) (schur_degree = 0, the fixed approximation Section 3.4 names for GMRES):
    the Schur inverse equals diag(M_p)^-1 r to rounding, and GMRES with it converges with the
    oracle's iteration count."""
    p, m, G, ops, F = uniform_oracle("cube16")
    o = gmres_options(capi)
    o.schur_degree = 0
    ctx = capi.stokes_setup_problem(p, options=o)
    rng = np.random.default_rng(3)
    rp = rng.uniform(-1, 1, m.n_p)
    zp = torch.zeros(m.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_schur_inverse(ctx, torch.tensor(rp, device="cuda"), zp)
    Pc = krylov.StokesPreconditioner(ops, G, schur_degree=0)
    ref = Pc.schur_inverse(rp)
    assert np.abs(zp.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    b = np.concatenate([F, np.zeros(m.n_p)])
    _, its_o, _ = krylov.gmres(ops.apply_stokes, Pc.apply, b, rtol=1e-8, max_it=5000)
    up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    info = capi.stokes_solve(ctx, capi.STOKES_FP64, None, up, rtol=1e-8, max_it=5000)
    x = up.cpu().numpy()
    assert np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b) <= 1e-8
    assert abs(info.iterations - its_o) <= 1, (info.iterations, its_o)
    ctx.close()
