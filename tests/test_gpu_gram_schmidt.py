"""GPU parity of FGMRES with delayed re-orthogonalisation (option gram_schmidt = 1: two passes over
the double-float basis per iteration) through the C ABI: iteration counts within 2 of the oracle's
FGMRES (modified Gram-Schmidt), true residuals recomputed by the oracle's operator, solutions equal
to the three-pass variant's; restart lengths 7, 50 and 64 (every basis-size bound of the kernels,
restarts that reset the delayed record), and an adaptive mesh with an odd number of unknowns (the
last entry pair is half full)."""
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


def options(capi, gs, restart=50):
    o = capi.stokes_default_options()
    o.gram_schmidt = gs
    o.restart = restart
    return o


@pytest.mark.parametrize("name,restart", [("cube16", 50), ("cube16", 7), ("cube8", 64)])
def test_delayed_fgmres(capi, name, restart):
    p, m, G, ops, F = uniform_oracle(name)
    b = np.concatenate([F, np.zeros(m.n_p)])
    _, its_o, _ = krylov.fgmres(ops.apply_stokes, krylov.StokesPreconditioner(ops, G).apply, b, rtol=1e-8,
                                restart=restart, max_it=5000)
    sols = {}
    for gs in (1, 0):
        ctx = capi.stokes_setup_problem(p, options=options(capi, gs, restart))
        for prec in (capi.STOKES_FP64, capi.STOKES_FP32):
            for _ in range(2):
                up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
                info = capi.stokes_solve(ctx, prec, None, up, rtol=1e-8, max_it=5000)
                x = up.cpu().numpy()
                true = np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b)
                assert true <= 1e-8, (gs, prec, true)
                if prec == capi.STOKES_FP64:
                    assert abs(info.iterations - its_o) <= 2, (gs, info.iterations, its_o)
            sols[(gs, prec)] = x
        ctx.close()
    for prec in (capi.STOKES_FP64, capi.STOKES_FP32):
        a, c = sols[(1, prec)], sols[(0, prec)]
        assert np.abs(a - c).max() <= 1e-5 * np.abs(c).max()


def test_delayed_fgmres_octree_odd(capi):
    p = si.octree_workload("oct_xs")
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    S = adaptive.AdaptiveStokes(octree.Octree(lv, p.coarsest_level), p)
    assert (S.n_u + S.n_p) % 2 == 1
    b = np.concatenate([S.F, np.zeros(S.n_p)])
    _, its_o, _ = krylov.fgmres(S.apply_stokes, S.precondition, b, rtol=1e-8, max_it=2000)
    ctx = capi.stokes_setup_octree_problem(p, options=options(capi, 1))
    up = torch.zeros(S.n_u + S.n_p, dtype=torch.float64, device="cuda")
    info = capi.stokes_solve(ctx, capi.STOKES_FP64, None, up, rtol=1e-8, max_it=2000)
    assert np.linalg.norm(b - S.apply_stokes(up.cpu().numpy())) / np.linalg.norm(b) <= 1e-8
    assert abs(info.iterations - its_o) <= 2
    ctx.close()
