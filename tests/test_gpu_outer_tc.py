"""The outer Stokes operator on the tensor cores (outer_arith = 2: exact products of the integer
element table with fixed-point digit slices) through the C ABI, against the FP64 oracle at the
1e-12 bound of the outer operator: sinker problems with several 128-cell tiles and a ragged tail,
the viscosity over 24 decades with inputs over 12, and solves that reach the true residual."""
import numpy as np
import pytest

import sinker_inputs as si
from oracle import krylov, mesh, operators, sinker

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
TRUE_TOL = 1e-8 * (1.0 + 1e-3)


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06696_gb300 import build as B
    from paper_1907_06696_gb300 import capi as api
    B.build()
    api.load()
    return api


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tc_options(capi):
    o = capi.stokes_default_options()
    o.outer_arith = 2
    return o


@pytest.mark.parametrize("prob", [lambda: si.workload("cube8"), lambda: si.dr_problem(12, 3, 2, 1e3, 2001, "n12"),
                                  lambda: si.workload("cube16")], ids=["cube8", "n12", "cube16"])
def test_tensor_core_outer_operator_matches_oracle(capi, prob):
    p = prob()
    m = mesh.Mesh(p.n)
    mu = sinker.level_viscosities(m, p, p.n_levels)[-1]
    ops = operators.Operators(m, mu)
    ctx = capi.stokes_setup_problem(p, options=tc_options(capi))
    up = si.uniform(501, m.n_u + m.n_p)
    out = torch.empty(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, dev(up), out)
    capi.stokes_device_status(ctx)   # no wait ran out
    got, ref = host(out), ops.apply_stokes(up)
    assert rel(got, ref) <= F64_TOL, rel(got, ref)
    assert rel(got[:m.n_u], ref[:m.n_u]) <= F64_TOL and rel(got[m.n_u:], ref[m.n_u:]) <= F64_TOL
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.array_equal(got[:m.n_u][m.dirichlet], up[:m.n_u][m.dirichlet])   # identity rows
    ctx.close()


def test_tensor_core_outer_operator_wide_scale_spread(capi):
    """Cell viscosity log-uniform over 1e-12..1e12 and inputs of magnitude 1e-6..1e6 with random
    signs (cells where the scaled pressure exceeds the velocity by more than 2^8 take the
    double-float moments for B u): within 1e-12 of the oracle on the operator and each block."""
    n, L = 16, 3
    m = mesh.Mesh(n)
    mu_c = 10.0 ** (24.0 * si.uniform01(3310, m.n_cells) - 12.0)
    N = m.n_u + m.n_p
    up = si.uniform(3312, N) * 10.0 ** (12.0 * si.uniform01(3311, N) - 6.0)
    ctx = capi.stokes_setup(n, L, mu_q=np.repeat(mu_c, 27), options=tc_options(capi))
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, dev(up), out)
    capi.stokes_device_status(ctx)
    mu = np.empty(m.n_cells)
    mu_dev = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    capi.stokes_get_viscosity(ctx, -1, mu_dev)
    mu[:] = host(mu_dev)
    ref = operators.Operators(m, mu).apply_stokes(up)
    got = host(out)
    assert rel(got, ref) <= F64_TOL
    assert rel(got[:m.n_u], ref[:m.n_u]) <= F64_TOL and rel(got[m.n_u:], ref[m.n_u:]) <= F64_TOL
    ctx.close()


def test_tensor_core_outer_solve_matches_dense_direct(capi):
    p = si.workload("cube4")
    m = mesh.Mesh(p.n)
    mus = sinker.level_viscosities(m, p, p.n_levels)
    ops = operators.Operators(m, mus[-1])
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    xd = krylov.dense_stokes_solve(ops, F)
    ctx = capi.stokes_setup_problem(p, options=tc_options(capi))
    up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-12, max_it=500)
    assert np.abs(host(up) - xd).max() <= 1e-9 * np.abs(xd).max()
    ctx.close()


def test_tensor_core_outer_solve_iterations(capi):
    """cube16 (viscosity ratio 1e4) to 1e-8: the true residual met, iterations within 2 of the
    double-float outer operator's."""
    p = si.workload("cube16")
    m = mesh.Mesh(p.n)
    its = []
    for arith in (1, 2):
        o = capi.stokes_default_options()
        o.outer_arith = arith
        ctx = capi.stokes_setup_problem(p, options=o)
        up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
        info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=500)
        assert info.status == capi.STOKES_OK and info.rel_residual_true <= 1e-8
        its.append(info.iterations)
        if arith == 2:
            mus = sinker.level_viscosities(m, p, p.n_levels)
            ops = operators.Operators(m, mus[-1])
            F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
            b = np.concatenate([F, np.zeros(m.n_p)])
            x = host(up)
            assert np.linalg.norm(b - ops.apply_stokes(x)) <= TRUE_TOL * np.linalg.norm(b)
        ctx.close()
    assert abs(its[1] - its[0]) <= 2, its
