"""GPU parity: every step of the path, called through the C ABI, against the
CPU FP64 oracle on the same seeded inputs.

Tolerances (derived from the arithmetic):
* FP64 kernels: the oracle and the GPU evaluate the same sums in a different
  order (sum factorisation vs element matrices, atomics vs bincount). Each
  output is a sum of <= 8 cells x 81 terms of similar magnitude, so the
  rounding difference is a few hundred ulp at most: relative 2-norm error
  <= 1e-12 (the required FP64 bound) and max-norm error <= 1e-12 ||ref||_inf.
* FP32 operator / transfer kernels: inputs rounded to FP32 (2^-24 relative)
  and ~100 FP32 operations per output: relative error <= 2e-6.
* FP32 smoothing and V-cycle: the same per-kernel error, propagated through
  up to ~10 operator applications per level and the level recursion, with
  Chebyshev coefficients of magnitude <= 1/delta: relative error <= 2e-5.
"""
import functools

import numpy as np
import pytest

import sinker_inputs as si
from oracle import gmg, krylov, mesh, operators, sinker

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-6
F32_CYCLE_TOL = 2e-5
# Solves stop when the library's own native-FP64 true residual is <= rtol = 1e-8. The oracle
# recomputes b - K x in another summation order: the two K x agree to ~1e-13 ||b|| (the FP64
# operator bound), which is ~1e-5 of a residual of 1e-8 ||b||. So the oracle's relative true
# residual is <= 1e-8 (1 + 1e-3).
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


# sizes: several 128-cell tiles and a ragged tail (12^3 = 1728 cells = 13.5 tiles)
PROBLEMS = {
    "cube8": lambda: si.workload("cube8"),
    "n12": lambda: si.dr_problem(12, 3, 2, 1e3, 2001, "n12"),
    "cube16": lambda: si.workload("cube16"),
    "n24": lambda: si.dr_problem(24, 4, 4, 1e4, 2002, "n24"),
    # coarsest meshes of 5^3 and 6^3 cells (2,187 and 3,993 free DoFs in the dense FP64 solve)
    "n10c5": lambda: si.dr_problem(10, 2, 2, 1e3, 2003, "n10c5"),
    "n12c6": lambda: si.dr_problem(12, 2, 2, 1e3, 2004, "n12c6"),
}


@functools.lru_cache(maxsize=None)
def oracle_problem(name):
    p = PROBLEMS[name]()
    m = mesh.Mesh(p.n)
    mus = sinker.level_viscosities(m, p, p.n_levels)
    G = gmg.GMG(p.n, p.n_levels, mus)
    ops = G.levels[-1].ops
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    return p, m, mus, G, ops, F


_ctx_cache = {}


def gpu_ctx(capi, name, kernel=0):
    """Context of a named problem; kernel selects the V-cycle level operator
    (0 = cell-parallel with atomic adds, component-split on the FP32 levels up to 16^3, 1 =
    brick-tiled deterministic, 2 = brick-tiled with the FP32 cell products on the tensor cores, 3 =
    component-split on every FP32 level)."""
    key = (name, kernel)
    if key not in _ctx_cache:
        p = oracle_problem(name)[0]
        opt = capi.stokes_default_options()
        opt.vmult_kernel = kernel
        _ctx_cache[key] = capi.stokes_setup_problem(p, options=opt)
    return _ctx_cache[key]


def dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def assert_close(got, ref, tol):
    assert rel(got, ref) <= tol, rel(got, ref)
    assert np.abs(got - ref).max() <= tol * max(np.abs(ref).max(), 1e-300) * 10


# ----------------------------------------------------------------- set-up data
@pytest.mark.parametrize("name", ["cube8", "n12", "cube16"])
def test_viscosity_levels_and_rhs(capi, name):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name)
    for l in range(p.n_levels):
        out = torch.empty(len(mus[l]), dtype=torch.float64, device="cuda")
        capi.stokes_get_viscosity(ctx, l, out)
        assert_close(host(out), mus[l], 1e-13)
    Fd = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    capi.stokes_get_rhs(ctx, Fd)
    assert_close(host(Fd), F, 1e-12)


@pytest.mark.parametrize("name", ["cube8", "n12"])
def test_inverse_diagonal_and_lambda(capi, name):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name)
    for l, lev in enumerate(G.levels):
        out = torch.empty(lev.mesh.n_u, dtype=torch.float64, device="cuda")
        capi.stokes_get_inv_diagonal(ctx, l, out)
        assert_close(host(out), lev.Dinv, 1e-13)
        if l >= 1:
            lam = capi.stokes_get_lambda_max(ctx, l)
            assert abs(lam - lev.lam_max) <= 1e-10 * lev.lam_max, (l, lam, lev.lam_max)


# ----------------------------------------------------------------- operators
@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["cube8", "n12", "cube16", "n24"])
def test_vmult_A_all_levels(capi, name, kernel):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name, kernel)
    for l, lev in enumerate(G.levels):
        x = si.uniform(300 + l, lev.mesh.n_u)          # includes constrained entries
        ref = lev.ops.apply_A(x)
        for prec, dt, tol in ((capi.STOKES_FP64, torch.float64, F64_TOL), (capi.STOKES_FP32, torch.float32, F32_TOL)):
            src = dev(x, dt)
            dst = torch.full_like(src, float("nan"))
            capi.stokes_vmult(ctx, l, capi.BLOCK_A, prec, src, dst)
            got = host(dst)
            assert_close(got, ref, tol)
            assert np.array_equal(got[lev.mesh.dirichlet], np.asarray(src.cpu().double())[lev.mesh.dirichlet])


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("name", ["cube8", "n12"])
def test_pressure_blocks_and_stokes_operator(capi, name, arith):
    """Both arithmetics of the outer blocks: native FP64 and double-float."""
    p, m, mus, G, ops, F = oracle_problem(name)
    opt = capi.stokes_default_options()
    opt.outer_arith = arith
    ctx = capi.stokes_setup_problem(p, options=opt)
    u = si.uniform(401, m.n_u)
    q = si.uniform(402, m.n_p)
    out_p = torch.empty(m.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_vmult(ctx, -1, capi.BLOCK_B, capi.STOKES_FP64, dev(u), out_p)
    assert_close(host(out_p), ops.apply_B(u), F64_TOL)
    out_u = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
    capi.stokes_vmult(ctx, -1, capi.BLOCK_BT, capi.STOKES_FP64, dev(q), out_u)
    assert_close(host(out_u), ops.apply_BT(q), F64_TOL)
    capi.stokes_vmult(ctx, -1, capi.BLOCK_MP, capi.STOKES_FP64, dev(q), out_p)
    assert_close(host(out_p), ops.apply_Mp(q), F64_TOL)
    up = np.concatenate([u, q])
    out = torch.empty(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, dev(up), out)
    assert_close(host(out), ops.apply_stokes(up), F64_TOL)
    ctx.close()


# ----------------------------------------------------------------- multigrid pieces
@pytest.mark.parametrize("name", ["cube8", "n12"])
def test_transfers(capi, name):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name)
    for l in range(1, p.n_levels):
        fine, coarse = G.levels[l], G.levels[l - 1]
        xc = si.uniform(500 + l, coarse.mesh.n_u)
        xf = si.uniform(600 + l, fine.mesh.n_u) * fine.free
        ref_p = (G.P[l] @ xc) * fine.free
        ref_r = (G.P[l].T @ xf) * coarse.free
        for prec, dt, tol in ((capi.STOKES_FP64, torch.float64, 1e-14), (capi.STOKES_FP32, torch.float32, F32_TOL)):
            out = torch.empty(fine.mesh.n_u, dtype=dt, device="cuda")
            capi.stokes_prolongate(ctx, l, prec, dev(xc, dt), out, add=False)
            assert_close(host(out), ref_p, tol)
            base = dev(xf, dt)
            capi.stokes_prolongate(ctx, l, prec, dev(xc, dt), base, add=True)
            assert_close(host(base), xf + ref_p, tol)
            outc = torch.empty(coarse.mesh.n_u, dtype=dt, device="cuda")
            capi.stokes_restrict(ctx, l, prec, dev(xf, dt), outc)
            assert_close(host(outc), ref_r, tol)


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["cube8", "n12"])
def test_chebyshev_smoother(capi, name, kernel):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name, kernel)
    for l in range(1, p.n_levels):
        lev = G.levels[l]
        b = si.uniform(700 + l, lev.mesh.n_u) * lev.free
        x0 = si.uniform(800 + l, lev.mesh.n_u) * lev.free
        for zero in (True, False):
            ref = G.smooth(l, b, None if zero else x0, zero)
            for prec, dt, tol in ((capi.STOKES_FP64, torch.float64, 1e-11),
                                  (capi.STOKES_FP32, torch.float32, F32_CYCLE_TOL)):
                x = dev(x0, dt)
                capi.stokes_smooth(ctx, l, prec, dev(b, dt), x, zero)
                assert_close(host(x), ref, tol)


@pytest.mark.parametrize("name", ["cube8", "n12", "n10c5", "n12c6"])
def test_coarse_solve(capi, name):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name)
    c = G.levels[0]
    b = si.uniform(900, c.mesh.n_u) * c.free
    ref = G.coarse_solve(b)
    for prec, dt, tol in ((capi.STOKES_FP64, torch.float64, 1e-12), (capi.STOKES_FP32, torch.float32, F32_TOL)):
        x = torch.full((c.mesh.n_u,), float("nan"), dtype=dt, device="cuda")
        capi.stokes_coarse_solve(ctx, prec, dev(b, dt), x)
        assert_close(host(x), ref, tol)


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["cube8", "n12", "cube16", "n24", "n10c5", "n12c6"])
def test_vcycle(capi, name, kernel):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name, kernel)
    rhs = si.uniform(1000, m.n_u)
    ref = G.vcycle(rhs)
    for prec, dt, tol in ((capi.STOKES_FP64, torch.float64, 1e-10), (capi.STOKES_FP32, torch.float32, F32_CYCLE_TOL)):
        x = torch.full((m.n_u,), float("nan"), dtype=dt, device="cuda")
        capi.gmg_vcycle(ctx, prec, dev(rhs, dt), x)
        assert_close(host(x), ref, tol)


# ----------------------------------------------------------------- outer solve pieces
@pytest.mark.parametrize("name", ["cube8", "n12"])
def test_schur_and_block_preconditioner(capi, name):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name)
    Pc = krylov.StokesPreconditioner(ops, G)
    rp = si.uniform(1100, m.n_p)
    zp = torch.empty(m.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_schur_inverse(ctx, dev(rp), zp)
    assert_close(host(zp), Pc.schur_inverse(rp), 1e-12)
    r = si.uniform(1101, m.n_u + m.n_p)
    ref = Pc.apply(r)
    z = torch.empty(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_precondition(ctx, capi.STOKES_FP64, dev(r), z)
    assert_close(host(z), ref, 1e-10)
    capi.stokes_precondition(ctx, capi.STOKES_FP32, dev(r), z)
    assert_close(host(z), ref, F32_CYCLE_TOL)


@pytest.mark.parametrize("kernel", [0, 2, 3])
@pytest.mark.parametrize("name", ["cube8", "n12", "n10c5"])
def test_solve_fp64_and_fp32_vcycle(capi, name, kernel):
    p, m, mus, G, ops, F = oracle_problem(name)
    ctx = gpu_ctx(capi, name, kernel)
    b = np.concatenate([F, np.zeros(m.n_p)])
    Pc = krylov.StokesPreconditioner(ops, G)
    xo, its_o, _ = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-8)
    xo = krylov.zero_mean_pressure(ops, xo)
    its = {}
    for prec in (capi.STOKES_FP64, capi.STOKES_FP32):
        up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
        info = capi.stokes_solve(ctx, prec, None, up, rtol=1e-8, max_it=500)
        x = host(up)
        # property: the true FP64 residual, recomputed by the oracle's operator
        true = np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b)
        assert info.status == capi.STOKES_OK
        assert true <= TRUE_TOL, (prec, true)
        assert abs(info.rel_residual_true - true) <= 1e-3 * true + 1e-14
        assert np.abs(x - xo).max() <= 1e-5 * np.abs(xo).max()
        its[prec] = info.iterations
    assert abs(its[capi.STOKES_FP64] - its_o) <= 2, (its, its_o)
    assert its[capi.STOKES_FP32] <= 1.2 * its[capi.STOKES_FP64] + 1


@pytest.mark.parametrize("arith", [0, 1])
def test_solve_matches_dense_direct(capi, arith):
    p = si.workload("cube4")
    m = mesh.Mesh(p.n)
    mus = sinker.level_viscosities(m, p, p.n_levels)
    ops = operators.Operators(m, mus[-1])
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    xd = krylov.dense_stokes_solve(ops, F)
    opt = capi.stokes_default_options()
    opt.outer_arith = arith
    ctx = capi.stokes_setup_problem(p, options=opt)
    for prec in (capi.STOKES_FP64, capi.STOKES_FP32):
        up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
        capi.stokes_solve(ctx, prec, None, up, rtol=1e-12, max_it=500)
        assert np.abs(host(up) - xd).max() <= 1e-9 * np.abs(xd).max()
    # host-buffer entry point
    out = np.zeros(m.n_u + m.n_p)
    info = capi.stokes_solve_host(ctx, capi.STOKES_FP32, None, out, rtol=1e-12, max_it=500)
    assert np.abs(out - xd).max() <= 1e-9 * np.abs(xd).max() and info.iterations > 0
    ctx.close()


@pytest.mark.parametrize("solver", [0, 1, 2, 3])
def test_status_follows_true_residual_at_max_it(capi, solver):
    """Every outer solver's status is OK exactly when its true residual meets rtol: with max_it
    equal to the count a solve needed (the recurrence converges on the last allowed iteration),
    one fewer, and 1. (solver: 0 FGMRES, 1 IDR(2), 2 GMRES, 3 MINRES with P_D.)"""
    p = oracle_problem("cube8")[0]
    opt = capi.stokes_default_options()
    opt.outer_solver = solver
    if solver == 3:
        opt.precond_kind = 1
    ctx = capi.stokes_setup_problem(p, options=opt)
    N = ctx.n_u + ctx.n_p
    up = torch.zeros(N, dtype=torch.float64, device="cuda")
    k = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=2000).iterations
    for max_it in (k, k - 1, 1):
        up.zero_()
        info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=max_it, check=False)
        assert info.iterations <= max_it
        assert (info.status == capi.STOKES_OK) == (info.rel_residual_true <= 1e-8), (max_it, info.status,
                                                                                    info.rel_residual_true)
        if max_it == 1:
            assert info.status == capi.STOKES_NOT_CONVERGED
    ctx.close()


def test_allocation_failure_frees_what_it_took(capi):
    """Device allocations that fail (the stokes_debug_alloc_limit hook) give ENOMEM from set-up and
    from the first solve (which allocates the Krylov basis); the failed set-up frees what it had
    taken, and the same calls succeed once the limit is lifted."""
    p = oracle_problem("cube8")[0]
    lib = capi.load()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for limit in (0, 1 << 12, 1 << 20):
            assert lib.stokes_debug_alloc_limit(limit) == capi.STOKES_OK
            with pytest.raises(capi.StokesError) as e:
                capi.stokes_setup_problem(p)
            assert e.value.status == capi.STOKES_ENOMEM
        lib.stokes_debug_alloc_limit(-1)
        ctx = capi.stokes_setup_problem(p)
        lib.stokes_debug_alloc_limit(0)
        up = torch.zeros(ctx.n_u + ctx.n_p, dtype=torch.float64, device="cuda")
        with pytest.raises(capi.StokesError) as e:
            capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=200)
        assert e.value.status == capi.STOKES_ENOMEM
    finally:
        lib.stokes_debug_alloc_limit(-1)
    info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=200)
    assert info.status == capi.STOKES_OK
    ctx.close()
    del up
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)


def test_double_float_outer_operator_wide_scale_spread(capi):
    """The double-float outer operator (float exponent range, ~47-bit significands, the unchecked
    addition of its hi/lo pairs) against the native FP64 kernel at h = 1/128 with the cell viscosity
    log-uniform over 1e-12..1e12 and inputs log-uniform over 1e-6..1e6 in magnitude: relative
    2-norm difference <= 1e-12 on [A B^T; B 0] and on each block."""
    n, L = 128, 6
    cells = n ** 3
    mu_c = 10.0 ** (24.0 * si.uniform01(3300, cells) - 12.0)
    mu_q = np.repeat(mu_c, 27)
    outs = []
    N = si.n_velocity(n) + si.n_pressure(n)
    mag = 10.0 ** (12.0 * si.uniform01(3301, N) - 6.0)
    up = dev(si.uniform(3302, N) * mag)
    for arith in (1, 0):
        opt = capi.stokes_default_options()
        opt.outer_arith = arith
        ctx = capi.stokes_setup(n, L, mu_q=mu_q, options=opt)
        out = torch.empty_like(up)
        capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, up, out)
        outs.append(host(out))
        ctx.close()
        del out
        torch.cuda.empty_cache()
    got, ref = outs
    n_u = si.n_velocity(n)
    assert rel(got, ref) <= F64_TOL, rel(got, ref)
    assert rel(got[:n_u], ref[:n_u]) <= F64_TOL and rel(got[n_u:], ref[n_u:]) <= F64_TOL
    assert np.all(np.isfinite(got))


# ----------------------------------------------------------------- edge cases
def test_tensor_core_operator_wait_timeout(capi):
    """A bounded device wait that runs out: with wait_limit_s = 0 the tensor-core operator gives up
    on its MMAs at once, records STOKES_TIMEOUT in the context's status word (read and cleared by
    stokes_device_status, and by stokes_solve) and leaves; the context and the device stay usable
    and the next call with a normal limit is correct."""
    p, m, mus, G, ops, F = oracle_problem("n12")
    opt = capi.stokes_default_options()
    opt.vmult_kernel = 2
    opt.wait_limit_s = 0.0
    ctx = capi.stokes_setup_problem(p, options=opt)
    x = si.uniform(310, m.n_u)
    src = dev(x, torch.float32)
    dst = torch.empty_like(src)
    capi.stokes_vmult(ctx, -1, capi.BLOCK_A, capi.STOKES_FP32, src, dst)
    with pytest.raises(capi.StokesError) as e:
        capi.stokes_device_status(ctx)
    assert e.value.status == capi.STOKES_TIMEOUT
    capi.stokes_device_status(ctx)          # cleared
    up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=20, check=False)
    assert info.status == capi.STOKES_TIMEOUT
    ctx.close()
    ok = gpu_ctx(capi, "n12", 2)
    capi.stokes_vmult(ok, -1, capi.BLOCK_A, capi.STOKES_FP32, src, dst)
    capi.stokes_device_status(ok)
    assert_close(host(dst), G.levels[-1].ops.apply_A(x), F32_TOL)


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_kernel_launches(capi, prec, kernel):
    """The captured V-cycle graph runs the same kernels in the same order, over two replays with
    different right-hand sides: bitwise equal output with the deterministic brick operator (1); with
    the atomic operators (0, 3; 2, whose shared and global atomic adds vary their order from run to
    run) equal to rounding."""
    p = oracle_problem("n12")[0]
    outs = []
    for graphs in (0, 1):
        opt = capi.stokes_default_options()
        opt.graphs = graphs
        opt.vmult_kernel = kernel
        ctx = capi.stokes_setup_problem(p, options=opt)
        dt = torch.float64 if prec == 0 else torch.float32
        res = []
        for seed in (5000, 5001):
            rhs = dev(si.uniform(seed, ctx.n_u), dt)
            x = torch.empty_like(rhs)
            capi.gmg_vcycle(ctx, prec, rhs, x)
            res.append(host(x))
        outs.append(res)
        ctx.close()
    for a, b in zip(outs[0], outs[1]):
        if kernel == 1:
            assert np.array_equal(a, b)
        else:
            assert rel(a, b) <= (1e-13 if prec == 0 else 1e-6)


@pytest.mark.parametrize("kernel", [0, 3])
def test_vmult_into_unaligned_views(capi, kernel):
    """The FP32 cell kernels add a row's node pairs with 8-byte atomics when the output is 8-byte
    aligned; a caller's output view at an odd element offset takes the single-add scatter. Both
    give the same product (to the rounding of the atomic sums' order) on every level."""
    p, m, mus, G, ops, F = oracle_problem("n12")
    ctx = gpu_ctx(capi, "n12", kernel)
    for l in range(p.n_levels):
        nu = ctx.size(l, 0)
        x = dev(si.uniform(5400 + l, nu), torch.float32)
        y = torch.empty(nu, dtype=torch.float32, device="cuda")
        buf = torch.empty(nu + 1, dtype=torch.float32, device="cuda")
        capi.stokes_vmult(ctx, l, capi.BLOCK_A, capi.STOKES_FP32, x, y)
        capi.stokes_vmult(ctx, l, capi.BLOCK_A, capi.STOKES_FP32, x, buf[1:])
        assert rel(host(buf[1:]), host(y)) <= 1e-6


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kernel", [0, 3])
def test_fused_smoother_matches_separate_passes(capi, prec, kernel):
    """The smoother with each Chebyshev step carried by the next product (fused_smoother 1)
    computes what the separate vector passes (0, the default) compute: the same per-node arithmetic,
    so smoothing steps of every level (zero and non-zero initial guess) and whole V-cycles agree to
    the rounding of the atomic sums' order."""
    p, m, mus, G, ops, F = oracle_problem("n12")
    dt = torch.float64 if prec == 0 else torch.float32
    out = []
    for fused in (0, 1):
        opt = capi.stokes_default_options()
        opt.vmult_kernel = kernel
        opt.fused_smoother = fused
        ctx = capi.stokes_setup_problem(p, options=opt)
        res = []
        for l in range(1, p.n_levels):
            lev = G.levels[l]
            b = dev(si.uniform(5100 + l, lev.mesh.n_u) * lev.free, dt)
            for zero in (True, False):
                x = dev(si.uniform(5200 + l, lev.mesh.n_u) * lev.free, dt)
                capi.stokes_smooth(ctx, l, prec, b, x, zero)
                res.append(host(x))
        rhs = dev(si.uniform(5300, ctx.n_u), dt)
        x = torch.empty_like(rhs)
        capi.gmg_vcycle(ctx, prec, rhs, x)
        res.append(host(x))
        out.append(res)
        ctx.close()
    for a, b in zip(out[0], out[1]):
        assert rel(b, a) <= (1e-13 if prec == 0 else 1e-6)


def test_batch_solve_matches_individual_solves(capi):
    """stokes_batch_solve over problems of different sizes and level counts runs the same FGMRES as
    stokes_solve: iteration counts within 1 (the batched V-cycle and the single-problem graph sum
    their FP32 atomic adds in different orders), the same solutions to that rounding, and each true
    FP64 residual (recomputed by the oracle) <= 1e-8 (to the oracle's rounding)."""
    probs = [si.dr_problem(8, 4, 1, 1e2, 6001), si.dr_problem(12, 3, 3, 1e4, 6002),
             si.dr_problem(16, 5, 2, 1e3, 6003), si.dr_problem(8, 2, 4, 1e5, 6004)]
    ctxs = [capi.stokes_setup_problem(p) for p in probs]
    ups = [torch.zeros(c.n_u + c.n_p, dtype=torch.float64, device="cuda") for c in ctxs]
    infos = capi.stokes_batch_solve(ctxs, capi.STOKES_FP32, ups, rtol=1e-8, max_it=500)
    for p, ctx, up, info in zip(probs, ctxs, ups, infos):
        ref = torch.zeros_like(up)
        ri = capi.stokes_solve(ctx, capi.STOKES_FP32, None, ref, rtol=1e-8, max_it=500)
        assert abs(info.iterations - ri.iterations) <= 1 and info.status == 0
        x, xr = host(up), host(ref)
        assert np.abs(x - xr).max() <= 1e-6 * np.abs(xr).max()
        m = mesh.Mesh(p.n)
        ops = operators.Operators(m, sinker.level_viscosities(m, p, p.n_levels)[-1])
        F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
        b = np.concatenate([F, np.zeros(m.n_p)])
        assert np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b) <= TRUE_TOL
    for c in ctxs:
        c.close()


# nine problems: rounds with at least eight at their preconditioner run the batched kernel, the
# tail of the solve (fewer problems left) the per-problem graphs
BATCH_PROBLEMS = [(8, 4, 1, 1e2, 6101), (12, 3, 3, 1e4, 6102), (16, 5, 2, 1e3, 6103), (8, 2, 4, 1e5, 6104),
                  (10, 2, 2, 1e3, 6105), (20, 3, 5, 1e6, 6106), (24, 4, 3, 1e4, 6107), (16, 3, 2, 1e2, 6108),
                  (12, 2, 1, 1e3, 6109)]


def batch_contexts(capi, batch_vcycle, wait_limit_s=1.0):
    probs = [si.dr_problem(*a) for a in BATCH_PROBLEMS]
    ctxs = []
    for p in probs:
        opt = capi.stokes_default_options()
        opt.batch_vcycle = batch_vcycle
        opt.wait_limit_s = wait_limit_s
        ctxs.append(capi.stokes_setup_problem(p, options=opt))
    return probs, ctxs


def test_batched_vcycle_kernel_matches_per_problem_graphs(capi):
    """The batch solved with one persistent V-cycle launch per round (batch_vcycle 1: work queue of
    (problem, tile) items over problems of 8^3..24^3 cells with 2 to 5 levels and coarsest meshes of
    1 to 6 cells, converged problems left out; rounds with fewer than eight problems at their
    preconditioner replay the per-problem graphs) runs the same FGMRES as the per-problem captured
    graphs throughout (batch_vcycle 0): iteration counts within 1 (the atomic adds of both sum in varying
    order) and solutions equal to the FP32 V-cycle's rounding; every true residual, recomputed by
    the oracle from its own viscosity, <= 1e-8."""
    res = {}
    for mode in (1, 0):
        probs, ctxs = batch_contexts(capi, mode)
        ups = [torch.zeros(c.n_u + c.n_p, dtype=torch.float64, device="cuda") for c in ctxs]
        infos = capi.stokes_batch_solve(ctxs, capi.STOKES_FP32, ups, rtol=1e-8, max_it=1000)
        res[mode] = ([i.iterations for i in infos], [host(u) for u in ups], [i.status for i in infos])
        for c in ctxs:
            c.close()
    for i, p in enumerate(probs):
        assert res[1][2][i] == capi.STOKES_OK
        assert abs(res[1][0][i] - res[0][0][i]) <= 1, (i, res[1][0][i], res[0][0][i])
        x, xr = res[1][1][i], res[0][1][i]
        assert np.abs(x - xr).max() <= 1e-6 * np.abs(xr).max()
        m = mesh.Mesh(p.n)
        ops = operators.Operators(m, sinker.level_viscosities(m, p, p.n_levels)[-1])
        F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
        b = np.concatenate([F, np.zeros(m.n_p)])
        assert np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b) <= TRUE_TOL


def test_batched_vcycle_kernel_barrier_timeout(capi):
    """The grid barriers of the batched V-cycle are bounded: with wait_limit_s = 0 every barrier
    gives up at once, the kernel leaves, and the batch solve returns STOKES_TIMEOUT (per problem
    too); the device stays usable and the same problems then solve normally."""
    probs, ctxs = batch_contexts(capi, 1, wait_limit_s=0.0)
    ups = [torch.zeros(c.n_u + c.n_p, dtype=torch.float64, device="cuda") for c in ctxs]
    infos = capi.stokes_batch_solve(ctxs, capi.STOKES_FP32, ups, rtol=1e-8, max_it=3, check=False)
    assert all(i.status == capi.STOKES_TIMEOUT for i in infos)
    with pytest.raises(capi.StokesError) as e:
        capi.stokes_batch_solve(ctxs, capi.STOKES_FP32, ups, rtol=1e-8, max_it=3)
    assert e.value.status == capi.STOKES_TIMEOUT
    for c in ctxs:
        c.close()
    probs, ctxs = batch_contexts(capi, 1)
    for u in ups:
        u.zero_()
    ups = [torch.zeros(c.n_u + c.n_p, dtype=torch.float64, device="cuda") for c in ctxs]
    infos = capi.stokes_batch_solve(ctxs, capi.STOKES_FP32, ups, rtol=1e-8, max_it=1000)
    assert all(i.status == capi.STOKES_OK and i.rel_residual_true <= 1e-8 for i in infos)
    for c in ctxs:
        c.close()


def test_autotune_keeps_the_solve_correct(capi):
    p, m, mus, G, ops, F = oracle_problem("cube16")
    ctx = capi.stokes_setup_problem(p)
    block, degree = capi.stokes_autotune(ctx, 3)
    assert block in (64, 128, 256) and 3 <= degree <= 6
    up = torch.zeros(m.n_u + m.n_p, dtype=torch.float64, device="cuda")
    info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=1000)
    b = np.concatenate([F, np.zeros(m.n_p)])
    assert np.linalg.norm(b - ops.apply_stokes(host(up))) / np.linalg.norm(b) <= TRUE_TOL
    assert info.iterations > 0 and info.status == capi.STOKES_OK
    ctx.close()


def test_single_level_and_two_level_meshes(capi):
    for n, L in ((1, 1), (2, 2), (3, 1), (4, 1)):
        p = si.dr_problem(n, L, 1, 1e2, 3000 + n)
        m = mesh.Mesh(n)
        mus = sinker.level_viscosities(m, p, L)
        G = gmg.GMG(n, L, mus)
        ctx = capi.stokes_setup_problem(p)
        rhs = si.uniform(3100 + n, m.n_u)
        x = torch.empty(m.n_u, dtype=torch.float64, device="cuda")
        capi.gmg_vcycle(ctx, capi.STOKES_FP64, dev(rhs), x)
        assert_close(host(x), G.vcycle(rhs), 1e-10)
        ctx.close()


def test_quadrature_point_viscosity_input(capi):
    n, L = 8, 4
    m = mesh.Mesh(n)
    mu_q = 1.0 + 9.0 * si.uniform01(3200, m.n_cells * 27).reshape(m.n_cells, 27)
    ctx = capi.stokes_setup(n, L, mu_q=mu_q)
    out = torch.empty(m.n_cells, dtype=torch.float64, device="cuda")
    capi.stokes_get_viscosity(ctx, -1, out)
    assert_close(host(out), sinker.harmonic_cell_average(mu_q), 1e-14)
    ctx.close()


def test_invalid_arguments_on_device(capi):
    ctx = gpu_ctx(capi, "cube8")
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.StokesError):
        capi.stokes_vmult(ctx, 7, capi.BLOCK_A, capi.STOKES_FP64, x, x)
    with pytest.raises(capi.StokesError):
        capi.stokes_vmult(ctx, 0, capi.BLOCK_B, capi.STOKES_FP64, x, x)      # B only on the finest level
    with pytest.raises(capi.StokesError):
        capi.stokes_vmult(ctx, -1, capi.BLOCK_BT, capi.STOKES_FP32, x, x)    # FP64 only
    with pytest.raises(capi.StokesError):
        capi.stokes_smooth(ctx, 0, capi.STOKES_FP64, x, x, True)


# ----------------------------------------------------------------- full size, sampled
@functools.lru_cache(maxsize=2)
def oracle_cell_viscosity(name):
    """The oracle's finest-level cell viscosity of a full-size workload (Sections 2.3, 3.2): mu at
    the 27 Gauss points of every cell, quadrature-weighted harmonic mean per cell, computed slab by
    slab (the same formula as sinker.level_viscosities, without the global cell tables)."""
    from oracle import fe
    p = si.workload(name)
    n = p.n
    pts, _ = fe.quadrature_3d()
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    out = np.empty(n ** 3)
    for ck in range(n):
        ijk = np.stack([ci.ravel(), cj.ravel(), np.full(n * n, ck)], 1)
        q = (ijk[:, None, :] + pts[None]) / n
        out[ck * n * n:(ck + 1) * n * n] = sinker.harmonic_cell_average(sinker.viscosity(q, p))
    return out


def check_gpu_viscosity(capi, ctx, name):
    """Every cell of the GPU's finest-level viscosity against the oracle's."""
    p = si.workload(name)
    mu = torch.empty(p.n ** 3, dtype=torch.float64, device="cuda")
    capi.stokes_get_viscosity(ctx, -1, mu)
    assert_close(host(mu), oracle_cell_viscosity(name), 1e-13)
    del mu


@pytest.mark.parametrize("name", ["cube64", "cube128"])
def test_full_size_vmult_sampled_rows(capi, name):
    """The benchmark workloads at full size: the GPU viscosity on every cell against the oracle's,
    then rows sampled uniformly plus rows next to the boundary and at tile corners, recomputed one
    by one by the oracle from its own viscosity."""
    p = si.workload(name)
    n = p.n
    M = 2 * n + 1
    n_u = 3 * M ** 3
    ctx = gpu_ctx_full(capi, p)
    check_gpu_viscosity(capi, ctx, name)
    mu_o = oracle_cell_viscosity(name)
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([rng.integers(0, n_u, 400),
                                     [M * M + M + 1, 2 * M ** 3 - M * M - M - 2, M ** 3 // 2, n_u - 1, 0]]))
    x = si.uniform(4000, n_u)
    ref = operators.apply_A_rows(n, mu_o, x, rows)
    for prec, dt, tol in ((capi.STOKES_FP64, torch.float64, F64_TOL), (capi.STOKES_FP32, torch.float32, F32_TOL)):
        src = dev(x, dt)
        dst = torch.empty_like(src)
        capi.stokes_vmult(ctx, -1, capi.BLOCK_A, prec, src, dst)
        got = host(dst)[rows]
        assert np.abs(got - ref).max() <= tol * 10 * np.abs(ref).max(), (prec, np.abs(got - ref).max())
        del src, dst
    # the tensor-core FP32 operator (vmult_kernel 2), launched as the benchmark launches it
    opt = capi.stokes_default_options()
    opt.vmult_kernel = 2
    tctx = capi.stokes_setup_problem(p, options=opt)
    src = dev(x, torch.float32)
    dst = torch.empty_like(src)
    capi.stokes_vmult(tctx, -1, capi.BLOCK_A, capi.STOKES_FP32, src, dst)
    capi.stokes_device_status(tctx)
    got = host(dst)[rows]
    assert np.abs(got - ref).max() <= F32_TOL * 10 * np.abs(ref).max(), np.abs(got - ref).max()
    tctx.close()


_full_cache = {}


def gpu_ctx_full(capi, p):
    if p.name not in _full_cache:
        _full_cache.clear()
        _full_cache[p.name] = capi.stokes_setup_problem(p)
    return _full_cache[p.name]


@pytest.mark.parametrize("name", ["cube64", "cube128"])
def test_full_size_solve_residual(capi, name):
    """64^3 (8 sinkers, DR 1e4) and 128^3 (16 sinkers, DR 1e6): the FP32 V-cycle inside FP64 FGMRES
    reaches a true FP64 residual <= 1e-8, recomputed by the oracle's element-by-element operator
    from the oracle's own viscosity and right-hand side."""
    p = si.workload(name)
    ctx = gpu_ctx_full(capi, p)
    n_u, n_p = ctx.n_u, ctx.n_p
    up = torch.zeros(n_u + n_p, dtype=torch.float64, device="cuda")
    info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=2000)
    x = host(up)
    del up
    m = mesh.Mesh(p.n)
    ops = operators.Operators(m, oracle_cell_viscosity(name))
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    b = np.concatenate([F, np.zeros(m.n_p)])
    true = np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b)
    assert info.status == capi.STOKES_OK
    assert true <= TRUE_TOL, true
    assert abs(info.rel_residual_true - true) <= 1e-3 * true
    assert info.iterations < 2000
