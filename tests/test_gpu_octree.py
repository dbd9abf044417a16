"""GPU parity of the adaptive (octree) path through the C ABI against the CPU oracle
(oracle/octree.py, oracle/adaptive.py) on the same seeded inputs.

* tables (integer work): leaves, active velocity nodes and pressure vertices, every level's
  nodes and boundary / refinement-edge flags, copy levels, hanging counts: bit-exact;
* FP64 active blocks with hanging-node constraints and FP64 level operators: relative 2-norm
  error <= 1e-12 (same sums, another order; outputs sum <= 8 cells x 81 terms, constrained
  nodes add <= 9 weighted terms);
* FP32 level operators: <= 2e-6 (inputs rounded to FP32, ~100 operations per output);
* V-cycle: FP64 <= 1e-9 (Lanczos estimates agree to rounding, so the Chebyshev coefficients
  differ at 1e-14 and the cycle propagates that); FP32 <= 1e-4 (FP32 rounding through the
  recursion of up to 5 levels);
* solves: status OK and the oracle's own operator confirms the GPU solution's true residual:
  <= 1e-8 (1 + 1e-3) with rtol 1e-8 (the library stops on its own native-FP64 true residual;
  the two evaluations of b - K x differ by ~1e-12 ||b||, ~1e-4 of that residual), iteration
  counts within 20% of the oracle's FGMRES.
"""
import functools

import numpy as np
import pytest

import sinker_inputs as si
from oracle import adaptive, krylov, octree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = ["oct_s", "oct_m"]


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
def oracle(name):
    p = si.octree_workload(name)
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    t = octree.Octree(lv, p.coarsest_level)
    return p, t, adaptive.AdaptiveStokes(t, p)


_CTX = {}


def context(capi, name):
    if name not in _CTX:
        p = si.octree_workload(name)
        _CTX[name] = capi.stokes_setup_octree_problem(p)
    return _CTX[name]


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name", CASES)
def test_tables(capi, name):
    p, t, S = oracle(name)
    ctx = context(capi, name)
    assert np.array_equal(capi.stokes_octree_table(ctx, 0), np.array(sorted(octree.cell_key(c) for c in t.leaves),
                                                                     dtype=np.uint64))
    assert np.array_equal(capi.stokes_octree_table(ctx, 1), t.u_keys.astype(np.uint64))
    assert np.array_equal(capi.stokes_octree_table(ctx, 2), t.p_keys.astype(np.uint64))
    nl = t.lmax - t.coarsest + 1
    assert ctx.size(-1, 4) == nl
    for li in range(nl):
        l = t.coarsest + li
        assert np.array_equal(capi.stokes_octree_table(ctx, 3, li), t.level_keys[l].astype(np.uint64))
        flags = t.level_boundary[l].astype(np.uint8) + 2 * t.level_edge[l].astype(np.uint8)
        assert np.array_equal(capi.stokes_octree_table(ctx, 4, li), flags)
        assert ctx.size(li, 2) == len(t.level_cells[l])
    assert np.array_equal(capi.stokes_octree_table(ctx, 5), (t.copy_level - t.coarsest).astype(np.int32))
    assert capi.stokes_octree_table(ctx, 6) == len(t.hanging_u)
    assert capi.stokes_octree_table(ctx, 7) == len(t.hanging_p)
    assert ctx.n_u == S.n_u and ctx.n_p == S.n_p


@pytest.mark.parametrize("name", CASES)
def test_active_blocks_fp64(capi, name):
    p, t, S = oracle(name)
    ctx = context(capi, name)
    x = si.uniform(3001, S.n_u)
    q = si.uniform(3002, S.n_p)
    cases = [(capi.BLOCK_A, x, S.apply_A(x), S.n_u), (capi.BLOCK_B, x, S.apply_B(x), S.n_p),
             (capi.BLOCK_BT, q, S.apply_BT(q), S.n_u), (capi.BLOCK_MP, q, S.apply_Mp(q), S.n_p)]
    for blk, src, ref, n_out in cases:
        out = torch.empty(n_out, dtype=torch.float64, device="cuda")
        capi.stokes_vmult(ctx, -1, blk, capi.STOKES_FP64, dev(src), out)
        assert rel(out.cpu().numpy(), ref) <= 1e-12, blk
    up = np.concatenate([x, q])
    out = torch.empty(S.n_u + S.n_p, dtype=torch.float64, device="cuda")
    capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, dev(up), out)
    assert rel(out.cpu().numpy(), S.apply_stokes(up)) <= 1e-12


@pytest.mark.parametrize("name", CASES)
def test_level_operators(capi, name):
    p, t, S = oracle(name)
    ctx = context(capi, name)
    for li in range(t.lmax - t.coarsest + 1):
        l = t.coarsest + li
        n = 3 * S.lev[l]["nn"]
        assert ctx.size(li, 0) == n
        x = si.uniform(3100 + li, n)
        ref = S.level_A(l, x)
        y64 = torch.empty(n, dtype=torch.float64, device="cuda")
        capi.stokes_vmult(ctx, li, capi.BLOCK_A, capi.STOKES_FP64, dev(x), y64)
        assert rel(y64.cpu().numpy(), ref) <= 1e-12, li
        y32 = torch.empty(n, dtype=torch.float32, device="cuda")
        capi.stokes_vmult(ctx, li, capi.BLOCK_A, capi.STOKES_FP32, dev(x, torch.float32), y32)
        assert rel(y32.double().cpu().numpy(), ref) <= 2e-6, li


@pytest.mark.parametrize("name", CASES)
def test_rhs_diagonal_lambda(capi, name):
    p, t, S = oracle(name)
    ctx = context(capi, name)
    F = torch.empty(S.n_u, dtype=torch.float64, device="cuda")
    capi.stokes_get_rhs(ctx, F)
    assert rel(F.cpu().numpy(), S.F) <= 1e-12
    for li in range(t.lmax - t.coarsest + 1):
        l = t.coarsest + li
        d = torch.empty(3 * S.lev[l]["nn"], dtype=torch.float64, device="cuda")
        capi.stokes_get_inv_diagonal(ctx, li, d)
        assert rel(d.cpu().numpy(), S.lev[l]["Dinv"]) <= 1e-12
        if li >= 1:
            lam = capi.stokes_get_lambda_max(ctx, li)
            assert lam == pytest.approx(S.lev[l]["lam_hi"] / 1.2, rel=1e-9)


@pytest.mark.parametrize("name", CASES)
def test_vcycle(capi, name):
    p, t, S = oracle(name)
    ctx = context(capi, name)
    b = si.uniform(3201, S.n_u)
    ref = S.vcycle(b)
    for prec, tol in ((capi.STOKES_FP64, 1e-9), (capi.STOKES_FP32, 1e-4)):
        for _ in range(2):      # level buffers are reused: a second cycle gives the same answer
            x = torch.empty(S.n_u, dtype=torch.float64, device="cuda")
            capi.gmg_vcycle(ctx, prec, dev(b), x)
            assert rel(x.cpu().numpy(), ref) <= tol, prec


@functools.lru_cache(maxsize=None)
def oracle_solve(name):
    p, t, S = oracle(name)
    b = np.concatenate([S.F, np.zeros(S.n_p)])
    _, its, _ = krylov.fgmres(S.apply_stokes, S.precondition, b, rtol=1e-8, restart=50, max_it=1000)
    return its


@pytest.mark.parametrize("name", ["oct_s"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve(capi, name, prec):
    p, t, S = oracle(name)
    ctx = context(capi, name)
    pr = capi.STOKES_FP64 if prec == "fp64" else capi.STOKES_FP32
    up = torch.zeros(S.n_u + S.n_p, dtype=torch.float64, device="cuda")
    info = capi.stokes_solve(ctx, pr, None, up, rtol=1e-8, max_it=2000)
    x = up.cpu().numpy()
    b = np.concatenate([S.F, np.zeros(S.n_p)])
    res = np.linalg.norm(b - S.apply_stokes(x)) / np.linalg.norm(b)
    assert info.status == capi.STOKES_OK
    assert res <= 1e-8 * 1.001
    assert info.rel_residual_true <= 1e-8
    its_ref = oracle_solve(name)
    assert abs(info.iterations - its_ref) <= max(3, 0.2 * its_ref), (info.iterations, its_ref)
    w = S.pressure_weights()
    assert abs(w @ x[S.n_u:]) <= 1e-10 * np.abs(w * x[S.n_u:]).sum()     # zero-mean pressure


def test_uniform_only_entry_points_refuse(capi):
    ctx = context(capi, "oct_s")
    lib = capi.load()
    assert lib.stokes_smooth(ctx.handle, 1, capi.STOKES_FP64, None, None, 1, None) == capi.STOKES_EMESH
    assert lib.stokes_coarse_solve(ctx.handle, capi.STOKES_FP64, None, None, None) == capi.STOKES_EMESH
