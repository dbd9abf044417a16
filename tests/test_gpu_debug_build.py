"""The STOKES_DEBUG build of the library: index-map checks on the octree path, through the C ABI.

In that build every octree kernel compares each entry it reads from a host-built index map
(cell -> nodes, node -> parent cell and position, leaf -> nodes or constraints, constraint ->
nodes, copy lists) with the size of what it indexes; a bad entry is skipped, never trapped on,
and the call that ran the kernel returns STOKES_EMESH naming the table and the entry.

* The checked build computes what the release build computes (FP64 active Stokes operator and
  level operators to 1e-12, a V-cycle to 1e-9, a solve to its true residual).
* The checks fire without any out-of-range access: stokes_debug_index_cut lowers the bound a
  check accepts below every valid entry of one table, so each of its reads counts as bad and is
  skipped. Each table gives EMESH from the call that reads it, and after the cut is lifted the
  same call succeeds and agrees with the release build again (the status words were cleared).
* The release build has no checks: stokes_debug_build() is 0 and the hook is EINVAL.
"""
import numpy as np
import pytest

import sinker_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TABLES = ["cell_nodes", "parent", "pos", "leaf_u", "ucon_node", "leaf_p", "pcon_node", "copy_active",
          "copy_level"]
CUT_ALL = 1 << 40   # above every table's size: all entries of the table read as bad


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06696_gb300 import build as B
    from paper_1907_06696_gb300 import capi
    B.build()
    B.build(debug=True)
    capi.load()
    return capi, capi.open_library(capi.DEBUG_LIB_PATH)


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def seeded(seed, n):
    return torch.tensor(si.uniform(seed, n), dtype=torch.float64, device="cuda")


def calls(capi, ctx):
    """The calls that read each table, as functions returning their output."""
    nu, npr, nl = ctx.n_u, ctx.n_p, ctx.n_levels
    up = seeded(4101, nu + npr)
    u = seeded(4102, nu)
    lev = nl - 1
    ul = seeded(4103, ctx.size(lev, 0))

    def stokes():
        out = torch.empty_like(up)
        capi.stokes_vmult(ctx, -1, capi.BLOCK_STOKES, capi.STOKES_FP64, up, out)
        return out

    def level_op():
        out = torch.empty_like(ul)
        capi.stokes_vmult(ctx, lev, capi.BLOCK_A, capi.STOKES_FP64, ul, out)
        return out

    def vcycle():
        out = torch.empty_like(u)
        capi.gmg_vcycle(ctx, capi.STOKES_FP64, u, out)
        return out

    reader = {"cell_nodes": level_op, "parent": vcycle, "pos": vcycle, "leaf_u": stokes, "ucon_node": stokes,
              "leaf_p": stokes, "pcon_node": stokes, "copy_active": vcycle, "copy_level": vcycle}
    return {"stokes": stokes, "level_op": level_op, "vcycle": vcycle}, reader


def test_release_build_has_no_checks(libs):
    capi, _ = libs
    lib = capi.load()
    assert lib.stokes_debug_build() == 0
    ctx = capi.stokes_setup_octree_problem(si.octree_workload("oct_s"))
    assert lib.stokes_debug_index_cut(ctx.handle, 0, 1) == capi.STOKES_EINVAL
    ctx.close()


def test_debug_build_matches_release(libs):
    capi, dbg = libs
    p = si.octree_workload("oct_s")
    ctx_r = capi.stokes_setup_octree_problem(p)
    fr, _ = calls(capi, ctx_r)
    ref = {k: f() for k, f in fr.items()}
    up_r = torch.zeros(ctx_r.n_u + ctx_r.n_p, dtype=torch.float64, device="cuda")
    info_r = capi.stokes_solve(ctx_r, capi.STOKES_FP32, None, up_r, rtol=1e-8, max_it=300)
    with capi.use_library(dbg):
        assert dbg.stokes_debug_build() == 1
        ctx_d = capi.stokes_setup_octree_problem(p)
        fd, _ = calls(capi, ctx_d)
        got = {k: f() for k, f in fd.items()}
        up_d = torch.zeros_like(up_r)
        info_d = capi.stokes_solve(ctx_d, capi.STOKES_FP32, None, up_d, rtol=1e-8, max_it=300)
        ctx_d.close()
    torch.cuda.synchronize()
    assert rel(got["stokes"], ref["stokes"]) <= 1e-12
    assert rel(got["level_op"], ref["level_op"]) <= 1e-12
    assert rel(got["vcycle"], ref["vcycle"]) <= 1e-9
    assert info_d.status == capi.STOKES_OK and info_r.status == capi.STOKES_OK
    assert info_d.rel_residual_true <= 1e-8 * 1.001
    assert abs(info_d.iterations - info_r.iterations) <= max(2, info_r.iterations // 10)
    ctx_r.close()


@pytest.mark.parametrize("table", range(len(TABLES)))
def test_bad_entries_are_reported_not_trapped(libs, table):
    capi, dbg = libs
    name = TABLES[table]
    p = si.octree_workload("oct_s")
    ctx_r = capi.stokes_setup_octree_problem(p)
    _, reader_r = calls(capi, ctx_r)
    ref = reader_r[name]()
    with capi.use_library(dbg):
        ctx = capi.stokes_setup_octree_problem(p)
        _, reader = calls(capi, ctx)
        assert dbg.stokes_debug_index_cut(ctx.handle, table, CUT_ALL) == capi.STOKES_OK
        with pytest.raises(capi.StokesError) as e:
            reader[name]()
        assert e.value.status == capi.STOKES_EMESH
        assert ("index map %s:" % name) in str(e.value)
        assert dbg.stokes_debug_index_cut(ctx.handle, table, 0) == capi.STOKES_OK
        again = reader[name]()          # status words were cleared with the report
        assert dbg.stokes_device_status(ctx.handle, None) == capi.STOKES_OK
        ctx.close()
    torch.cuda.synchronize()
    assert rel(again, ref) <= (1e-9 if reader_r[name].__name__ == "vcycle" else 1e-12)
    ctx_r.close()
