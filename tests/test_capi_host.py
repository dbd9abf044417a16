"""Host-side checks of the C ABI: the library builds, loads and exports every
function that include/stokes.h declares; argument validation that happens
before any device work. No GPU is needed."""
import ctypes as C

import pytest

from paper_1907_06696_gb300 import build as B
from paper_1907_06696_gb300 import capi


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def test_exports_every_header_function(lib):
    names = capi.header_functions()
    assert "stokes_setup" in names and "gmg_vcycle" in names and len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(capi._SIGS) == set(names), set(capi._SIGS) ^ set(names)


def test_defaults_and_strerror(lib):
    o = capi.stokes_default_options()
    assert (o.cheb_degree, o.lanczos_steps, o.schur_degree, o.restart) == (4, 12, 5, 50)
    # the last fields of the struct: their defaults pin the ctypes layout against the header's
    assert abs(o.wait_limit_s - 1.0) < 1e-15 and o.batch_vcycle == 0 and o.fused_smoother == 0
    assert (o.vmult_kernel, o.outer_arith, o.graphs) == (0, 1, 1)
    assert abs(o.smoothing_range - 15.0) < 1e-15 and abs(o.eig_safety - 1.2) < 1e-15
    assert lib.stokes_strerror(capi.STOKES_EMESH) == b"unsupported mesh"


@pytest.mark.parametrize("n,levels,bc,expect", [
    (12, 3, 0x3F, capi.STOKES_OK),       # valid: c = 3 -> not run here (needs a GPU)
    (10, 3, 0x3F, capi.STOKES_EMESH),    # 10 is not c * 4
    (40, 3, 0x3F, capi.STOKES_EMESH),    # coarsest 10 cells per axis > 6 (dense coarse solve)
    (56, 2, 0x3F, capi.STOKES_EMESH),    # coarsest 28 cells per axis
    (8, 4, 0x1F, capi.STOKES_EMESH),     # one wall not no-slip
    (8, 0, 0x3F, capi.STOKES_EINVAL),
    (0, 1, 0x3F, capi.STOKES_EINVAL),
])
def test_setup_validation(lib, n, levels, bc, expect):
    if expect == capi.STOKES_OK:
        return
    mesh = capi.stokes_mesh(0, n, levels)
    mu = capi.stokes_mu()
    mu.kind = 0
    out = C.c_void_p()
    st = lib.stokes_setup(C.byref(mesh), C.byref(mu), C.byref(capi.stokes_bc(bc)), None, None, C.byref(out))
    assert st == expect
    assert out.value is None
    assert lib.stokes_last_error() != b""


def test_null_arguments(lib):
    out = C.c_void_p()
    assert lib.stokes_setup(None, None, None, None, None, C.byref(out)) == capi.STOKES_EINVAL
    assert lib.stokes_vmult(None, -1, 0, 0, None, None, None) == capi.STOKES_EINVAL
    assert lib.gmg_vcycle(None, 0, None, None, None) == capi.STOKES_EINVAL
    assert lib.stokes_size(None, 0, 0) == 0
    lib.stokes_destroy(None)


@pytest.mark.parametrize("field,value", [("outer_solver", 4), ("outer_solver", -1), ("idr_s", 9),
                                         ("precond_kind", 2), ("outer_solver", 3), ("outer_arith", 3),
                                         ("outer_arith", -1), ("vmult_kernel", 4), ("fused_smoother", 2)])
def test_option_validation(lib, field, value):
    """Options are checked before any device work: out-of-range solvers, and MINRES (outer_solver 3)
    without the symmetric positive definite P_D (precond_kind 1), are EINVAL."""
    mesh = capi.stokes_mesh(0, 8, 4)
    mu = valid_sinker_mu()
    o = capi.stokes_default_options()
    setattr(o, field, value)
    out = C.c_void_p()
    st = lib.stokes_setup(C.byref(mesh), C.byref(mu), C.byref(capi.stokes_bc(0x3F)), C.byref(o), None, C.byref(out))
    assert st == capi.STOKES_EINVAL
    assert out.value is None


def valid_sinker_mu():
    mu = capi.stokes_mu()
    mu.kind = 0
    mu.mu_min, mu.mu_max, mu.delta, mu.omega, mu.beta = 1.0, 100.0, 200.0, 0.1, 10.0
    return mu


def setup_status(lib, mesh, mu):
    out = C.c_void_p()
    st = lib.stokes_setup(C.byref(mesh), C.byref(mu), C.byref(capi.stokes_bc(0x3F)), None, None, C.byref(out))
    assert out.value is None
    return st


@pytest.mark.parametrize("field,value", [("mu_min", -1.0), ("mu_max", 0.0), ("mu_min", float("nan")),
                                         ("mu_max", float("inf")), ("delta", float("nan")), ("omega", -0.1)])
def test_sinker_viscosity_validated_on_host(lib, field, value):
    """A non-positive or non-finite viscosity bound, or non-finite sinker parameters, are refused
    before any device work (Section 3.2: mu_min, mu_max > 0; the 1/mu mass matrix needs mu > 0)."""
    mu = valid_sinker_mu()
    setattr(mu, field, value)
    assert setup_status(lib, capi.stokes_mesh(0, 8, 4), mu) == capi.STOKES_EINVAL
    assert b"mu" in lib.stokes_last_error() or b"delta" in lib.stokes_last_error()


def test_nonfinite_sinker_centre_refused(lib):
    import numpy as np
    cen = np.array([[0.5, float("nan"), 0.5]])
    mu = valid_sinker_mu()
    mu.n_sinkers = 1
    mu.centres = cen.ctypes.data_as(C.POINTER(C.c_double))
    assert setup_status(lib, capi.stokes_mesh(0, 8, 4), mu) == capi.STOKES_EINVAL


@pytest.mark.parametrize("bad", [-1.0, 0.0, float("nan"), float("inf")])
def test_quadrature_point_viscosity_validated_on_host(lib, bad):
    import numpy as np
    n = 4
    q = np.ones(n ** 3 * 27)
    q[5 * 27 + 13] = bad
    mu = capi.stokes_mu()
    mu.kind = 1
    mu.mu_q = q.ctypes.data_as(C.POINTER(C.c_double))
    assert setup_status(lib, capi.stokes_mesh(0, n, 3), mu) == capi.STOKES_EINVAL


def octree_status(lib, keys, coarsest):
    import numpy as np
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    mesh = capi.stokes_octree(coarsest, k.size, k.ctypes.data_as(C.POINTER(C.c_uint64)))
    out = C.c_void_p()
    st = lib.stokes_setup_octree(C.byref(mesh), C.byref(valid_sinker_mu()), C.byref(capi.stokes_bc(0x3F)), None,
                                 None, C.byref(out))
    assert out.value is None
    return st


def key(l, i, j, k):
    return (l << 48) | (k << 32) | (j << 16) | i


def test_unbalanced_leaves_refused_on_host(lib):
    """A leaf set that tiles the cube but is not 2:1 balanced (a level-3 leaf against a level-1
    leaf across a vertex) is EMESH, found by the host tables before any device work."""
    leaves = [key(1, i, j, k) for k in range(2) for j in range(2) for i in range(2) if (i, j, k) != (0, 0, 0)]
    leaves += [key(2, i, j, k) for k in range(2) for j in range(2) for i in range(2) if (i, j, k) != (1, 1, 1)]
    leaves += [key(3, i, j, k) for k in (2, 3) for j in (2, 3) for i in (2, 3)]
    assert octree_status(lib, leaves, 1) == capi.STOKES_EMESH
    # the same cells with the level-3 leaves merged back into their level-2 parent are accepted by
    # the host checks (they get as far as the device, which this CPU test does not have)
    ok = leaves[:14] + [key(2, 1, 1, 1)]
    assert octree_status(lib, ok, 1) != capi.STOKES_EMESH


def test_malformed_leaves_refused_on_host(lib):
    """Leaves that overlap or leave a hole are EMESH before any device work."""
    full = [key(1, i, j, k) for k in range(2) for j in range(2) for i in range(2)]
    assert octree_status(lib, full[:-1], 1) == capi.STOKES_EMESH                  # a hole
    assert octree_status(lib, full + [key(2, 0, 0, 0)], 1) == capi.STOKES_EMESH   # an overlap


def test_debug_build_exports_and_reports_itself(lib):
    """The STOKES_DEBUG build links, exports the same functions, and says which build it is; the
    index-cut hook validates its arguments on the host in both builds."""
    dbg = capi.open_library(B.build(debug=True))
    missing = [n for n in capi.header_functions() if not hasattr(dbg, n)]
    assert not missing, missing
    assert lib.stokes_debug_build() == 0 and dbg.stokes_debug_build() == 1
    assert lib.stokes_debug_index_cut(None, 0, 1) == capi.STOKES_EINVAL
    assert b"STOKES_DEBUG builds only" in lib.stokes_last_error()
    assert dbg.stokes_debug_index_cut(None, 0, 1) == capi.STOKES_EINVAL
    assert b"octree context" in dbg.stokes_last_error()
