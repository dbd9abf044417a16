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
    assert abs(o.smoothing_range - 15.0) < 1e-15 and abs(o.eig_safety - 1.2) < 1e-15
    assert lib.stokes_strerror(capi.STOKES_EMESH) == b"unsupported mesh"


@pytest.mark.parametrize("n,levels,bc,expect", [
    (12, 3, 0x3F, capi.STOKES_OK),       # valid: c = 3 -> not run here (needs a GPU)
    (10, 3, 0x3F, capi.STOKES_EMESH),    # 10 is not c * 4
    (40, 3, 0x3F, capi.STOKES_EMESH),    # coarsest 10 cells per axis > 4
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
                                         ("precond_kind", 2), ("outer_solver", 3)])
def test_option_validation(lib, field, value):
    """Options are checked before any device work: out-of-range solvers, and MINRES (outer_solver 3)
    without the symmetric positive definite P_D (precond_kind 1), are EINVAL."""
    mesh = capi.stokes_mesh(0, 8, 4)
    mu = capi.stokes_mu()
    mu.kind = 0
    o = capi.stokes_default_options()
    setattr(o, field, value)
    out = C.c_void_p()
    st = lib.stokes_setup(C.byref(mesh), C.byref(mu), C.byref(capi.stokes_bc(0x3F)), C.byref(o), None, C.byref(out))
    assert st == capi.STOKES_EINVAL
    assert out.value is None
