"""Host side of the adaptive path through the C ABI (no GPU): the library's sinker-shell
refinement and 2:1 balance give exactly the oracle's leaves (integer work, bit-exact)."""
import numpy as np
import pytest

import sinker_inputs as si
from oracle import octree


@pytest.fixture(scope="module")
def capi():
    from paper_1907_06696_gb300 import build as B
    from paper_1907_06696_gb300 import capi as api
    B.build()
    api.load()
    return api


@pytest.mark.parametrize("name", ["oct_xs", "oct_s", "oct_m"])
def test_sinker_mesh_matches_oracle(capi, name):
    p = si.octree_workload(name)
    keys = capi.stokes_octree_sinker_mesh(p.base_level, p.centres, p.max_levels, p.shell_radius, p.shell_half_width)
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    ref = np.array(sorted(octree.cell_key(c) for c in lv), dtype=np.uint64)
    assert keys.dtype == np.uint64
    assert np.array_equal(keys, ref)


def test_sinker_mesh_arguments(capi):
    import ctypes as C
    lib = capi.load()
    n = C.c_int64(0)
    cen = np.array([0.5, 0.5, 0.5])
    lv = np.array([4], dtype=np.int32)
    # capacity too small with a buffer: EINVAL, count still reported
    buf = np.empty(3, dtype=np.uint64)
    st = lib.stokes_octree_sinker_mesh(2, 1, cen.ctypes.data, lv.ctypes.data, 0.05, 0.02, buf.ctypes.data, 3,
                                       C.byref(n))
    assert st == capi.STOKES_EINVAL and n.value > 3
    assert lib.stokes_octree_sinker_mesh(16, 0, None, None, 0.05, 0.02, None, 0, C.byref(n)) == capi.STOKES_EINVAL
    assert lib.stokes_octree_sinker_mesh(2, 0, None, None, 0.05, 0.02, None, 0, None) == capi.STOKES_EINVAL
    # no sinkers: the uniform base grid
    assert lib.stokes_octree_sinker_mesh(2, 0, None, None, 0.05, 0.02, None, 0, C.byref(n)) == capi.STOKES_OK
    assert n.value == 64


@pytest.mark.parametrize("name", ["oct_xs", "oct_s"])
def test_gradient_refinement_matches_oracle(capi, name):
    """Host gradient-indicator refinement (Section 3.3 reading) against oracle/refine.py on the
    same random active velocity: indicators to rounding, new leaves bit-exact; a second cycle
    from the refined mesh too."""
    from oracle import adaptive, refine
    p = si.octree_workload(name)
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    rng = np.random.default_rng(31)
    for cycle in range(2):
        t = octree.Octree(lv, p.coarsest_level)
        S = adaptive.AdaptiveStokes(t, p, mu_leaf=np.ones(len(t.leaves)))
        u = rng.uniform(-1, 1, 3 * t.n_nodes)
        keys = np.array([octree.cell_key(c) for c in t.leaves], dtype=np.uint64)
        new, eta = capi.stokes_octree_refine_gradient(keys[::-1], p.coarsest_level, u)   # any input order
        eta_o = refine.gradient_indicator(S, u)
        assert np.max(np.abs(eta - eta_o)) <= 1e-13 * np.max(eta_o)
        lv = refine.refine_by_indicator(t.leaves, eta_o)
        assert np.array_equal(new, np.array([octree.cell_key(c) for c in lv], dtype=np.uint64))


def test_gradient_refinement_arguments(capi):
    import ctypes as C
    lib = capi.load()
    keys = np.array([octree.cell_key((1, i, j, k)) for k in range(2) for j in range(2) for i in range(2)],
                    dtype=np.uint64)
    mesh = capi.stokes_octree(1, keys.size, keys.ctypes.data_as(C.POINTER(C.c_uint64)))
    u = np.zeros(3 * 5 ** 3)
    n = C.c_int64(0)
    for frac in (0.0, 1.5, -1.0):
        assert lib.stokes_octree_refine_gradient(C.byref(mesh), u.ctypes.data, frac, None, None, 0,
                                                 C.byref(n)) == capi.STOKES_EINVAL
    assert lib.stokes_octree_refine_gradient(C.byref(mesh), None, 0.5, None, None, 0, C.byref(n)) == capi.STOKES_EINVAL
    u[7] = np.nan
    assert lib.stokes_octree_refine_gradient(C.byref(mesh), u.ctypes.data, 0.5, None, None, 0,
                                             C.byref(n)) == capi.STOKES_EINVAL
    u[7] = 0.0
    # all-zero velocity: every indicator 0, ties by key: the first 4 leaves are split
    assert lib.stokes_octree_refine_gradient(C.byref(mesh), u.ctypes.data, 0.5, None, None, 0,
                                             C.byref(n)) == capi.STOKES_OK
    assert n.value == 4 + 4 * 8
    bad = keys[:7].copy()                     # not a tiling of the cube
    mesh_bad = capi.stokes_octree(1, bad.size, bad.ctypes.data_as(C.POINTER(C.c_uint64)))
    assert lib.stokes_octree_refine_gradient(C.byref(mesh_bad), u.ctypes.data, 0.5, None, None, 0,
                                             C.byref(n)) == capi.STOKES_EMESH
