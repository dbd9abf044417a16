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
