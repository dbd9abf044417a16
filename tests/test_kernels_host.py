"""Kernel arithmetic on the CPU, part 2: the per-thread bodies of the cell-wise level transfers
(csrc/transfer.cuh, as k_prolong_cells and k_restrict_cells run them) and of the pressure-side
gathers of the preconditioner (csrc/pressure.cuh, as k_bt_gather and k_schur_cheb run them),
compiled with the host compiler (tests/native/transfer_host.cpp, tests/native/pressure_host.cpp)
and run over every thread index of a launch, against the oracle:

* prolongation (plain and added) and restriction against the oracle's P and P^T on the free
  entries, FP64 to 1e-14 and FP32 to 2e-6 (the GPU parity bounds), on levels whose coarse mesh
  has 1, 2 and 3 cells per axis (the last-cell ownership of the shared fine nodes);
* B^T against the oracle's element-assembled B^T on every row, 1e-12 relative (double-float
  products; the GPU bound);
* one S_hat^-1 Chebyshev step (M_p gathered per vertex in double-float, the update fused) against
  the same step formed with the oracle's M_p and diagonal, 1e-13 relative.

These pin the kernels' arithmetic and indexing without a GPU; the GPU tests check the compiled
kernels."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import sinker_inputs as si
from oracle import gmg, mesh, operators

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1907_06696_gb300", "csrc")


def host_build(tmp_path_factory, source):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    out = str(tmp_path_factory.mktemp("native") / (os.path.splitext(source)[0] + ".so"))
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I" + CSRC,
           "-I" + os.path.join(ROOT, "include"), "-I" + cuda_inc,
           os.path.join(ROOT, "tests", "native", source), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("host build failed:\n" + r.stderr)
    return C.CDLL(out)


@pytest.fixture(scope="module")
def transfer_lib(tmp_path_factory):
    L = host_build(tmp_path_factory, "transfer_host.cpp")
    for f in (L.prolong_host_f64, L.prolong_host_f32):
        f.restype = C.c_int
        f.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int]
    for f in (L.restrict_host_f64, L.restrict_host_f32):
        f.restype = C.c_int
        f.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
    return L


@pytest.fixture(scope="module")
def pressure_lib(tmp_path_factory):
    L = host_build(tmp_path_factory, "pressure_host.cpp")
    L.bt_apply_host.restype = C.c_int
    L.bt_apply_host.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_void_p]
    L.schur_step_host.restype = C.c_int
    L.schur_step_host.argtypes = [C.c_int] + [C.c_void_p] * 7 + [C.c_double, C.c_double]
    return L


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def free_masks(nc):
    """Free-entry masks (all walls no-slip) of the coarse level (nc cells) and the fine one (2 nc)."""
    return ~mesh.Mesh(nc).dirichlet, ~mesh.Mesh(2 * nc).dirichlet


@pytest.mark.parametrize("nc", [1, 2, 3])
def test_cell_prolongation_matches_oracle(transfer_lib, nc):
    free_c, free_f = free_masks(nc)
    P = gmg.prolongation(nc)
    rng = np.random.default_rng(50 + nc)
    xc = np.where(free_c, rng.uniform(-1, 1, free_c.size), 0.0)
    old = rng.uniform(-1, 1, free_f.size)
    ref = np.where(free_f, P @ xc, 0.0)
    for dtype, fn, tol in ((np.float64, transfer_lib.prolong_host_f64, 1e-14),
                           (np.float32, transfer_lib.prolong_host_f32, 2e-6)):
        xs = np.ascontiguousarray(xc, dtype=dtype)
        out = np.full(free_f.size, np.nan, dtype=dtype)   # every fine entry must be written
        assert fn(nc, xs.ctypes.data, out.ctypes.data, 0) == 0
        assert not np.isnan(out).any(), dtype
        assert np.all(out[~free_f] == 0), dtype
        assert rel(out.astype(np.float64), ref) <= tol, dtype
        # fine += P coarse: free entries gain P xc, constrained ones keep their value
        acc = np.array(old, dtype=dtype)   # a copy: the kernel writes into it
        assert fn(nc, xs.ctypes.data, acc.ctypes.data, 1) == 0
        want = old.astype(dtype).astype(np.float64) + ref
        assert np.array_equal(acc[~free_f], old.astype(dtype)[~free_f]), dtype
        assert rel(acc.astype(np.float64), want) <= tol, dtype


@pytest.mark.parametrize("nc", [1, 2, 3])
def test_cell_restriction_matches_oracle(transfer_lib, nc):
    free_c, free_f = free_masks(nc)
    P = gmg.prolongation(nc)
    rng = np.random.default_rng(60 + nc)
    r = np.where(free_f, rng.uniform(-1, 1, free_f.size), 0.0)   # a residual: zero where constrained
    ref = np.where(free_c, P.T @ r, 0.0)
    for dtype, fn, tol in ((np.float64, transfer_lib.restrict_host_f64, 1e-14),
                           (np.float32, transfer_lib.restrict_host_f32, 2e-6)):
        rs = np.ascontiguousarray(r, dtype=dtype)
        out = np.full(free_c.size, np.nan, dtype=dtype)
        assert fn(nc, rs.ctypes.data, out.ctypes.data) == 0
        assert np.all(out[~free_c] == 0), dtype
        assert rel(out.astype(np.float64), ref) <= tol, dtype


def test_cell_transfers_are_transposes(transfer_lib):
    """<P x, y> = <x, P^T y> on the free entries, in FP64, for the kernel pair itself."""
    nc = 3
    free_c, free_f = free_masks(nc)
    rng = np.random.default_rng(70)
    x = np.where(free_c, rng.standard_normal(free_c.size), 0.0)
    y = np.where(free_f, rng.standard_normal(free_f.size), 0.0)
    px = np.empty(free_f.size)
    pty = np.empty(free_c.size)
    assert transfer_lib.prolong_host_f64(nc, x.ctypes.data, px.ctypes.data, 0) == 0
    assert transfer_lib.restrict_host_f64(nc, y.ctypes.data, pty.ctypes.data) == 0
    a, b = float(px @ y), float(x @ pty)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 8])
def test_bt_gather_matches_oracle(pressure_lib, n):
    m = mesh.Mesh(n)
    ops = operators.Operators(m, np.ones(m.n_cells))   # B^T carries no viscosity
    rng = np.random.default_rng(80 + n)
    p = rng.uniform(-1, 1, m.n_p)
    ref = ops.apply_BT(p)
    out = np.full(m.n_u, np.nan)
    assert pressure_lib.bt_apply_host(n, m.h, p.ctypes.data, out.ctypes.data) == 0
    assert np.all(out[m.dirichlet] == 0)
    assert rel(out, ref) <= 1e-12
    assert np.abs(out - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["cube4", "cube8"])
@pytest.mark.parametrize("c1", [0.0, 0.37])
def test_schur_step_matches_oracle(pressure_lib, name, c1):
    """d' = c1 d + c2 D^-1 (r - M_p z), z' = z + d' with the oracle's 1/mu-weighted M_p and its
    diagonal, on the finest-level sinker viscosity (jumps between neighbouring cells)."""
    from oracle import sinker
    prob = si.workload(name)
    m = mesh.Mesh(prob.n)
    mu = sinker.level_viscosities(m, prob, prob.n_levels)[-1]
    ops = operators.Operators(m, mu)
    rng = np.random.default_rng(90)
    r, z, d = (rng.uniform(-1, 1, m.n_p) for _ in range(3))
    dinv = 1.0 / ops.diag_Mp()
    c2 = 1.9
    d_ref = c1 * d + c2 * dinv * (r - ops.apply_Mp(z))
    z_ref = z + d_ref
    scale = np.ascontiguousarray(m.h ** 3 / mu)
    z_new = np.empty(m.n_p)
    d_new = np.empty(m.n_p)
    assert pressure_lib.schur_step_host(prob.n, scale.ctypes.data, r.ctypes.data, dinv.ctypes.data, z.ctypes.data,
                                        d.ctypes.data, z_new.ctypes.data, d_new.ctypes.data, c1, c2) == 0
    assert rel(d_new, d_ref) <= 1e-13
    assert rel(z_new, z_ref) <= 1e-13


def log_uniform(rng, size, lo, hi):
    return 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size)


def test_bt_gather_wide_magnitudes(pressure_lib):
    """Double-float B^T (float exponent range, ~47-bit significands) with pressures of magnitude
    1e-6..1e6 and random signs, h = 1/8: still within 1e-12 of the oracle's FP64 B^T."""
    n = 8
    m = mesh.Mesh(n)
    ops = operators.Operators(m, np.ones(m.n_cells))
    rng = np.random.default_rng(100)
    p = rng.choice([-1.0, 1.0], m.n_p) * log_uniform(rng, m.n_p, 1e-6, 1e6)
    ref = ops.apply_BT(p)
    out = np.empty(m.n_u)
    assert pressure_lib.bt_apply_host(n, m.h, p.ctypes.data, out.ctypes.data) == 0
    assert rel(out, ref) <= 1e-12


def test_schur_step_wide_viscosity(pressure_lib):
    """The S_hat^-1 step with the cell viscosity log-uniform over 1e-12..1e12 (s_K = h^3 / mu_K over
    24 decades) and z, d, r of magnitude 1e-6..1e6: within 1e-12 of the FP64 step."""
    n = 8
    m = mesh.Mesh(n)
    rng = np.random.default_rng(101)
    mu = log_uniform(rng, m.n_cells, 1e-12, 1e12)
    ops = operators.Operators(m, mu)
    r, z, d = (rng.choice([-1.0, 1.0], m.n_p) * log_uniform(rng, m.n_p, 1e-6, 1e6) for _ in range(3))
    dinv = 1.0 / ops.diag_Mp()
    c1, c2 = 0.37, 1.9
    d_ref = c1 * d + c2 * dinv * (r - ops.apply_Mp(z))
    scale = np.ascontiguousarray(m.h ** 3 / mu)
    z_new = np.empty(m.n_p)
    d_new = np.empty(m.n_p)
    assert pressure_lib.schur_step_host(n, scale.ctypes.data, r.ctypes.data, dinv.ctypes.data, z.ctypes.data,
                                        d.ctypes.data, z_new.ctypes.data, d_new.ctypes.data, c1, c2) == 0
    assert rel(d_new, d_ref) <= 1e-12
    assert rel(z_new, z + d_ref) <= 1e-12
