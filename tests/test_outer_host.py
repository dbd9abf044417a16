"""Kernel arithmetic on the CPU: device functions compiled with the host compiler and run thread
by thread, against the oracle on sinker viscosity with random sources.

* the double-float outer Stokes kernel (csrc/outer.cuh phases, tests/native/outer_host.cpp)
  against the oracle's FP64 [A B^T; B 0], to the 1e-12 relative bound of the GPU parity test:
  sum factorisation, the symmetric-pair exchange through shared memory, the rotated local frames;
* the V-cycle level operator's cell computation (csrc/brick.cuh brick_compute with the scatter
  rule of k_cell_atomic, tests/native/level_host.cpp) against the oracle's A: FP64 to 1e-12,
  FP32 to 2e-6 (the GPU parity bounds).

These pin the kernels' arithmetic without a GPU; the GPU tests check the compiled kernels."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import sinker_inputs as si
from oracle import mesh, operators, sinker

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
def lib(tmp_path_factory):
    L = host_build(tmp_path_factory, "outer_host.cpp")
    L.outer_apply_host.restype = C.c_int
    L.outer_apply_host.argtypes = [C.c_int] + [C.c_void_p] * 5
    return L


@pytest.fixture(scope="module")
def level_lib(tmp_path_factory):
    L = host_build(tmp_path_factory, "level_host.cpp")
    for f in (L.level_apply_f64, L.level_apply_f32):
        f.restype = C.c_int
        f.argtypes = [C.c_int] + [C.c_void_p] * 3
    return L


@pytest.mark.parametrize("name", ["cube4", "cube8"])
def test_outer_kernel_phases_match_oracle(lib, name):
    p = si.workload(name)
    m = mesh.Mesh(p.n)
    mu = sinker.level_viscosities(m, p, p.n_levels)[-1]
    ops = operators.Operators(m, mu)
    rng = np.random.default_rng(41)
    x = rng.uniform(-1, 1, m.n_u + m.n_p)
    ref = ops.apply_stokes(x)
    du = np.empty(m.n_u)
    dp = np.empty(m.n_p)
    xu = np.ascontiguousarray(x[:m.n_u])
    xp = np.ascontiguousarray(x[m.n_u:])
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    assert lib.outer_apply_host(p.n, mu.ctypes.data, xu.ctypes.data, xp.ctypes.data, du.ctypes.data,
                                dp.ctypes.data) == 0
    got = np.concatenate([du, dp])
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["cube4", "cube8"])
def test_level_cell_kernel_matches_oracle(level_lib, name):
    p = si.workload(name)
    m = mesh.Mesh(p.n)
    mu = sinker.level_viscosities(m, p, p.n_levels)[-1]
    ops = operators.Operators(m, mu)
    rng = np.random.default_rng(42)
    x = rng.uniform(-1, 1, m.n_u)
    ref = ops.apply_A(x)
    for dtype, fn, tol in ((np.float64, level_lib.level_apply_f64, 1e-12), (np.float32, level_lib.level_apply_f32, 2e-6)):
        xs = np.ascontiguousarray(x, dtype=dtype)
        mus = np.ascontiguousarray(mu, dtype=dtype)
        out = np.empty(m.n_u, dtype=dtype)
        assert fn(p.n, mus.ctypes.data, xs.ctypes.data, out.ctypes.data) == 0
        assert np.linalg.norm(out.astype(np.float64) - ref) <= tol * np.linalg.norm(ref), dtype
