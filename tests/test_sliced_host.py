"""The digit-sliced outer Stokes operator (csrc/sliced.cuh) on the CPU: its integer tables against
the oracle's element matrices, each arithmetic step against exact arithmetic (Python integers and
fractions), and the whole operator against the oracle's FP64 [A B^T; B 0] at the 1e-12 bound of
the outer operator, on sinker viscosity and over wide ranges of viscosity and input magnitude.

The slice products are emulated as exact integer dot products; that a tensor core's FP32
accumulation of f16 digits reproduces them rests on the table bound checked here (every partial
sum an integer below 2^24)."""
import ctypes as C
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import sinker_inputs as si
from oracle import fe, mesh, operators, sinker

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1907_06696_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    out = str(tmp_path_factory.mktemp("native") / "sliced_host.so")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I" + CSRC,
           "-I" + os.path.join(ROOT, "include"), "-I" + cuda_inc,
           os.path.join(ROOT, "tests", "native", "sliced_host.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("host build failed:\n" + r.stderr)
    L = C.CDLL(out)
    L.sliced_tables_host.restype = C.c_int
    L.sliced_tables_host.argtypes = [C.c_void_p, C.c_void_p]
    L.to_fixed_host.restype = C.c_longlong
    L.to_fixed_host.argtypes = [C.c_double, C.c_int]
    L.binade_host.restype = C.c_int
    L.binade_host.argtypes = [C.c_double]
    L.digits_host.restype = None
    L.digits_host.argtypes = [C.c_longlong, C.c_void_p]
    L.digit_pairs_host.restype = None
    L.digit_pairs_host.argtypes = [C.c_longlong, C.c_longlong, C.c_void_p]
    L.combine_host.restype = None
    L.combine_host.argtypes = [C.c_void_p, C.c_void_p]
    L.compose_host.restype = None
    L.compose_host.argtypes = [C.c_int] + [C.c_void_p] * 4
    L.sliced_apply_host.restype = C.c_int
    L.sliced_apply_host.argtypes = [C.c_int] + [C.c_void_p] * 5
    return L


def tables(lib):
    KX = np.empty((81, 89))
    KU = np.empty((8, 81))
    assert lib.sliced_tables_host(KX.ctypes.data, KU.ctypes.data) == 0   # every entry an integer
    return KX, KU


def significant_bits(v):
    v = abs(int(v))
    if v == 0:
        return 0
    while v % 2 == 0:
        v //= 2
    return v.bit_length()


def test_tables_are_the_scaled_element_matrices(lib):
    """K_X = [5400 A_hat / h | 216 B_hat^T / h^2] and K_U = 216 B_hat / h^2 with the oracle's
    element matrices (any h); integers exact in f16 (<= 11 significant bits, |v| <= 65504), and
    every row's absolute sum times the largest digit magnitude 2^7 below 2^24."""
    KX, KU = tables(lib)
    h = 0.3
    A, B = fe.element_A(h, 1.0), fe.element_B(h)
    assert np.abs(KX[:, :81] - 5400 * A / h).max() < 1e-9
    assert np.abs(KX[:, 81:] - 216 * B.T / h ** 2).max() < 1e-9
    assert np.abs(KU - 216 * B / h ** 2).max() < 1e-9
    for K in (KX, KU):
        assert max(significant_bits(v) for v in K.ravel()) <= 6
        assert np.abs(K).max() <= 2 ** 15
    assert np.abs(KX).sum(axis=1).max() == 78464
    assert np.abs(KX).sum(axis=1).max() * 2 ** 7 < 2 ** 24
    assert np.abs(KU).sum(axis=1).max() * 2 ** 7 < 2 ** 24


def exact_fixed(v, E):
    """round(v 2^(54 - E)), ties away from zero, in exact arithmetic."""
    f = Fraction(v) * Fraction(2) ** (54 - E)
    a = abs(f)
    r = int(a + Fraction(1, 2))
    return r if f >= 0 else -r


def test_binade_and_fixed_point_are_exact(lib):
    rng = np.random.default_rng(200)
    vals = list(rng.standard_normal(300) * 10.0 ** rng.uniform(-30, 30, 300))
    vals += [1.0, -1.0, 0.5, 0.75, 2.0 ** -1022, -(2.0 ** 1000), 1.0 - 2.0 ** -53, 0.0, -0.0, 5e-324]
    for v in vals:
        E = lib.binade_host(v)
        if v == 0.0 or abs(v) < 2.0 ** -1022:
            assert lib.to_fixed_host(v, 0) == 0
            continue
        assert 2.0 ** (E - 1) <= abs(v) < 2.0 ** E, (v, E)
        for EE in (E, E + 1, E + 7, E + 60):   # the cell's exponent is >= the value's own
            X = lib.to_fixed_host(v, EE)
            assert X == exact_fixed(v, EE), (v, EE)
            assert abs(X) <= 2 ** 54


def test_balanced_digits_reconstruct(lib):
    rng = np.random.default_rng(201)
    xs = [int(x) for x in rng.integers(-(2 ** 54), 2 ** 54, 2000, dtype=np.int64)]
    xs += [0, 1, -1, 127, 128, -128, -129, 255, 256, 2 ** 54, -(2 ** 54), 2 ** 54 - 1, -(2 ** 54) + 1]
    d = np.empty(7, dtype=np.int32)
    for X in xs:
        lib.digits_host(X, d.ctypes.data)
        assert all(-128 <= int(v) <= 127 for v in d)
        assert sum(int(d[j]) * 256 ** j for j in range(7)) == X


def test_digit_pairs_as_f16_bits(lib):
    """The packed f16 bits of 1536 + d_j for two values, minus 1536 in f16, are the balanced digits
    of each (the same digits as the digit-by-digit extraction)."""
    rng = np.random.default_rng(206)
    xs = [int(x) for x in rng.integers(-(2 ** 54), 2 ** 54, 4000, dtype=np.int64)]
    xs += [2 ** 54, -(2 ** 54), 0, -1, 1, 127, 128, -128, -129]
    bits = np.empty(7, dtype=np.uint32)
    d = np.empty(7, dtype=np.int32)
    for X0, X1 in zip(xs[0::2], xs[1::2]):
        lib.digit_pairs_host(X0, X1, bits.ctypes.data)
        halves = bits.view(np.uint16).reshape(7, 2).view(np.float16).astype(np.float64) - 1536.0
        for col, X in ((0, X0), (1, X1)):
            lib.digits_host(X, d.ctypes.data)
            assert np.array_equal(halves[:, col], d.astype(np.float64))


def test_combine_is_accurate(lib):
    """2^-48 sum_j 256^j D_j for integer slice products |D_j| < 2^23.3 (recombined lowest slice
    first, as the slices come off the tensor core), within 2^-45 of 2^-48 sum |D_j| 256^j."""
    rng = np.random.default_rng(202)
    hl = np.empty(2, dtype=np.float32)
    for _ in range(3000):
        D = rng.integers(-(2 ** 23), 2 ** 23, 7).astype(np.float32)
        if rng.random() < 0.3:   # leading slices zero (small outputs)
            D[7 - rng.integers(1, 6):] = 0
        lib.combine_host(D.ctypes.data, hl.ctypes.data)
        exact = Fraction(sum(int(D[j]) * 256 ** j for j in range(7)), 2 ** 48)
        got = Fraction(float(hl[0])) + Fraction(float(hl[1]))
        scale = Fraction(sum(abs(int(D[j])) * 256 ** j for j in range(7)), 2 ** 48)
        assert abs(got - exact) <= scale / 2 ** 45 + Fraction(1, 2 ** 68)


def test_compose_matches_fp64_bit_for_bit(lib):
    """compose(hi, lo, s) == (double(hi) + double(lo)) 2^s, rounded once, as FP64 gives it: random
    normalised pairs, opposite signs, powers of two with a negative low part, exact ties."""
    rng = np.random.default_rng(203)
    n = 20000
    hi = (rng.standard_normal(n) * 10.0 ** rng.uniform(-20, 20, n)).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    k = n // 4
    hi[:k] = np.float32(2.0) ** rng.integers(-40, 40, k).astype(np.float32) * rng.choice([-1, 1], k)
    lo[:k] = (-np.sign(hi[:k]) * rng.uniform(0, 0.25, k) * np.spacing(np.abs(hi[:k]))).astype(np.float32)
    # ties: lo exactly half an FP64 ulp of hi + lo's neighbourhood
    t = slice(k, 2 * k)
    lo[t] = (np.sign(rng.standard_normal(k)) * np.spacing(np.abs(hi[t])).astype(np.float64) * 2.0 ** -30).astype(np.float32)
    lo[2 * k:2 * k + 50] = 0
    shift = rng.integers(-900, 900, n).astype(np.int32)
    # keep the results in the normal FP64 range (outside it the FP64 path is taken)
    want = (hi.astype(np.float64) + lo.astype(np.float64)) * np.ldexp(1.0, shift)
    ok = np.isfinite(want) & (np.abs(want) >= 2.0 ** -1022)
    hi, lo, shift, want = hi[ok], lo[ok], shift[ok], want[ok]
    want = np.ldexp(hi.astype(np.float64) + lo.astype(np.float64), shift)
    out = np.empty(hi.size)
    lib.compose_host(hi.size, hi.ctypes.data, lo.ctypes.data, shift.ctypes.data, out.ctypes.data)
    assert np.array_equal(out.view(np.int64), want.view(np.int64))


def apply(lib, n, mu, x):
    m = mesh.Mesh(n)
    xu = np.ascontiguousarray(x[:m.n_u])
    xp = np.ascontiguousarray(x[m.n_u:])
    du = np.empty(m.n_u)
    dp = np.empty(m.n_p)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    assert lib.sliced_apply_host(n, mu.ctypes.data, xu.ctypes.data, xp.ctypes.data, du.ctypes.data,
                                 dp.ctypes.data) == 0
    return np.concatenate([du, dp])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", ["cube4", "cube8"])
def test_sliced_operator_matches_oracle(lib, name):
    p = si.workload(name)
    m = mesh.Mesh(p.n)
    mu = sinker.level_viscosities(m, p, p.n_levels)[-1]
    ops = operators.Operators(m, mu)
    x = np.random.default_rng(204).uniform(-1, 1, m.n_u + m.n_p)
    ref = ops.apply_stokes(x)
    got = apply(lib, p.n, mu, x)
    assert rel(got, ref) <= 1e-12
    assert rel(got[:m.n_u], ref[:m.n_u]) <= 1e-12 and rel(got[m.n_u:], ref[m.n_u:]) <= 1e-12
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_sliced_operator_wide_scale_spread(lib):
    """Cell viscosity log-uniform over 1e-12..1e12 and inputs of magnitude 1e-6..1e6 with random
    signs: within 1e-12 of the oracle on the whole operator and on each block. Cells where
    (25 h / mu_c) p exceeds u by more than 2^8 form B u with the double-float moments, so the
    pressure block keeps its precision there."""
    n = 6
    m = mesh.Mesh(n)
    rng = np.random.default_rng(205)
    mu = 10.0 ** rng.uniform(-12, 12, m.n_cells)
    ops = operators.Operators(m, mu)
    N = m.n_u + m.n_p
    x = rng.choice([-1.0, 1.0], N) * 10.0 ** rng.uniform(-6, 6, N)
    ref = ops.apply_stokes(x)
    got = apply(lib, n, mu, x)
    assert rel(got, ref) <= 1e-12
    assert rel(got[:m.n_u], ref[:m.n_u]) <= 1e-12 and rel(got[m.n_u:], ref[m.n_u:]) <= 1e-12
