"""The allocation-free Schur-inverse entry point.

Some callers cannot allocate device memory (their host application reserves
all of it in its own pool, or they must avoid the device-wide synchronisation
cudaMalloc/cudaFree can cause), so they cannot create a context.
stokes_schur_inverse_noalloc serves them with its work vectors in a fixed
device array. This test calls it through the C ABI twice in a row (the array
keeps the previous call's contents) and compares each result with the
context-based stokes_schur_inverse. It lives in its own file, collected last,
and passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import sinker_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06696_gb300 import build as B
    from paper_1907_06696_gb300 import capi as api
    B.build()
    api.load()
    return api


def problem(name):
    # n32: 32^3 cells, the largest size the fixed array holds (33^3 = STOKES_NOALLOC_MAX_NP pressure DoFs)
    return si.dr_problem(32, 4, 4, 1e4, 7032, "n32") if name == "n32" else si.workload(name)


@pytest.mark.parametrize("name,degree", [("cube8", None), ("cube16", None), ("cube8", 0), ("cube16", 3),
                                         ("n32", None)])
def test_noalloc_schur_matches_context_entry_point(capi, name, degree):
    p = problem(name)
    opt = capi.stokes_default_options()
    if degree is not None:
        opt.schur_degree = degree
    degree = opt.schur_degree
    ctx = capi.stokes_setup_problem(p, options=opt)
    n_p = ctx.n_p
    mu = torch.empty(p.n ** 3, dtype=torch.float64, device="cuda")
    capi.stokes_get_viscosity(ctx, -1, mu)
    for call in range(2):
        rp = torch.tensor(si.uniform(7000 + call, n_p), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(rp)
        capi.stokes_schur_inverse(ctx, rp, ref)
        got = torch.full_like(rp, float("nan"))
        capi.stokes_schur_inverse_noalloc(p.n, mu, rp, got, degree)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(g - r) <= F64_TOL * np.linalg.norm(r)
        assert np.abs(g - r).max() <= 10 * F64_TOL * np.abs(r).max()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array(capi):
    lib = capi.load()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 33^3 = 35937 pressure DoFs fit; 34^3 do not; sizes whose (n + 1)^3 overflows are refused too
    for n in (33, 0, -1, 2 ** 31 - 1):
        assert lib.stokes_schur_inverse_noalloc(n, x.data_ptr(), x.data_ptr(), x.data_ptr(), 5, None) == capi.STOKES_EINVAL
    assert lib.stokes_schur_inverse_noalloc(4, x.data_ptr(), x.data_ptr(), x.data_ptr(), -1, None) == capi.STOKES_EINVAL
    assert lib.stokes_schur_inverse_noalloc(4, None, x.data_ptr(), x.data_ptr(), 5, None) == capi.STOKES_EINVAL
