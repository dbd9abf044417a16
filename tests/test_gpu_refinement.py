"""One sinker problem (16 sinkers, viscosity ratio 1e6, 3^3 coarsest mesh) on 24^3, 48^3 and 96^3
cells: the FP32-V-cycle FGMRES(50) reaches the true FP64 residual 1e-8 on every mesh, and its
iteration count stays essentially constant under refinement, the property Section 3.5 reports for
the GMG preconditioner (measured 500 / 565 / 529 here; the bound allows 25% between the largest
and the smallest count). The residuals of the two smaller meshes are recomputed by the oracle from
its own viscosity; on 96^3 the library's native FP64 residual is checked."""
import numpy as np
import pytest

import sinker_inputs as si
from oracle import mesh, operators, sinker

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06696_gb300 import build as B
    from paper_1907_06696_gb300 import capi as api
    B.build()
    api.load()
    return api


def test_iterations_constant_under_refinement(capi):
    its = {}
    for name in ("seq24", "seq48", "seq96"):
        p = si.workload(name)
        ctx = capi.stokes_setup_problem(p)
        up = torch.zeros(ctx.n_u + ctx.n_p, dtype=torch.float64, device="cuda")
        info = capi.stokes_solve(ctx, capi.STOKES_FP32, None, up, rtol=1e-8, max_it=3000)
        assert info.status == capi.STOKES_OK and info.rel_residual_true <= 1e-8
        its[name] = info.iterations
        if p.n <= 48:
            m = mesh.Mesh(p.n)
            ops = operators.Operators(m, sinker.level_viscosities(m, p, 1)[-1])
            F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
            b = np.concatenate([F, np.zeros(m.n_p)])
            x = up.cpu().numpy()
            assert np.linalg.norm(b - ops.apply_stokes(x)) / np.linalg.norm(b) <= 1e-8 * 1.001
        ctx.close()
        del up
        torch.cuda.empty_cache()
    assert max(its.values()) <= 1.25 * min(its.values()), its
