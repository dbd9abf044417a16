"""A solve-estimate-refine loop on the CPU (Section 3.3 reading): the oracle solves the adaptive
Stokes problem, the library's host refinement (C ABI) splits the 1/7 of the leaves with the largest
gradient indicator. Checks: each cycle splits floor(n/7 + 1/2) leaves (the leaf count grows by at
least 7 per split leaf, so it about doubles), the indicator is largest around the sinker (the
split leaves lie closer to it than the average leaf), and every mesh solves to 1e-8."""
import numpy as np
import pytest

import sinker_inputs as si
from oracle import adaptive, krylov, octree


@pytest.fixture(scope="module")
def capi():
    from paper_1907_06696_gb300 import build as B
    from paper_1907_06696_gb300 import capi as api
    B.build()
    api.load()
    return api


def test_adaptive_loop_oracle_solves(capi):
    p, cycles = si.adaptive_loop_workload("adapt_xs")
    leaves = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                                 p.shell_half_width))
    assert len(leaves) == 8 ** p.base_level
    c0 = np.asarray(p.centres)[0]
    for _ in range(cycles):
        t = octree.Octree(leaves, p.coarsest_level)
        S = adaptive.AdaptiveStokes(t, p)
        b = np.concatenate([S.F, np.zeros(S.n_p)])
        x, its, _ = krylov.fgmres(S.apply_stokes, S.precondition, b, rtol=1e-8, max_it=500)
        assert np.linalg.norm(b - S.apply_stokes(x)) <= 1e-8 * np.linalg.norm(b)
        keys = np.array([octree.cell_key(c) for c in t.leaves], dtype=np.uint64)
        new, eta = capi.stokes_octree_refine_gradient(keys, p.coarsest_level, x[:S.n_u])
        m = int(np.floor(len(keys) / 7 + 0.5))
        assert len(new) >= len(keys) + 7 * m
        centre = lambda c: (np.array(c[1:]) + 0.5) * 2.0 ** -c[0]
        dist = np.array([np.linalg.norm(centre(c) - c0) for c in t.leaves])
        split = np.argsort(-eta, kind="stable")[:m]
        assert dist[split].mean() < dist.mean()
        leaves = [(int(k >> 48), int(k & 0xFFFF), int((k >> 16) & 0xFFFF), int((k >> 32) & 0xFFFF)) for k in new]
        assert octree.is_balanced(leaves)
