"""Pins of the adaptive (octree) oracle against facts fixed by the mathematics.

* the refined and balanced leaves tile the cube, are 2:1 balanced, and balancing is idempotent;
* hanging-node constraints reproduce every quadratic velocity field and every trilinear
  pressure field exactly (they are the coarse cell's interpolants);
* with constant viscosity the unconstrained active operator applied to a quadratic field
  equals int phi_i (-div 2 mu eps(u)) (a constant vector times int phi_i) at every free row:
  element matrices, constraint weights and assembly all enter;
* the level prolongation reproduces quadratics;
* on an octree whose leaves form a uniform grid, the active operator and the local-smoothing
  V-cycle coincide with the uniform oracle (no refinement edge, one copy level);
* FGMRES with the local-smoothing preconditioner reaches the dense direct solution;
* with constant viscosity the local-smoothing V-cycle solves the velocity block in a handful
  of iterations (a wrong refinement-edge treatment destroys this).
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

import sinker_inputs as si
from oracle import adaptive, gmg, krylov, octree
from oracle.mesh import Mesh
from oracle.operators import Operators
from oracle.sinker import level_viscosities


def build(name):
    p = si.octree_workload(name)
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    return p, octree.Octree(lv, p.coarsest_level)


@pytest.fixture(scope="module")
def oct_s():
    return build("oct_s")


def lattice_coords(tree, keys):
    pts = np.array([tree._point(int(k)) for k in keys], dtype=np.float64)
    return pts / (tree.Mx - 1)


def test_tiling_and_balance(oct_s):
    p, t = oct_s
    vol = sum(8.0 ** (-c[0]) for c in t.leaves)
    assert vol == pytest.approx(1.0, abs=1e-15)
    for c in t.leaves:          # no leaf has a leaf ancestor
        a = c
        while a[0] > 0:
            a = octree.parent(a)
            assert a not in t.leaf_set
    assert octree.is_balanced(t.leaves)
    assert set(octree.balance(t.leaves)) == set(t.leaves)
    unbalanced = octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius, p.shell_half_width)
    assert not octree.is_balanced(unbalanced)


def test_hanging_constraints_reproduce_quadratics(oct_s):
    p, t = oct_s
    rng = np.random.default_rng(5)
    X = lattice_coords(t, t.u_keys)
    coef = rng.standard_normal((3, 10))

    def quad(x):
        x0, x1, x2 = x[..., 0], x[..., 1], x[..., 2]
        basis = np.stack([np.ones_like(x0), x0, x1, x2, x0 * x0, x1 * x1, x2 * x2, x0 * x1, x1 * x2, x0 * x2], -1)
        return basis @ coef.T                                   # (..., 3)

    u = quad(X).T.ravel()                                       # component-blocked
    C = adaptive.velocity_expand(adaptive.constraint_matrix(t.leaf_u, t.n_nodes, 27))
    local = (C @ u).reshape(len(t.leaves), 3, 27)
    pts = np.array([[t._point(t.key(q)) for q in t.cell_nodes_lattice(c)] for c in t.leaves]) / (t.Mx - 1)
    exact = np.transpose(quad(pts), (0, 2, 1))
    assert np.max(np.abs(local - exact)) < 1e-13 * np.max(np.abs(exact))
    assert len(t.hanging_u) > 100
    # pressure: trilinear fields
    Xp = lattice_coords(t, t.p_keys)
    a = rng.standard_normal(8)
    tri = lambda x: (a[0] + a[1] * x[..., 0] + a[2] * x[..., 1] + a[3] * x[..., 2] + a[4] * x[..., 0] * x[..., 1]
                     + a[5] * x[..., 1] * x[..., 2] + a[6] * x[..., 0] * x[..., 2] + a[7] * x[..., 0] * x[..., 1] * x[..., 2])
    Cp = adaptive.constraint_matrix(t.leaf_p, t.n_p, 8)
    lp = (Cp @ tri(Xp)).reshape(len(t.leaves), 8)
    ptsp = np.array([[t._point(t.key(q)) for q in t.cell_vertices_lattice(c)] for c in t.leaves]) / (t.Mx - 1)
    assert np.max(np.abs(lp - tri(ptsp))) < 1e-13 * np.max(np.abs(tri(ptsp)))
    assert len(t.hanging_p) > 50


def test_operator_quadratic_closed_form(oct_s):
    """u = (x^2 + y z, x y, z^2 - x z), mu = 1: -div(2 eps(u)) = -(lap u + grad div u)
    = -((2, 0, 0) + (2, 1, -1) + ... ) computed below; compare C^T E C u with C^T int phi g."""
    p, t = oct_s
    S = adaptive.AdaptiveStokes(t, p, mu_leaf=np.ones(len(t.leaves)))
    X = lattice_coords(t, t.u_keys)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    u = np.concatenate([x * x + y * z, x * y, z * z - x * z])
    # lap u = (2, 0, 2); div u = 2x + x + 2z - x = 2x + 2z; grad div = (2, 0, 2)
    g = -(np.array([2.0, 0.0, 2.0]) + np.array([2.0, 0.0, 2.0]))
    Y = ((S.Cu @ u).reshape(-1, 81) @ S.Ahat.T) * (S.mu_leaf * S.h_leaf)[:, None]
    Au = S.Cu.T @ Y.ravel()
    from oracle import fe
    Fe = np.stack([fe.element_F(h, np.tile(g, (27, 1))) for h in S.h_leaf])
    rhs = S.Cu.T @ Fe.ravel()
    free = ~S.dirichlet
    assert np.max(np.abs(Au[free] - rhs[free])) < 1e-11 * np.max(np.abs(rhs[free]))


def test_prolongation_reproduces_quadratics(oct_s):
    p, t = oct_s
    S = adaptive.AdaptiveStokes(t, p, mu_leaf=np.ones(len(t.leaves)))
    q = lambda X: 1.0 + X[:, 0] - 2 * X[:, 1] * X[:, 2] + 3 * X[:, 0] ** 2 - X[:, 2] ** 2
    for l in range(t.coarsest + 1, t.lmax + 1):
        Xc = lattice_coords(t, t.level_keys[l - 1])
        Xf = lattice_coords(t, t.level_keys[l])
        uc = np.concatenate([q(Xc)] * 3)
        uf = S.lev[l]["P"] @ uc
        assert np.max(np.abs(uf - np.concatenate([q(Xf)] * 3))) < 1e-13


def test_uniform_octree_matches_uniform_oracle():
    prob = si.workload("cube8")
    leaves = {(3, i, j, k) for i in range(8) for j in range(8) for k in range(8)}
    t = octree.Octree(leaves, 1)
    assert not any(e.any() for e in t.level_edge)
    mesh = Mesh(8)
    mu = level_viscosities(mesh, prob, 3)
    S = adaptive.AdaptiveStokes(t, prob)
    assert np.allclose(S.mu_leaf, mu[-1], rtol=1e-14, atol=0)
    ops = Operators(mesh, mu[-1])
    rng = np.random.default_rng(2)
    x = rng.standard_normal(mesh.n_u)
    ya, yu = S.apply_A(x), ops.apply_A(x)
    assert np.linalg.norm(ya - yu) <= 1e-12 * np.linalg.norm(yu)
    G = gmg.GMG(8, 3, mu)
    va, vu = S.vcycle(x), G.vcycle(x)
    assert np.linalg.norm(va - vu) <= 1e-11 * np.linalg.norm(vu)


def test_dense_solve_oct_xs():
    p, t = build("oct_xs")
    S = adaptive.AdaptiveStokes(t, p)
    b = np.concatenate([S.F, np.zeros(S.n_p)])
    x, its, _ = krylov.fgmres(S.apply_stokes, S.precondition, b, rtol=1e-10, restart=50, max_it=400)
    A = S.csr_A()
    B = S.csr_B()
    # B^T with zero Dirichlet rows, pin pressure DoF 0, then normalise the mean
    K = sp.bmat([[A, sp.diags(S.free) @ B.T], [B, None]]).tolil()
    K[S.n_u, :] = 0.0
    K[S.n_u, S.n_u] = 1.0
    rhs = b.copy()
    rhs[S.n_u] = 0.0
    xd = np.linalg.solve(K.toarray(), rhs)
    w = S.pressure_weights()
    for v in (x, xd):
        v[S.n_u:] -= (w @ v[S.n_u:]) / w.sum()
    assert np.linalg.norm(x[:S.n_u] - xd[:S.n_u]) <= 1e-8 * np.linalg.norm(xd[:S.n_u])
    assert np.linalg.norm(x[S.n_u:] - xd[S.n_u:]) <= 1e-7 * np.linalg.norm(xd[S.n_u:])


def test_local_smoothing_constant_mu(oct_s):
    p, t = oct_s
    S = adaptive.AdaptiveStokes(t, p, mu_leaf=np.ones(len(t.leaves)))
    rng = np.random.default_rng(0)
    b = rng.standard_normal(S.n_u)
    b[S.dirichlet] = 0.0
    _, its, _ = krylov.fgmres(S.apply_A, S.vcycle, b, rtol=1e-8, restart=50, max_it=100)
    assert its <= 12


def _sym_defect(S, seed=4):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(S.n_u)
    y = rng.standard_normal(S.n_u)
    x[S.dirichlet] = 0.0
    y[S.dirichlet] = 0.0
    a, b = y @ S.vcycle(x), x @ S.vcycle(y)
    return abs(a - b) / abs(a)


def test_local_smoothing_vcycle_symmetric(oct_s):
    """The local-smoothing V-cycle with variable viscosity is a symmetric operator on the free
    velocity DoFs: the same Chebyshev polynomial before and after the coarse correction, the
    restriction the transpose of the prolongation (edge rows included), the copy to and from the
    levels transposes of each other, an exact coarse solve. This is what lets MINRES use it in
    P_D. A restriction that is not P^T, or a smoother that differs between the two sweeps, breaks
    the identity by many orders of magnitude (checked on planted mistakes in the oracle)."""
    p, t = oct_s
    S = adaptive.AdaptiveStokes(t, p)
    assert _sym_defect(S) < 1e-12
    # planted mistake: post-smoothing one degree lower than pre-smoothing
    smooth = S.smooth

    def uneven(l, b, x, zero_guess):
        if zero_guess:
            return smooth(l, b, x, zero_guess)
        S.degree -= 1
        try:
            return smooth(l, b, x, zero_guess)
        finally:
            S.degree += 1
    S.smooth = uneven
    assert _sym_defect(S) > 1e-6
