"""Pins of the oracle's no-normal-flux walls (the extension the paper names in Section 2: u . n = 0
and zero tangential traction; `Mesh(n, noslip_faces)`, bit f of face f = 2 axis + side set =
no-slip):

* constraint masks: on a no-normal-flux face only the normal component is constrained;
* manufactured solution with every wall no-normal-flux, u = (A sx cy cz, B cx sy cz, C cx cy sz)
  (s = sin(pi .), c = cos(pi .), A + B + C = 0: divergence-free, u . n = 0 and every tangential
  strain component zero on the walls, so the traction condition holds for any viscosity),
  p = cx cy cz: velocity L2 error O(h^3), pressure O(h^2);
* the constant pressure stays the only null vector (B^T 1 = 0 on free rows), and the velocity
  block has none (no rigid motion keeps u . n = 0 on a cube);
* FGMRES with the GMG block preconditioner on the same walls reaches the dense direct solution.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import sinker_inputs as si
from oracle import fe, gmg, krylov, mesh, operators, sinker


def test_masks():
    n = 3
    M = 2 * n + 1
    free_all = mesh.Mesh(n, 0)
    assert free_all.dirichlet.sum() == 3 * 2 * M * M
    m = mesh.Mesh(n, 0b110011)          # no-slip on x and z faces, no-normal-flux on y faces
    nodes = m.n_nodes
    idx = np.arange(M)
    I, J, K = [a.transpose(2, 1, 0).ravel() for a in np.meshgrid(idx, idx, idx, indexing="ij")]
    xz = (I == 0) | (I == M - 1) | (K == 0) | (K == M - 1)
    yf = (J == 0) | (J == M - 1)
    for c in range(3):
        expect = xz | yf if c == 1 else xz
        assert np.array_equal(m.dirichlet[c * nodes:(c + 1) * nodes], expect)
    assert np.array_equal(mesh.Mesh(n).dirichlet, mesh.Mesh(n, 0x3F).dirichlet)


def _manufactured(n, a=(1.0, -2.0, 1.0)):
    pi = np.pi
    m = mesh.Mesh(n, 0)
    ops = operators.Operators(m, np.ones(m.n_cells))
    q = m.quad_points()
    x, y, z = q[..., 0], q[..., 1], q[..., 2]
    sx, sy, sz, cx, cy, cz = (np.sin(pi * x), np.sin(pi * y), np.sin(pi * z),
                              np.cos(pi * x), np.cos(pi * y), np.cos(pi * z))
    u = [a[0] * sx * cy * cz, a[1] * cx * sy * cz, a[2] * cx * cy * sz]
    gp = [-pi * sx * cy * cz, -pi * cx * sy * cz, -pi * cx * cy * sz]      # grad p, p = cx cy cz
    fq = np.stack([3 * pi * pi * u[c] + gp[c] for c in range(3)], -1)      # -lap u + grad p, div u = 0
    F = operators.assemble_rhs(m, fq)
    A, B = ops.csr_A(), ops.csr_B()
    w = sp.csr_matrix(ops.pressure_weights()[None, :])
    K = sp.bmat([[A, B.T, None], [B, None, w.T], [None, w, None]]).tocsc()
    sol = sla.spsolve(K, np.concatenate([F, np.zeros(m.n_p + 1)]))
    uh, ph = sol[:m.n_u], sol[m.n_u:m.n_u + m.n_p]
    pts, wq = fe.quadrature_3d()
    val, _ = fe.q2_3d_tables(pts)
    e2 = sum(np.sum((uh[m.cell_dofs[:, c * 27:(c + 1) * 27]] @ val.T - u[c]) ** 2 * wq[None, :]) * m.h ** 3
             for c in range(3))
    pq = ph[m.cell_verts] @ fe.q1_3d_values(pts).T
    ep2 = np.sum((pq - cx * cy * cz) ** 2 * wq[None, :]) * m.h ** 3
    return np.sqrt(e2), np.sqrt(ep2)


def test_manufactured_solution_no_normal_flux():
    errs = [_manufactured(n) for n in (2, 4, 8)]
    eu = [e[0] for e in errs]
    ep = [e[1] for e in errs]
    assert np.log2(eu[-2] / eu[-1]) > 2.6, eu
    assert np.log2(ep[-2] / ep[-1]) > 1.6, ep


def test_null_spaces_no_normal_flux():
    m = mesh.Mesh(2, 0)
    ops = operators.Operators(m, np.ones(m.n_cells))
    B = ops.csr_B().toarray()
    free = ~m.dirichlet
    assert np.abs(B[:, free].T @ np.ones(m.n_p)).max() < 1e-13       # constant pressure
    A = ops.csr_A().toarray()[np.ix_(free, free)]
    assert np.linalg.eigvalsh(A).min() > 1e-8                         # no velocity null vector


def test_gmg_fgmres_no_normal_flux_matches_dense():
    p = si.workload("cube4")
    walls = 0b001100                                                   # no-slip only on the y faces
    m = mesh.Mesh(p.n, walls)
    mus = sinker.level_viscosities(m, p, p.n_levels)
    G = gmg.GMG(p.n, p.n_levels, mus, noslip_faces=walls)
    ops = G.levels[-1].ops
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    b = np.concatenate([F, np.zeros(m.n_p)])
    x, its, _ = krylov.fgmres(ops.apply_stokes, krylov.StokesPreconditioner(ops, G).apply, b, rtol=1e-11)
    x = krylov.zero_mean_pressure(ops, x)
    A, B = ops.csr_A(), ops.csr_B()
    w = sp.csr_matrix(ops.pressure_weights()[None, :])
    K = sp.bmat([[A, B.T, None], [B, None, w.T], [None, w, None]]).tocsc()
    xd = sla.spsolve(K, np.concatenate([b, [0.0]]))[:m.n_u + m.n_p]
    assert np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max()
    assert its < 60
    assert np.abs(x[:m.n_u][m.dirichlet]).max() == 0.0
