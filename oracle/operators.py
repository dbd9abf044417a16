"""Global operators of the Stokes block system (Section 2.1, eq. stokes_linear_system).

A = sum_K P_K^T A_K P_K with A_K the full-quadrature element matrix; with the
cell-constant (averaged) viscosity of Section 2.3 and cube cells, A_K =
mu_K * A_hat(h) by linearity of the integrand in mu. Likewise B, M_p and F.

Constraints (homogeneous Dirichlet on all walls): the constrained velocity
operator keeps the couplings among unconstrained DoFs and replaces every
constrained row and column by the identity. So for a vector x,
  (A_c x)_i = sum_{j free} A_ij x_j   (i free),   (A_c x)_i = x_i   (i constrained).
B drops constrained velocity columns; B^T has zero constrained rows.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fe
from .mesh import Mesh


class Operators:
    """Element-by-element application of the blocks on one uniform level."""

    def __init__(self, mesh: Mesh, mu_cells):
        self.mesh = mesh
        self.mu = np.asarray(mu_cells, dtype=np.float64)
        h = mesh.h
        self.Ahat = fe.element_A(h, 1.0)           # mu = 1 element matrix
        self.Bhat = fe.element_B(h)
        self.Mhat = fe.element_Mp(h, 1.0)

    # -- velocity block ---------------------------------------------------
    def apply_A(self, x):
        """y = A_c x (element by element)."""
        m = self.mesh
        xf = np.where(m.dirichlet, 0.0, x)
        X = xf[m.cell_dofs]
        Y = (X @ self.Ahat.T) * self.mu[:, None]
        y = np.bincount(m.cell_dofs.ravel(), weights=Y.ravel(), minlength=m.n_u)
        y[m.dirichlet] = x[m.dirichlet]
        return y

    def apply_A_unconstrained(self, x):
        """y = A x with no boundary constraints (the plain assembled operator)."""
        m = self.mesh
        Y = (x[m.cell_dofs] @ self.Ahat.T) * self.mu[:, None]
        return np.bincount(m.cell_dofs.ravel(), weights=Y.ravel(), minlength=m.n_u)

    def diag_A(self):
        """Diagonal of A_c: sum over cells of mu_K diag(A_hat); 1 on constrained DoFs."""
        m = self.mesh
        Y = self.mu[:, None] * np.diag(self.Ahat)[None, :]
        d = np.bincount(m.cell_dofs.ravel(), weights=Y.ravel(), minlength=m.n_u)
        d[m.dirichlet] = 1.0
        return d

    # -- pressure blocks --------------------------------------------------
    def apply_B(self, x):
        """(B x)_l = -int div(u_h) psi_l, constrained velocity entries treated as 0."""
        m = self.mesh
        xf = np.where(m.dirichlet, 0.0, x)
        Y = xf[m.cell_dofs] @ self.Bhat.T
        return np.bincount(m.cell_verts.ravel(), weights=Y.ravel(), minlength=m.n_p)

    def apply_BT(self, p):
        """(B^T p)_i = -int div(phi_i) p_h on free rows, 0 on constrained rows."""
        m = self.mesh
        Y = p[m.cell_verts] @ self.Bhat
        y = np.bincount(m.cell_dofs.ravel(), weights=Y.ravel(), minlength=m.n_u)
        y[m.dirichlet] = 0.0
        return y

    def apply_Mp(self, p):
        """M_p p with [M_p]_lm = int mu^-1 psi_l psi_m (Section 2.2.2), cell viscosity."""
        m = self.mesh
        Y = (p[m.cell_verts] @ self.Mhat.T) / self.mu[:, None]
        return np.bincount(m.cell_verts.ravel(), weights=Y.ravel(), minlength=m.n_p)

    def diag_Mp(self):
        m = self.mesh
        Y = np.diag(self.Mhat)[None, :] / self.mu[:, None]
        return np.bincount(m.cell_verts.ravel(), weights=Y.ravel(), minlength=m.n_p)

    # -- full Stokes operator ----------------------------------------------
    def apply_stokes(self, up):
        """[A_c B^T; B 0] [u; p] (eq. stokes_linear_system)."""
        n_u = self.mesh.n_u
        u, p = up[:n_u], up[n_u:]
        return np.concatenate([self.apply_A(u) + self.apply_BT(p), self.apply_B(u)])

    # -- assembled matrices (small meshes) ---------------------------------
    def csr_A(self):
        m = self.mesh
        rows = np.repeat(m.cell_dofs, 81, axis=1).ravel()
        cols = np.tile(m.cell_dofs, (1, 81)).ravel()
        vals = (self.mu[:, None, None] * self.Ahat[None]).ravel()
        A = sp.coo_matrix((vals, (rows, cols)), shape=(m.n_u, m.n_u)).tocsr()
        free = (~m.dirichlet).astype(np.float64)
        Dfree = sp.diags(free)
        return (Dfree @ A @ Dfree + sp.diags(m.dirichlet.astype(np.float64))).tocsr()

    def csr_B(self):
        m = self.mesh
        rows = np.repeat(m.cell_verts, 81, axis=1).ravel()
        cols = np.tile(m.cell_dofs, (1, 8)).ravel()
        vals = np.broadcast_to(self.Bhat[None], (m.n_cells, 8, 81)).ravel()
        B = sp.coo_matrix((vals, (rows, cols)), shape=(m.n_p, m.n_u)).tocsr()
        return (B @ sp.diags((~m.dirichlet).astype(np.float64))).tocsr()

    def pressure_weights(self):
        """int psi_l dx for every Q1 vertex (used for the zero-mean pressure)."""
        m = self.mesh
        pts, w = fe.quadrature_3d()
        psi = fe.q1_3d_values(pts)
        loc = (w * m.h ** 3) @ psi
        Y = np.broadcast_to(loc[None], (m.n_cells, 8))
        return np.bincount(m.cell_verts.ravel(), weights=Y.ravel(), minlength=m.n_p)


def apply_A_rows(n, mu_cells, x, dofs):
    """Selected rows of A_c x on an n^3 mesh, element by element, without the
    global cell tables (for sampled checks at sizes where those do not fit).
    dofs: velocity DoF indices (component-blocked numbering)."""
    M = 2 * n + 1
    nodes = M ** 3
    Ahat = fe.element_A(1.0 / n, 1.0)
    dofs = np.asarray(dofs, dtype=np.int64)
    out = np.zeros(dofs.size)
    for t, dof in enumerate(dofs):
        c, node = divmod(int(dof), nodes)
        g = (node % M, (node // M) % M, node // (M * M))
        if min(g) == 0 or max(g) == M - 1:
            out[t] = x[dof]
            continue
        acc = 0.0
        axes = []
        for gi in g:     # (cell index, local index) along each axis
            axes.append([((gi - 1) // 2, 1)] if gi % 2 else
                        [(ci, li) for ci, li in ((gi // 2 - 1, 2), (gi // 2, 0)) if 0 <= ci < n])
        for cz, lz in axes[2]:
            for cy, ly in axes[1]:
                for cx, lx in axes[0]:
                    cell = cx + n * cy + n * n * cz
                    local = np.array([(2 * cx + i) + M * (2 * cy + j) + M * M * (2 * cz + k)
                                      for k in range(3) for j in range(3) for i in range(3)])
                    ldofs = np.concatenate([local + comp * nodes for comp in range(3)])
                    xb = x[ldofs].copy()
                    lg = np.stack([local % M, (local // M) % M, local // (M * M)], 1)
                    bnd = np.any((lg == 0) | (lg == M - 1), axis=1)
                    xb[np.concatenate([bnd] * 3)] = 0.0
                    row = c * 27 + lx + 3 * ly + 9 * lz
                    acc += mu_cells[cell] * (Ahat[row] @ xb)
        out[t] = acc
    return out


def assemble_rhs(mesh: Mesh, f_at_quad):
    """F_(c,node) = int phi . f dx with f sampled at each cell's Gauss points,
    shape (cells, 27, 3); constrained entries zero (Section 2.1, definition of F)."""
    pts, w = fe.quadrature_3d()
    val, _ = fe.q2_3d_tables(pts)
    h3w = w * mesh.h ** 3
    Fe = np.concatenate([np.einsum("q,cq,qa->ca", h3w, f_at_quad[:, :, c], val) for c in range(3)], axis=1)
    F = np.bincount(mesh.cell_dofs.ravel(), weights=Fe.ravel(), minlength=mesh.n_u)
    F[mesh.dirichlet] = 0.0
    return F
