"""Uniform hexahedral mesh of the unit cube and its DoF numbering (Section 2.1).

n cells per axis, h = 1/n. Q2 nodes form a (2n+1)^3 lattice of spacing h/2;
node (i,j,k) has index i + M j + M^2 k with M = 2n+1. Velocity vectors are
component-blocked: DoF (c, node) has index c M^3 + node, so N_u = 3 M^3
(boundary nodes included). Q1 pressure vertices form an (n+1)^3 lattice,
vertex (i,j,k) -> i + (n+1) j + (n+1)^2 k. Cell (ci,cj,ck) -> ci + n cj + n^2 ck.

Homogeneous Dirichlet data on all six walls (eq. stokes): every velocity DoF on
a boundary node is constrained. The walls can instead carry the no-normal-flux
condition the paper names as an extension (Section 2: u . n = 0 with zero
tangential traction, the latter natural in the weak form): face f = 2 axis + side
(side 0 at coordinate 0, side 1 at 1) is no-slip if bit f of `noslip_faces` is
set, else only the velocity component along its normal is constrained there.
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, n: int, noslip_faces: int = 0x3F):
        self.n = n
        self.noslip_faces = noslip_faces
        self.h = 1.0 / n
        self.M = 2 * n + 1
        self.n_nodes = self.M ** 3
        self.n_u = 3 * self.n_nodes
        self.n_p = (n + 1) ** 3
        self.n_cells = n ** 3
        ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        # cell index = ci + n cj + n^2 ck; order the arrays by that index
        ci = ci.transpose(2, 1, 0).ravel()
        cj = cj.transpose(2, 1, 0).ravel()
        ck = ck.transpose(2, 1, 0).ravel()
        self.cell_ijk = np.stack([ci, cj, ck], axis=1)
        M = self.M
        nodes = np.empty((self.n_cells, 27), dtype=np.int64)
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    nodes[:, i + 3 * j + 9 * k] = (2 * ci + i) + M * (2 * cj + j) + M * M * (2 * ck + k)
        self.cell_nodes = nodes
        self.cell_dofs = np.concatenate([nodes + c * self.n_nodes for c in range(3)], axis=1)
        P = n + 1
        verts = np.empty((self.n_cells, 8), dtype=np.int64)
        for k in range(2):
            for j in range(2):
                for i in range(2):
                    verts[:, i + 2 * j + 4 * k] = (ci + i) + P * (cj + j) + P * P * (ck + k)
        self.cell_verts = verts
        idx = np.arange(M)
        I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
        on_b = (I == 0) | (I == M - 1) | (J == 0) | (J == M - 1) | (K == 0) | (K == M - 1)
        self.boundary_node = on_b.transpose(2, 1, 0).ravel()
        face = []                                   # node masks of faces 0..5, node order
        for A in (I, J, K):
            face.append((A == 0).transpose(2, 1, 0).ravel())
            face.append((A == M - 1).transpose(2, 1, 0).ravel())
        comp = []
        for c in range(3):
            m = np.zeros(self.n_nodes, dtype=bool)
            for f in range(6):
                if (noslip_faces >> f) & 1 or f // 2 == c:
                    m |= face[f]
            comp.append(m)
        self.dirichlet = np.concatenate(comp)
        self.interior = ~self.dirichlet

    def node_coords(self):
        """Physical coordinates of all Q2 nodes, shape (M^3, 3), node order."""
        idx = np.arange(self.M) * (self.h / 2)
        X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij")
        return np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                         Z.transpose(2, 1, 0).ravel()], axis=1)

    def vertex_coords(self):
        idx = np.arange(self.n + 1) * self.h
        X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij")
        return np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                         Z.transpose(2, 1, 0).ravel()], axis=1)

    def cell_origins(self):
        return self.cell_ijk * self.h

    def quad_points(self):
        """Physical coordinates of the 27 Gauss points of every cell, shape (cells, 27, 3)."""
        from .fe import quadrature_3d
        pts, _ = quadrature_3d()
        return self.cell_origins()[:, None, :] + self.h * pts[None, :, :]
