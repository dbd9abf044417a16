"""Stokes operators and local-smoothing GMG on an adaptive octree (Abstract; Sections 2.1,
2.2, 2.3; local smoothing by citation of Janssen & Kanschat, Section 2.2.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Active system. Every leaf K of side h_K contributes its full-quadrature element matrices
(fe.py; with the cell-constant viscosity of Section 2.3, A_K = mu_K h_K A_hat, B_K =
h_K^2 B_hat, [M_p]_K = h_K^3 / mu_K M_hat, for the unit-cube matrices A_hat, B_hat,
M_hat). The global matrices are C^T E C with E block-diagonal over leaves and C mapping
active node values to the leaves' local nodes, hanging nodes through their constraint
weights. Dirichlet rows and columns of A are replaced by the identity, B drops Dirichlet
velocity columns and B^T has zero Dirichlet rows, as on the uniform mesh.

Local smoothing (parity unpinned beyond "oracle = the same algorithm": the paper cites the
method; pinned by equality with the uniform GMG on a uniform octree, by the symmetry of the
V-cycle with variable viscosity, and by a handful of iterations for constant viscosity). Level l holds all cells of level l; its operator A_l is assembled from them with
the level viscosity (a leaf's harmonic average, a refined cell's mean over its children)
and identity rows on the cube boundary, edge nodes kept as ordinary rows and columns.
Smoothing touches only nodes that are neither on the cube boundary nor on the refinement
edge (Jacobi-Chebyshev with D^-1 = 0 there). One V-cycle for an active right-hand side b:
  * copy: level l receives b at the active nodes whose coarsest leaf is of level l;
  * down, level l > coarsest: x = S_l(b_l, 0); t = b_l - A_l x (edge rows included);
    b_{l-1} += P_l^T t;
  * coarsest level: x = A_c^-1 b_c on its free nodes (the coarsest level covers the cube);
  * up: x += P_l x_{l-1} (every node, edge nodes included); x = S_l(b_l, x), whose residual
    b_l - A_l x uses the edge values, which the smoother leaves unchanged;
  * the active result takes each node's value on its level.
P_l is the Q2 embedding of a level-(l-1) field into the level-l cells (each level-l cell's
parent is a level-(l-1) cell).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import sinker_inputs

from . import fe
from .gmg import chebyshev_smooth, lanczos_lambda_max
from .octree import Octree
from .sinker import forcing, harmonic_cell_average, viscosity


def leaf_quad_points(tree: Octree):
    pts, _ = fe.quadrature_3d()
    out = np.empty((len(tree.leaves), 27, 3))
    for n, (l, i, j, k) in enumerate(tree.leaves):
        h = 2.0 ** (-l)
        out[n] = np.array([i * h, j * h, k * h]) + h * pts
    return out


def level_viscosities(tree: Octree, mu_leaf):
    """Viscosity of every cell of every level: leaves keep their harmonic average, a refined
    cell takes the arithmetic mean of its 8 children (Section 2.3)."""
    mu = {c: m for c, m in zip(tree.leaves, mu_leaf)}
    for l in range(tree.lmax, -1, -1):
        for c in tree.level_cells[l]:
            if c not in mu:
                _, i, j, k = c
                ch = [(l + 1, 2 * i + a, 2 * j + b, 2 * k + cc) for cc in (0, 1) for b in (0, 1) for a in (0, 1)]
                mu[c] = sum(mu[x] for x in ch) / 8.0
    return [np.array([mu[c] for c in tree.level_cells[l]]) for l in range(tree.lmax + 1)]


def constraint_matrix(rows_per_leaf, n_cols, per_leaf):
    """Sparse C with C[(leaf, a), col] = weight from rows_per_leaf[leaf][a] = [(col, w), ...]."""
    r, c, v = [], [], []
    for n, row in enumerate(rows_per_leaf):
        for a, terms in enumerate(row):
            for col, w in terms:
                r.append(n * per_leaf + a)
                c.append(col)
                v.append(w)
    return sp.csr_matrix((v, (r, c)), shape=(len(rows_per_leaf) * per_leaf, n_cols))


def velocity_expand(C1):
    """Component-blocked velocity: local DoF (c, a) -> c * 27 + a, global (c, node)."""
    n_b, n_a = C1.shape
    n_leaf = n_b // 27
    # rows: leaf * 81 + c * 27 + a ; cols: c * n_a + node
    C1 = C1.tocoo()
    leaf, a = np.divmod(C1.row, 27)
    rows = np.concatenate([leaf * 81 + c * 27 + a for c in range(3)])
    cols = np.concatenate([C1.col + c * n_a for c in range(3)])
    vals = np.concatenate([C1.data] * 3)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_leaf * 81, 3 * n_a))


class AdaptiveStokes:
    """Active operators, right-hand side and local-smoothing V-cycle of an octree problem."""

    def __init__(self, tree: Octree, prob, degree=4, smoothing_range=15.0, safety=1.2, lanczos_steps=12,
                 mu_leaf=None):
        self.tree = tree
        self.prob = prob
        self.degree = degree
        qp = leaf_quad_points(tree)
        if mu_leaf is None:
            mu_leaf = np.array([harmonic_cell_average(m) for m in viscosity(qp, prob)])
        self.mu_leaf = np.asarray(mu_leaf, dtype=np.float64)
        self.h_leaf = np.array([2.0 ** (-c[0]) for c in tree.leaves])
        self.Ahat = fe.element_A(1.0, 1.0)
        self.Bhat = fe.element_B(1.0)
        self.Mhat = fe.element_Mp(1.0, 1.0)
        self.Cu = velocity_expand(constraint_matrix(tree.leaf_u, tree.n_nodes, 27))
        self.Cp = constraint_matrix(tree.leaf_p, tree.n_p, 8)
        self.dirichlet = np.concatenate([tree.u_boundary] * 3)
        self.free = (~self.dirichlet).astype(np.float64)
        self.n_u = tree.n_u
        self.n_p = tree.n_p
        # right-hand side F = C^T (int phi f) per leaf
        pts, w = fe.quadrature_3d()
        val, _ = fe.q2_3d_tables(pts)
        f = forcing(qp, prob)                                            # (leaves, 27, 3)
        Fe = np.zeros((len(tree.leaves), 81))
        for c in range(3):
            Fe[:, c * 27:(c + 1) * 27] = np.einsum("n,q,nq,qa->na", self.h_leaf ** 3, w, f[:, :, c], val)
        F = self.Cu.T @ Fe.ravel()
        F[self.dirichlet] = 0.0
        self.F = F
        self.Mp_diag = self._mp_diag()
        self._setup_levels(smoothing_range, safety, lanczos_steps)

    # -- active operators -----------------------------------------------------
    def apply_A(self, x):
        xf = np.where(self.dirichlet, 0.0, x)
        X = (self.Cu @ xf).reshape(-1, 81)
        Y = (X @ self.Ahat.T) * (self.mu_leaf * self.h_leaf)[:, None]
        y = self.Cu.T @ Y.ravel()
        y[self.dirichlet] = x[self.dirichlet]
        return y

    def apply_B(self, x):
        xf = np.where(self.dirichlet, 0.0, x)
        X = (self.Cu @ xf).reshape(-1, 81)
        Y = (X @ self.Bhat.T) * (self.h_leaf ** 2)[:, None]
        return self.Cp.T @ Y.ravel()

    def apply_BT(self, p):
        P = (self.Cp @ p).reshape(-1, 8)
        Y = (P @ self.Bhat) * (self.h_leaf ** 2)[:, None]
        y = self.Cu.T @ Y.ravel()
        y[self.dirichlet] = 0.0
        return y

    def apply_Mp(self, p):
        P = (self.Cp @ p).reshape(-1, 8)
        Y = (P @ self.Mhat.T) * (self.h_leaf ** 3 / self.mu_leaf)[:, None]
        return self.Cp.T @ Y.ravel()

    def _mp_diag(self):
        """diag(C_p^T E_M C_p): sum over leaves and local pairs of C_la M_lm C_ma."""
        Cp = self.Cp.tocsr()
        d = np.zeros(self.n_p)
        scale = self.h_leaf ** 3 / self.mu_leaf
        for n in range(len(self.tree.leaves)):
            blk = Cp[n * 8:(n + 1) * 8].toarray()            # (8, n_p)
            cols = np.nonzero(np.any(blk != 0, axis=0))[0]
            b = blk[:, cols]
            d[cols] += scale[n] * np.einsum("la,lm,ma->a", b, self.Mhat, b)
        return d

    def apply_stokes(self, up):
        u, p = up[:self.n_u], up[self.n_u:]
        return np.concatenate([self.apply_A(u) + self.apply_BT(p), self.apply_B(u)])

    def pressure_weights(self):
        pts, w = fe.quadrature_3d()
        psi = fe.q1_3d_values(pts)
        loc = w @ psi
        Y = (self.h_leaf ** 3)[:, None] * loc[None, :]
        return self.Cp.T @ Y.ravel()

    def csr_A(self):
        E = sp.block_diag([sp.csr_matrix(self.Ahat * (m * h)) for m, h in zip(self.mu_leaf, self.h_leaf)], format="csr")
        A = (self.Cu.T @ E @ self.Cu).tocsr()
        Df = sp.diags(self.free)
        return (Df @ A @ Df + sp.diags(self.dirichlet.astype(np.float64))).tocsr()

    def csr_B(self):
        E = sp.block_diag([sp.csr_matrix(self.Bhat * h * h) for h in self.h_leaf], format="csr")
        return (self.Cp.T @ E @ self.Cu @ sp.diags(self.free)).tocsr()

    # -- level hierarchy ------------------------------------------------------
    def _setup_levels(self, smoothing_range, safety, lanczos_steps):
        t = self.tree
        self.mu_levels = level_viscosities(t, self.mu_leaf)
        self.lev = []
        for l in range(t.lmax + 1):
            cn = t.level_cell_nodes[l]
            nn = len(t.level_keys[l])
            bnd = np.concatenate([t.level_boundary[l]] * 3)
            edge = np.concatenate([t.level_edge[l]] * 3)
            dofs = np.concatenate([cn + c * nn for c in range(3)], axis=1)
            scale = self.mu_levels[l] * 2.0 ** (-l)
            d = np.bincount(dofs.ravel(), weights=(scale[:, None] * np.diag(self.Ahat)[None, :]).ravel(),
                            minlength=3 * nn)
            smooth_mask = ~(bnd | edge)
            Dinv = np.where(smooth_mask, 1.0 / np.where(smooth_mask, d, 1.0), 0.0)
            self.lev.append(dict(l=l, nn=nn, dofs=dofs, scale=scale, bnd=bnd, edge=edge,
                                 free=smooth_mask.astype(np.float64), Dinv=Dinv))
        for l in range(t.coarsest + 1, t.lmax + 1):
            self.lev[l]["P"] = self._prolongation(l)
        for l in range(t.coarsest + 1, t.lmax + 1):
            L = self.lev[l]
            lam = lanczos_lambda_max(lambda x, l=l: self.level_A(l, x), L["Dinv"], L["free"],
                                     sinker_inputs.lanczos_seed(l - t.coarsest), lanczos_steps)
            L["lam_hi"] = safety * lam
            L["lam_lo"] = L["lam_hi"] / smoothing_range
        c = t.coarsest
        Lc = self.lev[c]
        n = 3 * Lc["nn"]
        Ad = np.column_stack([self.level_A(c, e) for e in np.eye(n)])
        fr = np.nonzero(~Lc["bnd"])[0]
        self.coarse_free = fr
        self.coarse_matrix = Ad[np.ix_(fr, fr)]

    def level_A(self, l, x):
        """A_l x: level-l cells, identity rows on the cube boundary, boundary inputs ignored;
        edge nodes are ordinary rows and columns."""
        L = self.lev[l]
        xf = np.where(L["bnd"], 0.0, x)
        Y = (xf[L["dofs"]] @ self.Ahat.T) * L["scale"][:, None]
        y = np.bincount(L["dofs"].ravel(), weights=Y.ravel(), minlength=3 * L["nn"])
        y[L["bnd"]] = x[L["bnd"]]
        return y

    def _prolongation(self, l):
        """P_l (level l-1 -> level l), one component, from each level-l node's first cell's
        parent: the parent's Q2 basis at the node (tensor products of (1,0,0), (3/8,3/4,-1/8),
        (0,1,0), (-1/8,3/4,3/8), (0,0,1))."""
        t = self.tree
        cells = t.level_cells[l]
        parents = {c: n for n, c in enumerate(t.level_cells[l - 1])}
        cn_c = t.level_cell_nodes[l - 1]
        nn = len(t.level_keys[l])
        seen = np.zeros(nn, dtype=bool)
        r, cidx, v = [], [], []
        for n, c in enumerate(cells):
            par = (l - 1, c[1] >> 1, c[2] >> 1, c[3] >> 1)
            pn = parents[par]
            off = (c[1] & 1, c[2] & 1, c[3] & 1)
            for a in range(27):
                node = t.level_cell_nodes[l][n][a]
                if seen[node]:
                    continue
                seen[node] = True
                loc = (a % 3, (a // 3) % 3, a // 9)
                xi = [(2 * o + x) / 4.0 for o, x in zip(off, loc)]      # position in the parent
                w1 = [fe.q2_1d(np.array([x]))[0] for x in xi]
                for b in range(27):
                    w = w1[0][b % 3] * w1[1][(b // 3) % 3] * w1[2][b // 9]
                    if w != 0.0:
                        r.append(node)
                        cidx.append(cn_c[pn][b])
                        v.append(w)
        P1 = sp.csr_matrix((v, (r, cidx)), shape=(nn, len(t.level_keys[l - 1])))
        return sp.block_diag([P1] * 3, format="csr")

    def smooth(self, l, b, x, zero_guess):
        L = self.lev[l]
        return chebyshev_smooth(lambda y: self.level_A(l, y), L["Dinv"], b, x, self.degree,
                                L["lam_lo"], L["lam_hi"], zero_guess)

    def coarse_solve(self, b):
        x = np.zeros_like(b)
        x[self.coarse_free] = np.linalg.solve(self.coarse_matrix, b[self.coarse_free])
        return x

    def copy_to_levels(self, b_active):
        t = self.tree
        bl = [np.zeros(3 * L["nn"]) for L in self.lev]
        for c in range(3):
            vals = b_active[c * t.n_nodes:(c + 1) * t.n_nodes]
            for l in range(t.coarsest, t.lmax + 1):
                m = t.copy_level == l
                bl[l][c * self.lev[l]["nn"] + t.copy_index[m]] = vals[m]
        for l in range(len(bl)):
            bl[l][self.lev[l]["bnd"]] = 0.0
        return bl

    def copy_from_levels(self, xl):
        t = self.tree
        out = np.zeros(self.n_u)
        for c in range(3):
            for l in range(t.coarsest, t.lmax + 1):
                m = np.nonzero(t.copy_level == l)[0]
                out[c * t.n_nodes + m] = xl[l][c * self.lev[l]["nn"] + t.copy_index[m]]
        return out

    def vcycle(self, b_active):
        """One local-smoothing V-cycle; Dirichlet rows act as the identity."""
        t = self.tree
        bl = self.copy_to_levels(b_active)
        xl = [None] * len(self.lev)

        def level(l):
            L = self.lev[l]
            if l == t.coarsest:
                xl[l] = self.coarse_solve(bl[l])
                return
            x = self.smooth(l, bl[l], None, True)
            r = bl[l] - self.level_A(l, x)
            r[L["bnd"]] = 0.0
            bl[l - 1] = bl[l - 1] + L["P"].T @ r
            bl[l - 1][self.lev[l - 1]["bnd"]] = 0.0
            level(l - 1)
            x = x + L["P"] @ xl[l - 1]
            x[L["bnd"]] = 0.0
            xl[l] = self.smooth(l, bl[l], x, False)

        level(t.lmax)
        x = self.copy_from_levels(xl)
        return np.where(self.dirichlet, b_active, x)

    def schur_inverse(self, r_p, degree=5):
        if degree == 0:                         # S_hat = diag(M_p)
            return r_p / self.Mp_diag
        return chebyshev_smooth(self.apply_Mp, 1.0 / self.Mp_diag, r_p, None, degree, 1.0 / 8.0, 27.0 / 8.0, True)

    def precondition(self, r):
        r_u, r_p = r[:self.n_u], r[self.n_u:]
        z_p = -self.schur_inverse(r_p)
        z_u = self.vcycle(r_u - self.apply_BT(z_p))
        return np.concatenate([z_u, z_p])
