"""Geometric multigrid V-cycle for the velocity block (Section 2.2.1).

One V-cycle with zero initial guess approximates A^-1. Per level: one
pre-smoothing and one post-smoothing step of a degree-4 Jacobi-Chebyshev
smoother (Section 2.2.1), residual, restriction to the next coarser level,
recursive coarse correction, prolongation. Level operators are the
rediscretised fully coupled operators with the level viscosity (Section 2.3);
the coarsest level is solved exactly (dense, FP64).

Readings of points the paper leaves open:
* degree k = k applications of D^-1 A in the error polynomial; the
  eigenvalue interval is [beta/15, beta] with beta = 1.2 lambda_max(D^-1 A),
  lambda_max from 12 Lanczos steps on D^-1/2 A D^-1/2 started from a seeded
  splitmix64 vector.
* prolongation is the Q2 embedding (a coarse Q2 field evaluated at the fine
  nodes), restriction its transpose; constrained entries are zero on every level.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import sinker_inputs

from . import fe
from .mesh import Mesh
from .operators import Operators


def prolongation_1d(nc):
    """Evaluate every coarse 1D Q2 basis function at every fine node (fine mesh
    2 nc cells). Fine node i_f sits at i_f / (4 nc); its coarse cell is
    min(i_f // 4, nc - 1) and its local coordinate (i_f - 4 cell) / 4."""
    nf = 2 * nc
    rows, cols, vals = [], [], []
    for i_f in range(2 * nf + 1):
        cell = min(i_f // 4, nc - 1)
        xi = (i_f - 4 * cell) / 4.0
        l = fe.q2_1d(np.array([xi]))[0]
        for m in range(3):
            if l[m] != 0.0:
                rows.append(i_f)
                cols.append(2 * cell + m)
                vals.append(l[m])
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nf + 1, 2 * nc + 1))


def prolongation(nc):
    """Velocity prolongation, level with nc cells per axis -> 2 nc: the tensor-product
    Q2 basis evaluated at the fine nodes (x fastest), one copy per component."""
    P1 = prolongation_1d(nc)
    P3 = sp.kron(P1, sp.kron(P1, P1)).tocsr()
    return sp.block_diag([P3, P3, P3]).tocsr()


def chebyshev_smooth(apply_A, Dinv, b, x, degree, lam_lo, lam_hi, zero_guess):
    """Jacobi-preconditioned Chebyshev iteration (Y. Saad, Iterative Methods for
    Sparse Linear Systems, 2nd ed., Alg. 12.1) on [lam_lo, lam_hi]: returns x after
    `degree` updates, so the error is multiplied by the scaled Chebyshev
    polynomial of degree `degree` in D^-1 A. With zero_guess the first residual
    is D^-1 b and no operator application is needed."""
    theta = 0.5 * (lam_hi + lam_lo)
    delta = 0.5 * (lam_hi - lam_lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    if zero_guess:
        r = Dinv * b
        x = np.zeros_like(b)
    else:
        r = Dinv * (b - apply_A(x))
    d = r / theta
    x = x + d
    for _ in range(degree - 1):
        r = Dinv * (b - apply_A(x))
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        x = x + d
        rho = rho_new
    return x


def lanczos_lambda_max(apply_A, Dinv, free_mask, seed, steps=12):
    """Largest Ritz value of D^-1/2 A D^-1/2 (restricted to free DoFs) after
    `steps` plain Lanczos steps from the splitmix64 start vector u01(seed) - 1/2
    (one value per DoF index, constrained entries zeroed)."""
    n = free_mask.shape[0]
    s = np.sqrt(Dinv) * free_mask
    v = (sinker_inputs.uniform01(seed, n) - 0.5) * free_mask
    v = v / np.linalg.norm(v)
    v_prev = np.zeros(n)
    beta_prev = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        w = s * apply_A(s * v) * free_mask
        alpha = w @ v
        w = w - alpha * v - beta_prev * v_prev
        beta = np.linalg.norm(w)
        alphas.append(alpha)
        if beta <= 1e-12 * abs(alpha):
            break
        betas.append(beta)
        v_prev, v = v, w / beta
        beta_prev = beta
    k = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    return float(np.linalg.eigvalsh(T)[-1])


class Level:
    def __init__(self, n, mu_cells, level_index, noslip_faces=0x3F):
        self.mesh = Mesh(n, noslip_faces)
        self.ops = Operators(self.mesh, mu_cells)
        self.free = (~self.mesh.dirichlet).astype(np.float64)
        d = self.ops.diag_A()
        self.Dinv = np.where(self.mesh.dirichlet, 0.0, 1.0 / d)
        self.index = level_index
        self.lam_max = None

    def A(self, x):
        """Level operator on vectors whose constrained entries are zero."""
        return self.ops.apply_A(x) * self.free


class GMG:
    """V-cycle hierarchy: levels[0] is the coarsest (n_coarse cells per axis)."""

    def __init__(self, n_finest, n_levels, mu_levels, degree=4, smoothing_range=15.0,
                 safety=1.2, lanczos_steps=12, noslip_faces=0x3F):
        self.degree = degree
        self.levels = []
        for l in range(n_levels):
            n = n_finest >> (n_levels - 1 - l)
            self.levels.append(Level(n, mu_levels[l], l, noslip_faces))
        self.P = [None] + [prolongation(self.levels[l - 1].mesh.n) for l in range(1, n_levels)]
        for lev in self.levels[1:]:
            lev.lam_max = lanczos_lambda_max(lev.A, lev.Dinv, lev.free,
                                             sinker_inputs.lanczos_seed(lev.index), lanczos_steps)
            lev.lam_hi = safety * lev.lam_max
            lev.lam_lo = lev.lam_hi / smoothing_range
        c = self.levels[0]
        Ad = c.ops.csr_A().toarray()
        fr = c.mesh.interior
        self.coarse_free = np.nonzero(fr)[0]
        self.coarse_matrix = Ad[np.ix_(fr, fr)]

    def coarse_solve(self, b):
        x = np.zeros_like(b)
        if self.coarse_free.size:
            x[self.coarse_free] = np.linalg.solve(self.coarse_matrix, b[self.coarse_free])
        return x

    def smooth(self, l, b, x, zero_guess):
        lev = self.levels[l]
        return chebyshev_smooth(lev.A, lev.Dinv, b, x, self.degree, lev.lam_lo, lev.lam_hi, zero_guess)

    def vcycle_level(self, l, b):
        """x ~ A_l^-1 b, zero initial guess; b has zero constrained entries."""
        if l == 0:
            return self.coarse_solve(b)
        lev = self.levels[l]
        x = self.smooth(l, b, None, True)
        r = (b - lev.A(x)) * lev.free
        bc = (self.P[l].T @ r) * self.levels[l - 1].free
        xc = self.vcycle_level(l - 1, bc)
        x = x + (self.P[l] @ xc) * lev.free
        x = self.smooth(l, b, x, False)
        return x

    def vcycle(self, b):
        """One V-cycle on the finest level; constrained rows act as the identity."""
        fin = self.levels[-1]
        x = self.vcycle_level(len(self.levels) - 1, b * fin.free)
        return np.where(fin.mesh.dirichlet, b, x)
