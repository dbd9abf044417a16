"""Finite-element building blocks, written from the definitions (Section 2.1).

Taylor-Hood [Q2]^3 x Q1 on axis-aligned cube cells. Reference cell [0,1]^3;
local Q2 node (i,j,k), i,j,k in {0,1,2}, sits at (i/2, j/2, k/2) and has local
index a = i + 3 j + 9 k. Local Q1 vertex (i,j,k) in {0,1}^3 has index i + 2 j + 4 k.
A velocity element DoF is (c, a) with component c in {0,1,2}, local index c*27 + a.

Quadrature: tensor 3-point Gauss-Legendre on [0,1] (points 1/2 -+ sqrt(15)/10
and 1/2, weights 5/18, 8/18, 5/18), the reading the paper leaves open; it
integrates polynomials of degree <= 5 per axis exactly, so the Q2 element
matrices with a cell-constant viscosity are exact.
"""
from __future__ import annotations

import itertools

import numpy as np


def gauss3():
    """3-point Gauss-Legendre points and weights on [0, 1]."""
    s = np.sqrt(15.0) / 10.0
    return np.array([0.5 - s, 0.5, 0.5 + s]), np.array([5.0, 8.0, 5.0]) / 18.0


Q2_NODES_1D = np.array([0.0, 0.5, 1.0])


def q2_1d(x):
    """Quadratic Lagrange basis on nodes {0, 1/2, 1}: values, shape (len(x), 3)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty(x.shape + (3,))
    for m in range(3):
        v = np.ones_like(x)
        for k in range(3):
            if k != m:
                v = v * (x - Q2_NODES_1D[k]) / (Q2_NODES_1D[m] - Q2_NODES_1D[k])
        out[..., m] = v
    return out


def q2_1d_deriv(x):
    """Derivatives of the quadratic Lagrange basis, shape (len(x), 3) (product rule)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape + (3,))
    for m in range(3):
        others = [k for k in range(3) if k != m]
        den = np.prod([Q2_NODES_1D[m] - Q2_NODES_1D[k] for k in others])
        for skip in others:
            term = np.ones_like(x)
            for k in others:
                if k != skip:
                    term = term * (x - Q2_NODES_1D[k])
            out[..., m] += term / den
    return out


def q1_1d(x):
    x = np.asarray(x, dtype=np.float64)
    return np.stack([1.0 - x, x], axis=-1)


def q2_3d_tables(points):
    """Q2 basis values (P, 27) and reference gradients (P, 27, 3) at reference points (P, 3)."""
    p = np.asarray(points, dtype=np.float64)
    v = [q2_1d(p[:, d]) for d in range(3)]
    g = [q2_1d_deriv(p[:, d]) for d in range(3)]
    P = p.shape[0]
    val = np.empty((P, 27))
    grad = np.empty((P, 27, 3))
    for k, j, i in itertools.product(range(3), range(3), range(3)):
        a = i + 3 * j + 9 * k
        val[:, a] = v[0][:, i] * v[1][:, j] * v[2][:, k]
        grad[:, a, 0] = g[0][:, i] * v[1][:, j] * v[2][:, k]
        grad[:, a, 1] = v[0][:, i] * g[1][:, j] * v[2][:, k]
        grad[:, a, 2] = v[0][:, i] * v[1][:, j] * g[2][:, k]
    return val, grad


def q1_3d_values(points):
    p = np.asarray(points, dtype=np.float64)
    v = [q1_1d(p[:, d]) for d in range(3)]
    out = np.empty((p.shape[0], 8))
    for k, j, i in itertools.product(range(2), range(2), range(2)):
        out[:, i + 2 * j + 4 * k] = v[0][:, i] * v[1][:, j] * v[2][:, k]
    return out


def quadrature_3d():
    """27 tensor Gauss points on [0,1]^3 (index q = qx + 3 qy + 9 qz) and weights."""
    g, w = gauss3()
    pts = np.empty((27, 3))
    wts = np.empty(27)
    for qz, qy, qx in itertools.product(range(3), range(3), range(3)):
        q = qx + 3 * qy + 9 * qz
        pts[q] = (g[qx], g[qy], g[qz])
        wts[q] = w[qx] * w[qy] * w[qz]
    return pts, wts


def strain_tensors(grad_phys):
    """eps(phi_a e_c) = 1/2 (e_c (x) grad phi_a + grad phi_a (x) e_c) for all 81 vector
    basis functions at every quadrature point: shape (Q, 81, 3, 3)."""
    Q = grad_phys.shape[0]
    eps = np.zeros((Q, 81, 3, 3))
    for c in range(3):
        for a in range(27):
            G = np.zeros((Q, 3, 3))
            G[:, c, :] = grad_phys[:, a, :]          # (grad u)_{c d} = d_d u_c
            eps[:, c * 27 + a] = 0.5 * (G + np.transpose(G, (0, 2, 1)))
    return eps


def element_A(h, mu_q):
    """A_e[i, j] = int_K 2 mu eps(phi_i) : eps(phi_j) dx on a cube cell of side h
    (Section 2.1, definition of A), by 27-point Gauss quadrature with the
    viscosity mu_q given at the quadrature points."""
    pts, w = quadrature_3d()
    _, grad = q2_3d_tables(pts)
    eps = strain_tensors(grad / h)
    jw = w * h ** 3 * 2.0 * np.asarray(mu_q, dtype=np.float64) * np.ones(27)
    return np.einsum("q,qiab,qjab->ij", jw, eps, eps)


def element_B(h):
    """B_e[l, (c,a)] = -int_K (div phi_(c,a)) psi_l dx (Section 2.1, definition of B)."""
    pts, w = quadrature_3d()
    _, grad = q2_3d_tables(pts)
    psi = q1_3d_values(pts)
    B = np.zeros((8, 81))
    for c in range(3):
        for a in range(27):
            div = grad[:, a, c] / h                 # div(phi_a e_c) = d_c phi_a
            B[:, c * 27 + a] = -np.einsum("q,q,ql->l", w * h ** 3, div, psi)
    return B


def element_Mp(h, inv_mu_q):
    """[M_p]_e[l, m] = int_K mu^-1 psi_l psi_m dx (Section 2.2.2)."""
    pts, w = quadrature_3d()
    psi = q1_3d_values(pts)
    jw = w * h ** 3 * np.asarray(inv_mu_q, dtype=np.float64) * np.ones(27)
    return np.einsum("q,ql,qm->lm", jw, psi, psi)


def element_F(h, f_q):
    """F_e[(c,a)] = int_K phi_(c,a) . f dx with f given at the quadrature points, shape (27, 3)."""
    pts, w = quadrature_3d()
    val, _ = q2_3d_tables(pts)
    F = np.zeros(81)
    for c in range(3):
        F[c * 27:(c + 1) * 27] = np.einsum("q,q,qa->a", w * h ** 3, f_q[:, c], val)
    return F
