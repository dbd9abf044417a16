"""Sinker benchmark coefficients (Section 3.2) and viscosity averaging (Section 2.3)."""
from __future__ import annotations

import numpy as np

from .fe import quadrature_3d


def indicator(x, centres, delta, omega):
    """X(x) = prod_i [1 - exp(-delta max(0, |c_i - x| - omega/2)^2)] (Section 3.2)."""
    x = np.asarray(x, dtype=np.float64)
    X = np.ones(x.shape[:-1])
    for c in np.asarray(centres, dtype=np.float64):
        dist = np.sqrt(np.sum((x - c) ** 2, axis=-1))
        X = X * (1.0 - np.exp(-delta * np.maximum(0.0, dist - omega / 2.0) ** 2))
    return X


def viscosity(x, prob):
    """mu(x) = X(x) mu_min + (1 - X(x)) mu_max (Section 3.2)."""
    X = indicator(x, prob.centres, prob.delta, prob.omega)
    return X * prob.mu_min + (1.0 - X) * prob.mu_max


def forcing(x, prob):
    """f(x) = (0, 0, beta (X(x) - 1)) (Section 3.2). Shape (..., 3)."""
    X = indicator(x, prob.centres, prob.delta, prob.omega)
    f = np.zeros(X.shape + (3,))
    f[..., 2] = prob.beta * (X - 1.0)
    return f


def harmonic_cell_average(mu_q):
    """Cell viscosity from its quadrature-point values (Section 2.3): the
    quadrature-weighted harmonic mean (sum_q w_q) / (sum_q w_q / mu_q)."""
    _, w = quadrature_3d()
    mu_q = np.asarray(mu_q, dtype=np.float64)
    return w.sum() / ((1.0 / mu_q) @ w)


def restrict_cell_viscosity(mu_fine, n_fine):
    """Parent viscosity = arithmetic mean of its 8 children (Section 2.3, Q0 restriction)."""
    nc = n_fine // 2
    m = np.asarray(mu_fine).reshape(n_fine, n_fine, n_fine)      # [ck, cj, ci]
    parent = m.reshape(nc, 2, nc, 2, nc, 2).mean(axis=(1, 3, 5))
    return parent.ravel()


def level_viscosities(mesh_finest, prob, n_levels):
    """Cell viscosity on every level, coarsest first (Section 2.3)."""
    mu_q = viscosity(mesh_finest.quad_points(), prob)
    mu = harmonic_cell_average(mu_q)
    levels = [mu]
    n = mesh_finest.n
    for _ in range(n_levels - 1):
        mu = restrict_cell_viscosity(mu, n)
        n //= 2
        levels.append(mu)
    return levels[::-1]
