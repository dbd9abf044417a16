"""Pins of the gradient-indicator refinement oracle (oracle/refine.py, Section 3.3 reading):

* for a velocity field that is quadratic in each coordinate (which the Q2 space and its hanging-
  node constraints reproduce exactly), the indicator equals h^(5/2) |grad u(x_K)|_F computed from
  the closed-form gradient at every leaf away from the walls: this fixes the face-centre node
  pairs, their signs and axes, and the power of h;
* marking splits exactly floor(n/7 + 1/2) leaves, those with the largest indicator, and the
  result is 2:1 balanced with every split leaf gone from the leaf set.
"""
from __future__ import annotations

import numpy as np
import pytest

import sinker_inputs as si
from oracle import adaptive, octree, refine


@pytest.fixture(scope="module")
def oct_s():
    p = si.octree_workload("oct_s")
    lv = octree.balance(octree.refine_shells(p.base_level, p.centres, p.max_levels, p.shell_radius,
                                             p.shell_half_width))
    t = octree.Octree(lv, p.coarsest_level)
    return p, t, adaptive.AdaptiveStokes(t, p, mu_leaf=np.ones(len(t.leaves)))


def quad_field(coef, X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    basis = np.stack([np.ones_like(x), x, y, z, x * x, y * y, z * z, x * y, y * z, x * z], -1)
    return basis @ coef.T                                        # (points, 3)


def quad_grad(coef, X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    o, zr = np.ones_like(x), np.zeros_like(x)
    dx = np.stack([zr, o, zr, zr, 2 * x, zr, zr, y, zr, z], -1) @ coef.T
    dy = np.stack([zr, zr, o, zr, zr, 2 * y, zr, x, z, zr], -1) @ coef.T
    dz = np.stack([zr, zr, zr, o, zr, zr, 2 * z, zr, y, x], -1) @ coef.T
    return np.stack([dx, dy, dz], -1)                            # (points, 3 components, 3 axes)


def test_indicator_exact_for_quadratic_fields(oct_s):
    p, t, S = oct_s
    rng = np.random.default_rng(21)
    coef = rng.standard_normal((3, 10))
    X = np.array([t._point(int(k)) for k in t.u_keys], dtype=np.float64) / (t.Mx - 1)
    u = quad_field(coef, X).T.ravel()                            # component-blocked
    eta = refine.gradient_indicator(S, u)
    h = S.h_leaf
    centres = np.array([[(c[1] + 0.5) * 2.0 ** -c[0], (c[2] + 0.5) * 2.0 ** -c[0], (c[3] + 0.5) * 2.0 ** -c[0]]
                        for c in t.leaves])
    g = quad_grad(coef, centres)
    expect = h ** 2.5 * np.sqrt(np.sum(g * g, axis=(1, 2)))
    # leaves whose face-centre values (and their constraining coarse nodes) stay off the walls
    away = np.all((centres - 2.5 * h[:, None] > 0) & (centres + 2.5 * h[:, None] < 1), axis=1)
    assert away.sum() > 200
    assert np.max(np.abs(eta[away] - expect[away]) / expect[away]) < 1e-12
    # a field that vanishes on the walls is exact everywhere: x(1-x) y(1-y) z(1-z) per component
    bub = lambda X: X[:, 0] * (1 - X[:, 0]) * X[:, 1] * (1 - X[:, 1]) * X[:, 2] * (1 - X[:, 2])
    a = np.array([1.0, -2.0, 0.5])
    u = np.concatenate([a[c] * bub(X) for c in range(3)])
    eta = refine.gradient_indicator(S, u)
    x, y, z = centres[:, 0], centres[:, 1], centres[:, 2]
    gb = np.stack([(1 - 2 * x) * y * (1 - y) * z * (1 - z), x * (1 - x) * (1 - 2 * y) * z * (1 - z),
                   x * (1 - x) * y * (1 - y) * (1 - 2 * z)], -1)
    expect = h ** 2.5 * np.linalg.norm(a) * np.linalg.norm(gb, axis=1)
    assert np.max(np.abs(eta - expect)) < 1e-12 * np.max(expect)


def test_refine_by_indicator_marks_largest(oct_s):
    p, t, S = oct_s
    rng = np.random.default_rng(22)
    eta = rng.random(len(t.leaves))
    new = refine.refine_by_indicator(t.leaves, eta)
    m = refine.marked_count(len(t.leaves), 1.0 / 7.0)
    assert m == int(np.floor(len(t.leaves) / 7 + 0.5))
    top = set(np.argsort(-eta)[:m])
    new_set = set(new)
    for i, c in enumerate(t.leaves):
        if i in top:
            assert c not in new_set
            assert all(ch in new_set or any(g in new_set for g in octree.children(ch)) for ch in octree.children(c))
    assert octree.is_balanced(new)
    assert len(new) >= len(t.leaves) + 7 * m
    assert new == sorted(new, key=octree.cell_key)
