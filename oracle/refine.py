"""Adaptive refinement driven by a gradient indicator (Section 3.3).

Test infrastructure: a plain restatement that the CUDA library's host refinement is checked
against; only tests/, the smoke check and the benchmark's CPU legs use it.

The paper's AMG/GMG comparison starts from 4 global refinements and builds each new mesh with a
gradient-based estimator that refines roughly 1/7 of the cells, so that the cell count about
doubles per cycle; the estimator itself is not specified. Reading taken here:
  * indicator of leaf K (side h): eta_K = h^(5/2) |grad u_h(x_K)|_F, the Frobenius norm of the
    gradient of the Q2 velocity at the leaf centre x_K (the h^(1 + d/2) scaling of a gradient
    approximation, d = 3). The leaf's nodal values come from the active vector through the
    hanging-node constraints, with the Dirichlet values taken as 0 (the wall condition). At the
    centre the Q2 basis gives d/dx u = (u(1, 1/2, 1/2) - u(0, 1/2, 1/2)) / h per component, the
    face-centre nodes' difference, and likewise along y and z;
  * marking: the floor(n f + 1/2) leaves with the largest eta (f = 1/7; equal eta: smaller
    cell key first) are split into their 8 children; then the tree is 2:1 balanced.
"""
from __future__ import annotations

import numpy as np

from . import octree

# local Q2 node index i + 3 j + 9 k of the face centres: (minus, plus) pairs along x, y, z
FACE_PAIRS = ((12, 14), (10, 16), (4, 22))


def leaf_values(S, u):
    """(leaves, 3, 27) nodal velocity of every leaf from the active vector u (Dirichlet rows 0)."""
    v = np.array(u, dtype=np.float64, copy=True)
    v[S.dirichlet] = 0.0
    return (S.Cu @ v).reshape(len(S.tree.leaves), 3, 27)


def gradient_indicator(S, u):
    """eta_K = h^(5/2) |grad u_h(x_K)|_F for every leaf of S.tree (sorted leaf order)."""
    U = leaf_values(S, u)
    h = S.h_leaf
    sq = np.zeros(len(h))
    for lo, hi in FACE_PAIRS:
        d = (U[:, :, hi] - U[:, :, lo]) / h[:, None]
        sq += np.sum(d * d, axis=1)
    return h ** 2.5 * np.sqrt(sq)


def marked_count(n_leaves, fraction):
    return int(np.floor(n_leaves * fraction + 0.5))


def refine_by_indicator(leaves, eta, fraction=1.0 / 7.0):
    """Split the marked leaves (largest eta; ties by smaller key), then 2:1 balance.
    `leaves` as (l, i, j, k) tuples in the order eta refers to. Returns the sorted new leaves."""
    keys = np.array([octree.cell_key(c) for c in leaves], dtype=np.uint64)
    order = sorted(range(len(leaves)), key=lambda i: (-eta[i], int(keys[i])))
    marked = set(order[:marked_count(len(leaves), fraction)])
    out = set()
    for i, c in enumerate(leaves):
        if i in marked:
            out.update(octree.children(c))
        else:
            out.add(c)
    return sorted(octree.balance(out), key=octree.cell_key)
