"""Adaptive octree meshes of the unit cube: refinement around the sinkers, 2:1 balance,
hanging-node constraints and the level structure of local smoothing (Abstract; Section
2.2.1 by citation of Janssen & Kanschat; adaptive configuration of the sinker benchmark).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A cell is (l, i, j, k): level l, integer position 0 <= i, j, k < 2^l, side 2^-l. Leaves are
the active cells. Points are written on the lattice of spacing 2^-(Lmax+1) (half the finest
cell side), so the Q2 nodes of every cell are lattice points: a level-l cell with S =
2^(Lmax+1-l) lattice units per side has its nodes at (i S, j S, k S) + (a, b, c) S / 2 with
a, b, c in {0, 1, 2}. Point key = x + Mx (y + Mx z), Mx = 2^(Lmax+1) + 1; node numbers are
assigned in increasing key order, cells in increasing (l, k, j, i).

Readings (the paper cites its adaptive method instead of stating it):
* refinement: a leaf is split while its level is below a sinker's maximum level and its
  distance interval [min, max |x - c|] over the cell meets the shell r - w < |x - c| < r + w;
* balance: "full" 2:1 balance, leaves that share a face, an edge or a vertex differ by at
  most one level;
* hanging nodes: a node of a leaf that lies on a face or edge of a coarser neighbouring leaf
  and is not one of that leaf's nodes takes the value of the coarser leaf's Q2 (velocity) or
  Q1 (pressure) interpolant there; nodes on the boundary of the cube are Dirichlet instead;
* local smoothing: level l holds every cell of level l (leaf or refined); its nodes on the
  boundary of the union of those cells that are not on the cube's boundary are the
  refinement-edge nodes.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import fe

DIRS26 = [d for d in itertools.product((-1, 0, 1), repeat=3) if d != (0, 0, 0)]


def cell_key(c):
    l, i, j, k = c
    return (l << 48) | (k << 32) | (j << 16) | i


def parent(c):
    l, i, j, k = c
    return (l - 1, i >> 1, j >> 1, k >> 1)


def children(c):
    l, i, j, k = c
    return [(l + 1, 2 * i + a, 2 * j + b, 2 * k + cc) for cc in (0, 1) for b in (0, 1) for a in (0, 1)]


def distance_interval(c, centre):
    """min and max of |x - centre| over the closed box of cell c (plain per-axis formulas)."""
    l, i, j, k = c
    h = 2.0 ** (-l)
    lo = (i * h, j * h, k * h)
    dmin2 = 0.0
    dmax2 = 0.0
    for d in range(3):
        a = lo[d]
        b = lo[d] + h
        x = centre[d]
        gap = max(a - x, 0.0, x - b)
        far = max(abs(x - a), abs(x - b))
        dmin2 = dmin2 + gap * gap
        dmax2 = dmax2 + far * far
    return np.sqrt(dmin2), np.sqrt(dmax2)


def refine_shells(base_level, centres, max_levels, radius, half_width):
    """Leaves after splitting, until nothing changes, every leaf whose distance interval to a
    sinker centre meets (radius - half_width, radius + half_width) while its level is below
    that sinker's maximum level."""
    n = 1 << base_level
    leaves = {(base_level, i, j, k) for k in range(n) for j in range(n) for i in range(n)}
    lo_r = radius - half_width
    hi_r = radius + half_width
    changed = True
    while changed:
        changed = False
        nxt = set()
        for c in leaves:
            split = False
            for centre, lmax in zip(centres, max_levels):
                if c[0] >= lmax:
                    continue
                dmin, dmax = distance_interval(c, centre)
                if dmin < hi_r and dmax > lo_r:
                    split = True
                    break
            if split:
                nxt.update(children(c))
                changed = True
            else:
                nxt.add(c)
        leaves = nxt
    return leaves


def all_cells(leaves):
    cells = set()
    for c in leaves:
        while c[0] >= 0 and c not in cells:
            cells.add(c)
            if c[0] == 0:
                break
            c = parent(c)
    return cells


def balance(leaves):
    """Smallest refinement of `leaves` in which leaves sharing a face, edge or vertex differ by
    at most one level (processed from the finest level down; refining only ever adds cells)."""
    leaves = set(leaves)
    cells = all_cells(leaves)
    lmax = max(c[0] for c in leaves)
    for l in range(lmax, 1, -1):
        for c in sorted((c for c in leaves if c[0] == l), key=cell_key):
            _, i, j, k = c
            n = 1 << l
            for dx, dy, dz in DIRS26:
                ni, nj, nk = i + dx, j + dy, k + dz
                if not (0 <= ni < n and 0 <= nj < n and 0 <= nk < n):
                    continue
                target = (l - 1, ni >> 1, nj >> 1, nk >> 1)
                while target not in cells:
                    anc = parent(target)
                    while anc not in cells:
                        anc = parent(anc)
                    leaves.discard(anc)
                    for ch in children(anc):
                        leaves.add(ch)
                        cells.add(ch)
    return leaves


def is_balanced(leaves):
    """True if no two leaves touching by a face, edge or vertex differ by more than one level."""
    cells = all_cells(leaves)
    for c in leaves:
        l, i, j, k = c
        n = 1 << l
        for dx, dy, dz in DIRS26:
            ni, nj, nk = i + dx, j + dy, k + dz
            if not (0 <= ni < n and 0 <= nj < n and 0 <= nk < n):
                continue
            if l >= 2 and (l - 1, ni >> 1, nj >> 1, nk >> 1) not in cells:
                return False
    return True


class Octree:
    """Active mesh, constraints and level structure of a 2:1-balanced octree."""

    def __init__(self, leaves, coarsest_level):
        self.leaves = sorted(leaves, key=cell_key)
        self.leaf_set = set(self.leaves)
        self.cells = all_cells(self.leaf_set)
        self.lmax = max(c[0] for c in self.leaves)
        self.lmin_leaf = min(c[0] for c in self.leaves)
        self.coarsest = coarsest_level
        self.Mx = (1 << (self.lmax + 1)) + 1
        self._velocity()
        self._pressure()
        self._levels()

    # -- geometry helpers ---------------------------------------------------
    def S(self, l):
        return 1 << (self.lmax + 1 - l)

    def key(self, p):
        return p[0] + self.Mx * (p[1] + self.Mx * p[2])

    def on_boundary(self, p):
        top = self.Mx - 1
        return any(x == 0 or x == top for x in p)

    def cell_nodes_lattice(self, c):
        l, i, j, k = c
        S = self.S(l)
        h = S // 2
        return [(i * S + a * h, j * S + b * h, k * S + cc * h)
                for cc in range(3) for b in range(3) for a in range(3)]

    def cell_vertices_lattice(self, c):
        l, i, j, k = c
        S = self.S(l)
        return [(i * S + a * S, j * S + b * S, k * S + cc * S)
                for cc in range(2) for b in range(2) for a in range(2)]

    def coarse_neighbours(self, c):
        """(direction, coarser leaf) for every direction in which the same-level neighbour of
        leaf c does not exist (the region is covered by a leaf one level coarser)."""
        l, i, j, k = c
        n = 1 << l
        out = []
        for d in DIRS26:
            ni, nj, nk = i + d[0], j + d[1], k + d[2]
            if not (0 <= ni < n and 0 <= nj < n and 0 <= nk < n):
                continue
            if (l, ni, nj, nk) in self.cells:
                continue
            coarse = (l - 1, ni >> 1, nj >> 1, nk >> 1)
            assert coarse in self.leaf_set, "mesh is not 2:1 balanced"
            out.append((d, coarse))
        return out

    @staticmethod
    def on_side(local, d, top):
        """local lattice index (0..top per axis) lies on the part of the cell boundary facing d."""
        for x, dd in zip(local, d):
            if dd == 1 and x != top:
                return False
            if dd == -1 and x != 0:
                return False
        return True

    # -- velocity (Q2) ------------------------------------------------------
    def _velocity(self):
        hanging = {}        # key -> (coarse cell, lattice point)
        node_level = {}     # key -> coarsest leaf level having the point as a node
        for c in self.leaves:
            for p in self.cell_nodes_lattice(c):
                kk = self.key(p)
                if kk not in node_level or c[0] < node_level[kk]:
                    node_level[kk] = c[0]
        for c in self.leaves:
            l = c[0]
            S = self.S(l)
            pts = self.cell_nodes_lattice(c)
            for d, coarse in self.coarse_neighbours(c):
                for a, p in enumerate(pts):
                    loc = (a % 3, (a // 3) % 3, a // 9)
                    if not self.on_side(loc, d, 2):
                        continue
                    if self.on_boundary(p):
                        continue
                    if all(x % S == 0 for x in p):      # a node of the coarser leaf
                        continue
                    hanging.setdefault(self.key(p), (coarse, p))
        active = sorted(k for k in node_level if k not in hanging)
        self.u_keys = np.array(active, dtype=np.int64)
        self.u_index = {k: n for n, k in enumerate(active)}
        self.n_nodes = len(active)
        self.n_u = 3 * self.n_nodes
        self.u_node_level = np.array([node_level[k] for k in active], dtype=np.int64)
        self.u_boundary = np.array([self.on_boundary(self._point(k)) for k in active], dtype=bool)
        self.hanging_u = {}
        for kk, (coarse, p) in hanging.items():
            l, ci, cj, ck = coarse
            S = self.S(l)
            xi = [(p[0] - ci * S) / S, (p[1] - cj * S) / S, (p[2] - ck * S) / S]
            w1 = [fe.q2_1d(np.array([x]))[0] for x in xi]
            terms = []
            for a, q in enumerate(self.cell_nodes_lattice(coarse)):
                w = w1[0][a % 3] * w1[1][(a // 3) % 3] * w1[2][a // 9]
                if w != 0.0:
                    qk = self.key(q)
                    assert qk in self.u_index, "constraint chain (constraining node is hanging)"
                    terms.append((self.u_index[qk], w))
            self.hanging_u[kk] = terms
        # per leaf, per local node: list of (active node, weight)
        self.leaf_u = []
        for c in self.leaves:
            row = []
            for p in self.cell_nodes_lattice(c):
                kk = self.key(p)
                if kk in self.u_index:
                    row.append([(self.u_index[kk], 1.0)])
                else:
                    row.append(self.hanging_u[kk])
            self.leaf_u.append(row)

    def _point(self, kk):
        x = kk % self.Mx
        y = (kk // self.Mx) % self.Mx
        z = kk // (self.Mx * self.Mx)
        return (x, y, z)

    # -- pressure (Q1) ------------------------------------------------------
    def _pressure(self):
        verts = set()
        for c in self.leaves:
            for p in self.cell_vertices_lattice(c):
                verts.add(self.key(p))
        hanging = {}
        for c in self.leaves:
            l = c[0]
            S = self.S(l)
            pts = self.cell_vertices_lattice(c)
            for d, coarse in self.coarse_neighbours(c):
                for a, p in enumerate(pts):
                    loc = (a % 2, (a // 2) % 2, a // 4)
                    if not self.on_side(loc, d, 1):
                        continue
                    if all(x % (2 * S) == 0 for x in p):  # a vertex of the coarser leaf
                        continue
                    hanging.setdefault(self.key(p), (coarse, p))
        active = sorted(k for k in verts if k not in hanging)
        self.p_keys = np.array(active, dtype=np.int64)
        self.p_index = {k: n for n, k in enumerate(active)}
        self.n_p = len(active)
        self.hanging_p = {}
        for kk, (coarse, p) in hanging.items():
            l, ci, cj, ck = coarse
            S = self.S(l)
            xi = [(p[0] - ci * S) / S, (p[1] - cj * S) / S, (p[2] - ck * S) / S]
            terms = []
            for a, q in enumerate(self.cell_vertices_lattice(coarse)):
                w = 1.0
                for dd, x in enumerate(xi):
                    w = w * (x if ((a >> dd) & 1) else 1.0 - x)
                if w != 0.0:
                    terms.append((self.p_index[self.key(q)], w))
            self.hanging_p[kk] = terms
        self.leaf_p = []
        for c in self.leaves:
            row = []
            for p in self.cell_vertices_lattice(c):
                kk = self.key(p)
                row.append([(self.p_index[kk], 1.0)] if kk in self.p_index else self.hanging_p[kk])
            self.leaf_p.append(row)

    # -- levels (local smoothing) --------------------------------------------
    def _levels(self):
        self.level_cells = []
        self.level_keys = []
        self.level_index = []
        self.level_cell_nodes = []
        self.level_boundary = []
        self.level_edge = []
        for l in range(self.lmax + 1):
            cl = sorted((c for c in self.cells if c[0] == l), key=cell_key)
            cset = set(cl)
            keys = sorted({self.key(p) for c in cl for p in self.cell_nodes_lattice(c)})
            index = {k: n for n, k in enumerate(keys)}
            cn = np.array([[index[self.key(p)] for p in self.cell_nodes_lattice(c)] for c in cl], dtype=np.int64)
            S = self.S(l)
            n = 1 << l
            bnd = np.zeros(len(keys), dtype=bool)
            edge = np.zeros(len(keys), dtype=bool)
            for t, kk in enumerate(keys):
                p = self._point(kk)
                if self.on_boundary(p):
                    bnd[t] = True
                    continue
                # level-l cells whose closed box contains p
                rng = []
                for x in p:
                    q, r = divmod(x, S)
                    rng.append((q - 1, q) if r == 0 else (q,))
                for ci in rng[0]:
                    for cj in rng[1]:
                        for ck in rng[2]:
                            if 0 <= ci < n and 0 <= cj < n and 0 <= ck < n and (l, ci, cj, ck) not in cset:
                                edge[t] = True
            self.level_cells.append(cl)
            self.level_keys.append(np.array(keys, dtype=np.int64))
            self.level_index.append(index)
            self.level_cell_nodes.append(cn)
            self.level_boundary.append(bnd)
            self.level_edge.append(edge)
        # copy indices: active node -> (its level, index on that level)
        self.copy_level = self.u_node_level.copy()
        self.copy_index = np.array([self.level_index[l][int(k)] for k, l in zip(self.u_keys, self.copy_level)],
                                   dtype=np.int64)
