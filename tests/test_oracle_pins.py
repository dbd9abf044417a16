"""Pins of the CPU oracle against closed forms, invariants and published values.

Each test fixes one part of the oracle by something other than the oracle
itself, chosen so that a dropped term, wrong sign, transposed operand or wrong
index fails at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import sinker_inputs as si
from oracle import fe, gmg, krylov, mesh, operators, sinker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1) if ":" in line else line.split(None, 1)
            out[k.strip()] = v.split()
    return out


# ---------------------------------------------------------------- generator
def test_splitmix64_published_values():
    g = _golden("splitmix64.txt")
    assert [int(x) for x in si.splitmix64(1234567, 5)] == [int(x) for x in g["seed 1234567"]]
    assert [int(x) for x in si.splitmix64(0, 3)] == [int(x) for x in g["seed 0"]]
    u = si.uniform01(7, 10000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


# ---------------------------------------------------------------- 1D bases, quadrature
def test_gauss3_exactness_and_first_error_term():
    g, w = fe.gauss3()
    for k in range(6):
        assert abs(w @ g ** k - 1.0 / (k + 1)) < 1e-15
    # Gauss-Legendre error for n = 3 on [0,1]: (3!)^4 / (7 (6!)^3) f^(6) = 720/2800/720 -> 1/2800
    assert abs((1.0 / 7.0 - w @ g ** 6) - 1.0 / 2800.0) < 1e-15


def test_q2_lagrange_properties():
    x = np.linspace(0, 1, 11)
    v = fe.q2_1d(x)
    d = fe.q2_1d_deriv(x)
    assert np.allclose(fe.q2_1d(fe.Q2_NODES_1D), np.eye(3), atol=1e-15)
    assert np.allclose(v.sum(1), 1.0)
    assert np.allclose(d.sum(1), 0.0)
    # reproduces x^2 and its derivative 2x
    assert np.allclose(v @ fe.Q2_NODES_1D ** 2, x ** 2)
    assert np.allclose(d @ fe.Q2_NODES_1D ** 2, 2 * x)
    # closed forms: l0 = 2x^2 - 3x + 1, l1 = 4x - 4x^2, l2 = 2x^2 - x
    assert np.allclose(v, np.stack([2 * x ** 2 - 3 * x + 1, 4 * x - 4 * x ** 2, 2 * x ** 2 - x], 1))
    assert np.allclose(d, np.stack([4 * x - 3, 4 - 8 * x, 4 * x - 1], 1))


# ---------------------------------------------------------------- element matrices
def _nodal(h, field):
    """Element nodal vector (c*27 + a) of a vector field on [0,h]^3."""
    pts = np.array([[i / 2, j / 2, k / 2] for k in range(3) for j in range(3) for i in range(3)]) * h
    vals = np.array([field(p) for p in pts])          # (27, 3)
    return np.concatenate([vals[:, c] for c in range(3)])


def test_element_A_energies_closed_form():
    h, mu = 0.3, 2.5
    A = fe.element_A(h, mu)
    vol = h ** 3
    # int 2 mu eps:eps over the cell
    cases = [
        (lambda p: (p[0], 0, 0), 2 * mu * vol),          # eps_xx = 1
        (lambda p: (p[1], 0, 0), mu * vol),              # eps_xy = eps_yx = 1/2
        (lambda p: (p[1], p[0], 0), 4 * mu * vol),       # eps_xy = 1
        (lambda p: (p[1], -p[0], 0), 0.0),               # rotation
        (lambda p: (0, 0, p[2]), 2 * mu * vol),
        (lambda p: (p[2], 0, p[0]), 4 * mu * vol),
    ]
    for f, e in cases:
        u = _nodal(h, f)
        assert abs(u @ A @ u - e) < 1e-12 * max(1.0, e), (e, u @ A @ u)


def test_element_A_symmetric_rank_and_rigid_modes():
    h = 0.25
    A = fe.element_A(h, 1.0)
    assert np.abs(A - A.T).max() < 1e-14
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-12
    assert int((ev > 1e-10 * ev.max()).sum()) == 75
    modes = [lambda p: (1, 0, 0), lambda p: (0, 1, 0), lambda p: (0, 0, 1),
             lambda p: (-p[1], p[0], 0), lambda p: (0, -p[2], p[1]), lambda p: (p[2], 0, -p[0])]
    for f in modes:
        assert np.abs(A @ _nodal(h, f)).max() < 1e-13


def test_element_B_and_Mp_closed_forms():
    h = 0.5
    B = fe.element_B(h)
    # div u = 1 for u = (x, 0, 0): (B u)_l = -int psi_l = -h^3 / 8
    assert np.allclose(B @ _nodal(h, lambda p: (p[0], 0, 0)), -h ** 3 / 8)
    # u = (0, y, z): div = 2
    assert np.allclose(B @ _nodal(h, lambda p: (0, p[1], p[2])), -2 * h ** 3 / 8)
    # solenoidal u = (y, -x, 0): zero
    assert np.abs(B @ _nodal(h, lambda p: (p[1], -p[0], 0))).max() < 1e-15
    M = fe.element_Mp(h, 1.0 / 3.0)
    assert abs(M.sum() - h ** 3 / 3.0) < 1e-15
    px = np.array([(i % 2) * h for i in range(8)])       # p = x at the vertices
    assert abs(px @ fe.element_Mp(h, 1.0) @ px - h ** 5 / 3.0) < 1e-15



def _exact_1d_q2():
    """Exact 1D matrices of the Q2 Lagrange basis on [0, 1] (nodes 0, 1/2, 1), by integrating the
    polynomial products with rational arithmetic: K_pq = int l_p' l_q', M_pq = int l_p l_q,
    C_pq = int l_p' l_q."""
    from fractions import Fraction as Fr
    basis = [[Fr(1), Fr(-3), Fr(2)], [Fr(0), Fr(4), Fr(-4)], [Fr(0), Fr(-1), Fr(2)]]   # coefficients of 1, x, x^2

    def deriv(a):
        return [a[1], 2 * a[2], Fr(0)]

    def integral(a, b):   # int_0^1 a(x) b(x) dx
        return sum(a[i] * b[j] / (i + j + 1) for i in range(3) for j in range(3))

    d = [deriv(a) for a in basis]
    K = [[integral(d[p], d[q]) for q in range(3)] for p in range(3)]
    M = [[integral(basis[p], basis[q]) for q in range(3)] for p in range(3)]
    C = [[integral(d[p], basis[q]) for q in range(3)] for p in range(3)]
    return K, M, C


def test_element_A_is_the_exact_tensor_product_form():
    """The 81 x 81 element matrix of 2 mu eps:eps, entry by entry, against its closed form from
    exactly integrated 1D matrices. For test function phi_I e_a and trial function phi_J e_b,
    2 eps(phi_J e_b):eps(phi_I e_a) = delta_ab grad phi_I . grad phi_J + d_a phi_J d_b phi_I, and
    each integral over the cube [0, h]^3 is a product of 1D factors (K / h along an axis that
    carries both derivatives, the mixed C along an axis that carries one, h M elsewhere).
    So 5400 A_hat / (mu h) is an integer matrix (lcm of 3 * 30 * 30 and 6 * 6 * 30), with entries
    up to 2^15 on the diagonal."""
    from fractions import Fraction as Fr
    K, M, C = _exact_1d_q2()
    # the textbook forms: K = [7 -8 1; -8 16 -8; 1 -8 7] / 3, M = [4 2 -1; 2 16 2; -1 2 4] / 30
    assert K == [[Fr(7, 3), Fr(-8, 3), Fr(1, 3)], [Fr(-8, 3), Fr(16, 3), Fr(-8, 3)], [Fr(1, 3), Fr(-8, 3), Fr(7, 3)]]
    assert M == [[Fr(4, 30), Fr(2, 30), Fr(-1, 30)], [Fr(2, 30), Fr(16, 30), Fr(2, 30)], [Fr(-1, 30), Fr(2, 30), Fr(4, 30)]]
    h, mu = 0.37, 1.7
    idx = [(i, j, k) for k in range(3) for j in range(3) for i in range(3)]   # local node i + 3 j + 9 k
    want = np.zeros((81, 81))
    for a in range(3):
        for b in range(3):
            for I, ni in enumerate(idx):
                for J, nj in enumerate(idx):
                    grad = Fr(0)
                    if a == b:
                        for d in range(3):   # axis d carries both derivatives
                            t = K[ni[d]][nj[d]]
                            for e in range(3):
                                if e != d:
                                    t *= M[ni[e]][nj[e]]
                            grad += t
                    cpl = Fr(1)
                    for d in range(3):   # d_a phi_J d_b phi_I
                        if d == a and d == b:
                            cpl *= K[nj[d]][ni[d]]
                        elif d == a:
                            cpl *= C[nj[d]][ni[d]]
                        elif d == b:
                            cpl *= C[ni[d]][nj[d]]
                        else:
                            cpl *= M[nj[d]][ni[d]]
                    want[a * 27 + I, b * 27 + J] = float(grad + cpl)
    assert np.allclose(want * 5400, np.round(want * 5400), rtol=0, atol=1e-9)
    assert np.abs(np.round(want * 5400)).max() == 2 ** 15
    got = fe.element_A(h, mu)
    assert np.abs(got - mu * h * want).max() <= 1e-13 * np.abs(got).max()


def test_element_Mp_is_the_q1_mass_tensor_product():
    """M_p's element matrix with the cell value of 1/mu is (h^3 / mu) m1 x m1 x m1, m1 = [2 1; 1 2] / 6
    the exact 1D Q1 mass matrix on [0, 1], for every entry."""
    h, inv_mu = 0.4, 0.3
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
    want = inv_mu * h ** 3 * np.kron(m1, np.kron(m1, m1))
    assert np.abs(fe.element_Mp(h, inv_mu) - want).max() <= 1e-15 * want.max()


# ---------------------------------------------------------------- global operators
def _int_phi_1d(M):
    """int of the global 1D Q2 basis function of each node on [0,1] with spacing h/2:
    boundary vertex h/6, interior vertex h/3, midpoint 2h/3."""
    n = (M - 1) // 2
    h = 1.0 / n
    w = np.where(np.arange(M) % 2 == 1, 2 * h / 3, h / 3)
    w[0] = w[-1] = h / 6
    return w


def test_global_A_reproduces_quadratic_fields():
    """For constant mu and quadratic u, -div(2 mu eps(u)) = -mu(lap u + grad div u) = c is
    constant, so (A u)_i = c_comp * int phi_node for DoFs whose basis vanishes on the boundary."""
    n, mu = 4, 1.7
    m = mesh.Mesh(n)
    ops = operators.Operators(m, np.full(m.n_cells, mu))
    X = m.node_coords()
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    a, b, d, e, f = 1.0, 2.0, 3.0, 5.0, 7.0
    u = np.concatenate([a * x ** 2 + b * y ** 2 + e * y * z, x * z, d * z ** 2 + f * x * y])
    c = -mu * np.array([4 * a + 2 * b, 0.0, 4 * d])
    w1 = _int_phi_1d(m.M)
    intphi = np.einsum("k,j,i->kji", w1, w1, w1).ravel()
    y_ = ops.apply_A_unconstrained(u)
    inner = ~m.boundary_node
    for comp in range(3):
        got = y_[comp * m.n_nodes:(comp + 1) * m.n_nodes][inner]
        assert np.allclose(got, c[comp] * intphi[inner], rtol=1e-12, atol=1e-12)


def test_global_A_rigid_modes_and_constraints():
    n = 3
    m = mesh.Mesh(n)
    mu = 1.0 + si.uniform01(5, m.n_cells)
    ops = operators.Operators(m, mu)
    X = m.node_coords()
    for om in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        r = np.cross(np.array(om, float)[None, :], X)
        v = np.concatenate([r[:, 0], r[:, 1], r[:, 2]]) + 0.3
        assert np.abs(ops.apply_A_unconstrained(v)).max() < 1e-12
    A = ops.csr_A()
    assert abs(A - A.T).max() < 1e-14
    xr = si.uniform(3, m.n_u)
    assert np.allclose(A @ xr, ops.apply_A(xr), atol=1e-13)
    y = ops.apply_A(xr)
    assert np.array_equal(y[m.dirichlet], xr[m.dirichlet])


@pytest.mark.parametrize("n", [8, 12])
def test_row_evaluator_equals_element_operator_on_every_row(n):
    """operators.apply_A_rows (the row-by-row A_c x that the full-size GPU checks use, with no
    global cell tables) equals the element-by-element Operators.apply_A, itself pinned above by
    quadratic reproduction, rigid modes and the constraints, on every row of an 8^3 and a 12^3
    mesh: interior rows, rows next to each wall, edge and corner, and the identity rows on the
    walls. Cell viscosity varies by cell (1..100) and x is non-zero on constrained entries, so a
    wrong cell index, local index, boundary mask or mu lookup fails it."""
    m = mesh.Mesh(n)
    mu = 1.0 + 99.0 * si.uniform01(11 + n, m.n_cells)
    x = si.uniform(12 + n, m.n_u)
    ref = operators.Operators(m, mu).apply_A(x)
    got = operators.apply_A_rows(n, mu, x, np.arange(m.n_u))
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    # the comparison sees a boundary-mask mistake: rows that also took the constrained entries
    # of x (the unconstrained operator) differ from it by far more than rounding
    wrong = operators.Operators(m, mu).apply_A_unconstrained(x)
    free = ~m.dirichlet
    assert np.abs(wrong[free] - got[free]).max() > 1e-3 * np.abs(ref).max()


def test_BT_of_linear_pressure_and_adjointness():
    """(B^T p)_(c,node) = -int d_c phi p = int phi d_c p for interior nodes; for p = x that is
    int phi on the x component and 0 elsewhere. And (B u, p) = (u, B^T p)."""
    n = 4
    m = mesh.Mesh(n)
    ops = operators.Operators(m, np.ones(m.n_cells))
    V = m.vertex_coords()
    p = V[:, 0].copy()
    g = ops.apply_BT(p)
    w1 = _int_phi_1d(m.M)
    intphi = np.einsum("k,j,i->kji", w1, w1, w1).ravel()
    inner = ~m.boundary_node
    assert np.allclose(g[:m.n_nodes][inner], intphi[inner], atol=1e-14)
    assert np.abs(g[m.n_nodes:]).max() < 1e-14
    u = si.uniform(11, m.n_u) * (~m.dirichlet)
    q = si.uniform(12, m.n_p)
    assert abs(ops.apply_B(u) @ q - u @ ops.apply_BT(q)) < 1e-13


def _moments_1d(n, deriv):
    """Assembled 1D moments X[i, v] = int over [0, 1] of (l_i or l_i') psi_v for the Q2 nodes i
    (2n + 1, on n cells of side 1/n) against the Q1 vertices v (n + 1): the exact integrals of
    piecewise polynomials of degree <= 3, by 3-point Gauss-Legendre per cell (numpy's nodes),
    in reference-cell units (no powers of h)."""
    xg, wg = np.polynomial.legendre.leggauss(3)
    xg, wg = (xg + 1) / 2, wg / 2
    X = np.zeros((2 * n + 1, n + 1))
    for e in range(n):
        for x, w in zip(xg, wg):
            # Q2 nodes at 0, 1/2, 1 of the cell and Q1 vertices at 0, 1, by Lagrange's formula
            q2 = [2 * (x - 0.5) * (x - 1), -4 * x * (x - 1), 2 * x * (x - 0.5)]
            dq2 = [4 * x - 3, -8 * x + 4, 4 * x - 1]
            q1 = [1 - x, x]
            for a in range(3):
                for v in range(2):
                    X[2 * e + a, e + v] += w * (dq2[a] if deriv else q2[a]) * q1[v]
    return X


@pytest.mark.parametrize("n", [2, 3, 5])
def test_BT_is_a_tensor_product_of_assembled_1d_moments(n):
    """B^T carries no viscosity: component c of B^T p is -h^2 (X_z x X_y x X_x) p with the 1D
    moments X assembled along each axis (derivative moments along axis c, plain moments along the
    other two), on every free row; the rows of constrained velocity nodes are 0. Computed here from
    1D Gauss quadrature of the Lagrange bases, independent of the element matrices (the form the
    uniform-mesh B^T kernel evaluates)."""
    m = mesh.Mesh(n)
    mu = 0.5 + si.uniform01(31, m.n_cells) * 10     # any viscosity: B^T must not see it
    ops = operators.Operators(m, mu)
    p = si.uniform(32, m.n_p)
    got = ops.apply_BT(p)
    V, D = _moments_1d(n, False), _moments_1d(n, True)
    P = n + 1
    pg = p.reshape(P, P, P)   # [k][j][i], vertex = i + P j + P^2 k
    for c in range(3):
        X = [D if c == d else V for d in range(3)]
        want = -m.h ** 2 * np.einsum("ia,jb,kc,cba->kji", X[0], X[1], X[2], pg).ravel()
        rows = got[c * m.n_nodes:(c + 1) * m.n_nodes]
        free = ~m.dirichlet[c * m.n_nodes:(c + 1) * m.n_nodes]
        assert np.allclose(rows[free], want[free], rtol=1e-13, atol=1e-15 * np.abs(want).max())
        assert np.all(rows[~free] == 0.0)


def test_Mp_integrals_and_wathen_bound():
    n = 3
    m = mesh.Mesh(n)
    mu = 0.5 + si.uniform01(21, m.n_cells) * 10
    ops = operators.Operators(m, mu)
    one = np.ones(m.n_p)
    assert abs(one @ ops.apply_Mp(one) - np.sum(m.h ** 3 / mu)) < 1e-13
    M = np.column_stack([ops.apply_Mp(e) for e in np.eye(m.n_p)])
    D = ops.diag_Mp()
    ev = np.linalg.eigvals(M / D[:, None]).real
    assert ev.min() >= 1 / 8 - 1e-12 and ev.max() <= 27 / 8 + 1e-12
    assert abs(ops.pressure_weights().sum() - 1.0) < 1e-14


def test_rhs_of_constant_forcing():
    n = 4
    m = mesh.Mesh(n)
    fq = np.zeros((m.n_cells, 27, 3))
    fq[:, :, 2] = 1.0
    F = operators.assemble_rhs(m, fq)
    w1 = _int_phi_1d(m.M)
    intphi = np.einsum("k,j,i->kji", w1, w1, w1).ravel()
    inner = ~m.boundary_node
    assert np.allclose(F[2 * m.n_nodes:][inner], intphi[inner], atol=1e-15)
    assert np.abs(F[:2 * m.n_nodes]).max() == 0.0
    assert np.all(F[m.dirichlet] == 0.0)


def test_paper_sparsity_example_402_dofs():
    """Section 2.2.1 figure: 2x2x2 Q2-Q1 has 375 + 27 = 402 DoFs; full coupling has ~3x
    the velocity entries of the partial coupling (one diagonal block per component)."""
    g = _golden("stokes_2x2x2_dofs.txt")
    m = mesh.Mesh(int(g["n_cells_per_axis"][0]))
    assert m.n_u == int(g["velocity_dofs"][0]) and m.n_p == int(g["pressure_dofs"][0])
    assert m.n_u + m.n_p == int(g["total_dofs"][0])
    ops = operators.Operators(m, np.ones(m.n_cells))
    rows = np.repeat(m.cell_dofs, 81, axis=1).ravel()
    cols = np.tile(m.cell_dofs, (1, 81)).ravel()
    pattern = sp.coo_matrix((np.ones(rows.size), (rows, cols)), shape=(m.n_u, m.n_u)).tocsr()
    full = pattern.nnz
    comp = lambda i: i // m.n_nodes
    r, c = pattern.nonzero()
    partial = int(np.sum(comp(r) == comp(c)))
    assert full == int(g["full_over_partial_entries"][0]) * partial


# ---------------------------------------------------------------- sinker coefficients
def test_sinker_coefficient_limits_and_averaging():
    prob = si.SinkerProblem(n=4, n_levels=1, centres=np.array([[0.5, 0.5, 0.5]]), mu_min=0.01, mu_max=100.0)
    c = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.52], [0.0, 0.0, 0.0]])
    mu = sinker.viscosity(c, prob)
    f = sinker.forcing(c, prob)
    assert mu[0] == 100.0 and mu[1] == 100.0             # inside omega/2: X = 0
    assert abs(mu[2] - 0.01) < 1e-12                     # far away: X -> 1
    assert f[0, 2] == -10.0 and abs(f[2, 2]) < 1e-12
    d = 0.1                                              # distance 0.1: X = 1 - exp(-200 * 0.05^2)
    X = 1 - np.exp(-200 * 0.05 ** 2)
    assert abs(sinker.indicator(np.array([[0.6, 0.5, 0.5]]), prob.centres, 200, 0.1)[0] - X) < 1e-15
    # harmonic mean with quadrature weights: constant -> same; 1/mu linear in weights
    _, w = fe.quadrature_3d()
    assert abs(sinker.harmonic_cell_average(np.full(27, 3.0)) - 3.0) < 1e-15
    vals = np.where(np.arange(27) == 13, 2.0, 1.0)       # centre point has weight (8/18)^3
    expect = 1.0 / (1 - w[13] + w[13] / 2.0)
    assert abs(sinker.harmonic_cell_average(vals) - expect) < 1e-15
    fine = np.arange(64, dtype=float)
    par = sinker.restrict_cell_viscosity(fine, 4)
    assert abs(par[0] - np.mean([0, 1, 4, 5, 16, 17, 20, 21])) < 1e-15


# ---------------------------------------------------------------- transfers
def test_prolongation_is_q2_embedding():
    nc = 2
    P = gmg.prolongation(nc)
    cm, fm = mesh.Mesh(nc), mesh.Mesh(2 * nc)
    coarse = si.uniform(31, cm.n_u)
    fine = P @ coarse
    # evaluate the coarse field directly at the fine nodes with the 3D basis of the coarse cell
    X = fm.node_coords()
    cell = np.minimum((X / cm.h).astype(int), nc - 1)
    loc = X / cm.h - cell
    val, _ = fe.q2_3d_tables(loc)
    cid = cell[:, 0] + nc * cell[:, 1] + nc * nc * cell[:, 2]
    for comp in range(3):
        ref = np.einsum("pa,pa->p", val, coarse[cm.cell_dofs[cid, comp * 27:(comp + 1) * 27]])
        assert np.allclose(fine[comp * fm.n_nodes:(comp + 1) * fm.n_nodes], ref, atol=1e-14)
    # 1D weights at 1/4 and 3/4 of a coarse cell
    P1 = gmg.prolongation_1d(1).toarray()
    assert np.allclose(P1[1], [3 / 8, 3 / 4, -1 / 8]) and np.allclose(P1[3], [-1 / 8, 3 / 4, 3 / 8])


# ---------------------------------------------------------------- Chebyshev and Lanczos
def _cheb_T(k, x):
    x = np.asarray(x, dtype=float)
    return np.where(np.abs(x) <= 1, np.cos(k * np.arccos(np.clip(x, -1, 1))),
                    np.cosh(k * np.arccosh(np.maximum(np.abs(x), 1))) * np.sign(x) ** k)


def test_chebyshev_error_polynomial():
    """e_k = T_k((theta - lam)/delta) / T_k(theta/delta) e_0 per eigencomponent."""
    lam = np.linspace(0.05, 2.0, 40)
    lo, hi = 0.1, 1.8
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    b = si.uniform(41, lam.size)
    xstar = b / lam
    x0 = si.uniform(42, lam.size)
    A = lambda v: lam * v
    for k in (1, 2, 4, 5):
        x = gmg.chebyshev_smooth(A, np.ones_like(lam), b, x0, k, lo, hi, False)
        expect = _cheb_T(k, (theta - lam) / delta) / _cheb_T(k, theta / delta) * (x0 - xstar)
        assert np.allclose(x - xstar, expect, atol=1e-12)
        x = gmg.chebyshev_smooth(A, np.ones_like(lam), b, None, k, lo, hi, True)
        expect = _cheb_T(k, (theta - lam) / delta) / _cheb_T(k, theta / delta) * (-xstar)
        assert np.allclose(x - xstar, expect, atol=1e-12)


def test_lanczos_exact_on_small_spectrum():
    lam = np.array([0.5, 1.0, 1.5, 2.0, 3.0, 4.5, 7.0, 9.0])
    x = gmg.lanczos_lambda_max(lambda v: lam * v, np.ones(8), np.ones(8), 77, 12)
    assert abs(x - 9.0) < 1e-12
    d = 1.0 / (1.0 + np.arange(8))
    x = gmg.lanczos_lambda_max(lambda v: lam * v, d, np.ones(8), 78, 12)
    assert abs(x - np.max(lam * d)) < 1e-12


# ---------------------------------------------------------------- solver-level pins
def _problem(name):
    p = si.workload(name)
    m = mesh.Mesh(p.n)
    mus = sinker.level_viscosities(m, p, p.n_levels)
    G = gmg.GMG(p.n, p.n_levels, mus)
    ops = G.levels[-1].ops
    F = operators.assemble_rhs(m, sinker.forcing(m.quad_points(), p))
    return p, m, G, ops, F


def test_exact_preconditioner_two_iterations():
    """eq. stokes_precond: with exact A^-1 and S^-1, FGMRES converges in at most 2 iterations."""
    p, m, G, ops, F = _problem("cube2")
    A = ops.csr_A().toarray()
    B = ops.csr_B().toarray()
    Ainv = np.linalg.inv(A)
    S = B @ Ainv @ B.T
    Spinv = np.linalg.pinv(S, rcond=1e-10, hermitian=True)   # S is singular on constants only
    Pc = krylov.StokesPreconditioner(ops, G, exact_A=lambda t: Ainv @ t, exact_S=lambda r: Spinv @ r)
    b = np.concatenate([F, np.zeros(m.n_p)])
    _, its, hist = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-12)
    assert its <= 2
    x, its, _ = krylov.gmres(ops.apply_stokes, Pc.apply, b, rtol=1e-12)   # the same with GMRES
    assert its <= 2
    assert np.linalg.norm(b - ops.apply_stokes(x)) <= 1e-12 * np.linalg.norm(b)


def test_exact_block_diagonal_preconditioner_three_iterations():
    """P_D = diag(A, S) with exact blocks: the preconditioned Stokes matrix has the eigenvalues 1 and
    (1 +- sqrt 5) / 2 only (Murphy, Golub, Wathen, SIAM J. Sci. Comput. 21 (2000)), so FGMRES
    converges in at most 3 iterations; with -S instead of S the eigenvalues are 1 and (1 +- i sqrt 3)/2,
    also 3 values, so the sign is pinned by the eigenvalues themselves."""
    p, m, G, ops, F = _problem("cube2")
    A = ops.csr_A().toarray()
    B = ops.csr_B().toarray()
    Ainv = np.linalg.inv(A)
    S = B @ Ainv @ B.T
    Spinv = np.linalg.pinv(S, rcond=1e-10, hermitian=True)
    Pc = krylov.StokesPreconditioner(ops, G, exact_A=lambda t: Ainv @ t, exact_S=lambda r: Spinv @ r,
                                     kind="diagonal")
    b = np.concatenate([F, np.zeros(m.n_p)])
    _, its, _ = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-12)
    assert its == 3
    x, its, _ = krylov.minres(ops.apply_stokes, Pc.apply, b, rtol=1e-12)   # P_D is SPD: MINRES too
    assert its == 3
    assert np.linalg.norm(b - ops.apply_stokes(x)) <= 1e-12 * np.linalg.norm(b)
    # eigenvalues of P_D^-1 K on the free velocity DoFs and the non-constant pressures
    n_u = m.n_u
    free = np.nonzero(~m.dirichlet)[0]
    K = np.block([[A[np.ix_(free, free)], B[:, free].T], [B[:, free], np.zeros((m.n_p, m.n_p))]])
    Pinv = np.block([[np.linalg.inv(A[np.ix_(free, free)]), np.zeros((free.size, m.n_p))],
                     [np.zeros((m.n_p, free.size)), Spinv]])
    ev = np.linalg.eigvals(Pinv @ K)
    ev = ev[np.abs(ev) > 1e-8]                                   # the pressure constant
    targets = np.array([1.0, (1 + 5 ** 0.5) / 2, (1 - 5 ** 0.5) / 2])
    assert np.max(np.min(np.abs(ev[:, None] - targets[None, :]), axis=1)) < 1e-8


def test_block_diagonal_needs_more_iterations_than_triangular():
    """Table 1 context: with the GMG blocks, P_D takes more FGMRES iterations than the
    block-triangular P (the paper reports about twice as many)."""
    p, m, G, ops, F = _problem("cube4")
    b = np.concatenate([F, np.zeros(m.n_p)])
    _, its_t, _ = krylov.fgmres(ops.apply_stokes, krylov.StokesPreconditioner(ops, G).apply, b, rtol=1e-8)
    _, its_d, _ = krylov.fgmres(ops.apply_stokes, krylov.StokesPreconditioner(ops, G, kind="diagonal").apply, b,
                                rtol=1e-8)
    assert its_d > its_t


def test_fgmres_gmg_matches_dense_direct_solve():
    p, m, G, ops, F = _problem("cube4")
    Pc = krylov.StokesPreconditioner(ops, G)
    b = np.concatenate([F, np.zeros(m.n_p)])
    x, its, _ = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-13)
    xd = krylov.dense_stokes_solve(ops, F)
    xz = krylov.zero_mean_pressure(ops, x)
    assert np.abs(xz - xd).max() <= 1e-9 * np.abs(xd).max()
    assert its < 200


def test_vcycle_h_independent_constant_viscosity():
    rates = []
    for n, L in [(4, 3), (8, 4), (16, 5)]:
        mus = [np.ones((n >> (L - 1 - l)) ** 3) for l in range(L)]
        G = gmg.GMG(n, L, mus)
        lev = G.levels[-1]
        b = si.uniform(51, lev.mesh.n_u) * lev.free
        x = np.zeros_like(b)
        r0 = np.linalg.norm(b)
        for _ in range(5):
            x = x + G.vcycle(b - lev.A(x)) * lev.free
        rates.append((np.linalg.norm(b - lev.A(x)) / r0) ** (1 / 5))
    assert max(rates) < 0.15 and max(rates) - min(rates) < 0.05


@pytest.mark.slow
def test_manufactured_solution_convergence_order():
    """Divergence-free u = curl(0, 0, psi), psi = (x(1-x) y(1-y) z(1-z))^2, mu = 1,
    p = cos(pi x) cos(pi y) cos(pi z): velocity L2 error O(h^3), pressure O(h^2)."""
    sym = pytest.importorskip("sympy")
    X, Y, Z = sym.symbols("x y z")
    psi = (X * (1 - X) * Y * (1 - Y) * Z * (1 - Z)) ** 2
    u = [sym.diff(psi, Y), -sym.diff(psi, X), sym.Integer(0)]
    p = sym.cos(sym.pi * X) * sym.cos(sym.pi * Y) * sym.cos(sym.pi * Z)
    f = [-(sym.diff(u[c], X, 2) + sym.diff(u[c], Y, 2) + sym.diff(u[c], Z, 2)) + sym.diff(p, v)
         for c, v in enumerate((X, Y, Z))]
    uf = [sym.lambdify((X, Y, Z), e, "numpy") for e in u]
    ff = [sym.lambdify((X, Y, Z), e, "numpy") for e in f]
    pf = sym.lambdify((X, Y, Z), p, "numpy")
    errs_u, errs_p = [], []
    for n in (2, 4, 8):
        m = mesh.Mesh(n)
        ops = operators.Operators(m, np.ones(m.n_cells))
        q = m.quad_points()
        fq = np.stack([np.broadcast_to(ff[c](q[..., 0], q[..., 1], q[..., 2]), q.shape[:2]) for c in range(3)], -1)
        F = operators.assemble_rhs(m, fq)
        A = ops.csr_A()
        B = ops.csr_B()
        w = sp.csr_matrix(ops.pressure_weights()[None, :])
        K = sp.bmat([[A, B.T, None], [B, None, w.T], [None, w, None]]).tocsc()
        sol = sla.spsolve(K, np.concatenate([F, np.zeros(m.n_p + 1)]))
        uh, ph = sol[:m.n_u], sol[m.n_u:m.n_u + m.n_p]
        pts, wq = fe.quadrature_3d()
        val, _ = fe.q2_3d_tables(pts)
        e2 = 0.0
        for c in range(3):
            uq = uh[m.cell_dofs[:, c * 27:(c + 1) * 27]] @ val.T
            ex = np.broadcast_to(uf[c](q[..., 0], q[..., 1], q[..., 2]), uq.shape)
            e2 += np.sum((uq - ex) ** 2 * wq[None, :]) * m.h ** 3
        errs_u.append(np.sqrt(e2))
        psiq = fe.q1_3d_values(pts)
        pq = ph[m.cell_verts] @ psiq.T
        exq = pf(q[..., 0], q[..., 1], q[..., 2])
        errs_p.append(np.sqrt(np.sum((pq - exq) ** 2 * wq[None, :]) * m.h ** 3))
    rate_u = np.log2(errs_u[-2] / errs_u[-1])
    rate_p = np.log2(errs_p[-2] / errs_p[-1])
    assert rate_u > 2.6, errs_u
    assert rate_p > 1.6, errs_p


def test_galerkin_identity_and_symmetric_vcycle_constant_viscosity():
    """Nested Q2 spaces with exact quadrature and constant mu: the rediscretised coarse
    operator equals P^T A_fine P on free DoFs, and the V(1,1) cycle with equal pre/post
    Chebyshev smoothers is then a symmetric operator."""
    nc = 2
    P = gmg.prolongation(nc)
    cm, fm = mesh.Mesh(nc), mesh.Mesh(2 * nc)
    Af = operators.Operators(fm, np.full(fm.n_cells, 3.0)).csr_A()
    Ac = operators.Operators(cm, np.full(cm.n_cells, 3.0)).csr_A()
    ff, fc = sp.diags((~fm.dirichlet).astype(float)), sp.diags((~cm.dirichlet).astype(float))
    Pf = ff @ P @ fc
    G = (Pf.T @ Af @ Pf).toarray()
    Acf = (fc @ Ac @ fc).toarray()
    assert np.abs(G - Acf).max() < 1e-12 * np.abs(Acf).max()
    n, L = 8, 4
    mus = [np.full((n >> (L - 1 - l)) ** 3, 2.0) for l in range(L)]
    Gm = gmg.GMG(n, L, mus)
    free = Gm.levels[-1].free
    x = si.uniform(61, free.size) * free
    y = si.uniform(62, free.size) * free
    assert abs(Gm.vcycle(x) @ y - x @ Gm.vcycle(y)) < 1e-12 * abs(Gm.vcycle(x) @ y)


def _bicgstab(A, b, rt, steps):
    """Textbook BiCGSTAB (Saad, Iterative Methods, Alg. 7.7) with shadow vector rt, no preconditioner."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = rt @ r
    for _ in range(steps):
        Ap = A @ p
        alpha = rho / (rt @ Ap)
        sv = r - alpha * Ap
        As = A @ sv
        om = (As @ sv) / (As @ As)
        x = x + alpha * p + om * sv
        r = sv - om * As
        rho_new = rt @ r
        p = r + (rho_new / rho) * (alpha / om) * (p - om * Ap)
        rho = rho_new
    return x


def test_idr1_equals_bicgstab():
    """IDR(1) with omega = the local minimiser is BiCGSTAB in exact arithmetic: after 2k operator
    applications its iterate equals BiCGSTAB's after k steps with the same shadow vector."""
    rng = np.random.default_rng(11)
    n = 40
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    P = krylov.idr_shadow_space(n, 1, seed=77)
    for k in (1, 2, 3, 5):
        x_idr, its, _ = krylov.idr_s(lambda v: A @ v, lambda v: v, b, s=1, rtol=1e-30, max_it=2 * k, P=P,
                                     kappa=0.0)
        assert its == 2 * k
        x_bi = _bicgstab(A, b, P[:, 0], k)
        assert np.linalg.norm(x_idr - x_bi) <= 1e-10 * np.linalg.norm(x_bi)


def test_idr_s_finite_termination():
    """IDR(s) needs at most n + n/s operator applications for an n x n system (exact arithmetic);
    with s = 4 on n = 24 it reaches 1e-10 within that bound."""
    rng = np.random.default_rng(12)
    n, s = 24, 4
    A = np.diag(np.linspace(1, 10, n)) + 0.2 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    x, its, _ = krylov.idr_s(lambda v: A @ v, lambda v: v, b, s=s, rtol=1e-10, max_it=400)
    assert its <= n + n // s + 2
    assert np.linalg.norm(A @ x - b) <= 1e-9 * np.linalg.norm(b)


def test_idr_stokes_matches_fgmres():
    """IDR(2) with the block-triangular GMG preconditioner reaches the FGMRES solution (cube4)."""
    p, m, G, ops, F = _problem("cube4")
    Pc = krylov.StokesPreconditioner(ops, G)
    b = np.concatenate([F, np.zeros(m.n_p)])
    xf, _, _ = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-12)
    xi, its, _ = krylov.idr_s(ops.apply_stokes, Pc.apply, b, s=2, rtol=1e-12, max_it=3000)
    xf, xi = krylov.zero_mean_pressure(ops, xf), krylov.zero_mean_pressure(ops, xi)
    assert np.linalg.norm(b - ops.apply_stokes(xi)) <= 1e-10 * np.linalg.norm(b)
    assert np.abs(xi - xf).max() <= 1e-8 * np.abs(xf).max()


def test_gmres_minimises_residual_over_krylov_space():
    """GMRES with a right preconditioner M after k steps from x0 = 0 returns the x in
    M span{b, (A M) b, ..., (A M)^(k-1) b} with the smallest ||b - A x||: brute force by least
    squares over an explicitly built power basis; flexible GMRES with the same linear M agrees."""
    rng = np.random.default_rng(13)
    n = 30
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    M = np.eye(n) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    for k in range(1, 9):
        x, its, _ = krylov.gmres(lambda v: A @ v, lambda v: M @ v, b, rtol=1e-30, restart=k, max_it=k)
        assert its == k
        K = np.empty((n, k))
        K[:, 0] = b
        for i in range(1, k):
            K[:, i] = A @ (M @ K[:, i - 1])
        c = np.linalg.lstsq(A @ M @ K, b, rcond=None)[0]
        x_bf = M @ (K @ c)
        assert np.linalg.norm(x - x_bf) <= 1e-9 * np.linalg.norm(x_bf)
        xf, _, _ = krylov.fgmres(lambda v: A @ v, lambda v: M @ v, b, rtol=1e-30, restart=k, max_it=k)
        assert np.linalg.norm(x - xf) <= 1e-12 * np.linalg.norm(xf)


def test_gmres_restarted_converges_to_true_residual():
    """Restarted GMRES(5) on a system that needs several cycles stops only at the true residual."""
    rng = np.random.default_rng(14)
    n = 60
    A = np.diag(np.linspace(1, 20, n)) + 0.5 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    D = np.diag(1.0 / np.diag(A))
    x, its, hist = krylov.gmres(lambda v: A @ v, lambda v: D @ v, b, rtol=1e-10, restart=5, max_it=2000)
    assert its > 5
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)


def test_gmres_stokes_matches_fgmres():
    """GMRES(50) with the block-triangular GMG preconditioner (a fixed linear map) takes the
    FGMRES iteration count and reaches its solution (cube4)."""
    p, m, G, ops, F = _problem("cube4")
    Pc = krylov.StokesPreconditioner(ops, G)
    b = np.concatenate([F, np.zeros(m.n_p)])
    xf, its_f, _ = krylov.fgmres(ops.apply_stokes, Pc.apply, b, rtol=1e-10)
    xg, its_g, _ = krylov.gmres(ops.apply_stokes, Pc.apply, b, rtol=1e-10)
    assert abs(its_g - its_f) <= 1
    xf, xg = krylov.zero_mean_pressure(ops, xf), krylov.zero_mean_pressure(ops, xg)
    assert np.linalg.norm(b - ops.apply_stokes(xg)) <= 1e-10 * np.linalg.norm(b)
    assert np.abs(xg - xf).max() <= 1e-7 * np.abs(xf).max()


def test_minres_matches_library_and_minimises():
    """MINRES with an SPD preconditioner M = P^-1 after k steps equals scipy's minres after k
    steps, and is the minimiser of ||b - K x||_M over M times the Krylov space of K M from b
    (brute force by least squares over an explicit power basis)."""
    import scipy.sparse.linalg as sla
    rng = np.random.default_rng(15)
    n = 40
    Q = rng.standard_normal((n, n))
    K = (Q + Q.T) / 2 + np.diag(np.linspace(-3, 3, n))          # symmetric indefinite
    L = np.eye(n) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n)
    M = L @ L.T                                                   # SPD
    b = rng.standard_normal(n)
    for k in range(1, 9):
        x, its, _ = krylov.minres(lambda v: K @ v, lambda v: M @ v, b, rtol=1e-30, max_it=k)
        assert its == k
        xs, _ = sla.minres(K, b, M=M, rtol=1e-30, maxiter=k)
        assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)
        U = np.empty((n, k))
        U[:, 0] = M @ b
        for i in range(1, k):
            U[:, i] = M @ (K @ U[:, i - 1])
        c = np.linalg.lstsq(L.T @ K @ U, L.T @ b, rcond=None)[0]
        assert np.linalg.norm(x - U @ c) <= 1e-8 * np.linalg.norm(x)


def test_minres_stokes_block_diagonal():
    """MINRES with the GMG block-diagonal P_D (symmetric: V(1,1) with the same Chebyshev smoother
    both ways, R = P^T, polynomial S_hat^-1) reaches the FGMRES solution on cube4, with an
    iteration count close to FGMRES with the same P_D."""
    p, m, G, ops, F = _problem("cube4")
    b = np.concatenate([F, np.zeros(m.n_p)])
    Pd = krylov.StokesPreconditioner(ops, G, kind="diagonal")
    xf, its_f, _ = krylov.fgmres(ops.apply_stokes, Pd.apply, b, rtol=1e-10)
    xm, its_m, _ = krylov.minres(ops.apply_stokes, Pd.apply, b, rtol=1e-10, max_it=2000)
    assert np.linalg.norm(b - ops.apply_stokes(xm)) <= 1e-10 * np.linalg.norm(b)
    xf, xm = krylov.zero_mean_pressure(ops, xf), krylov.zero_mean_pressure(ops, xm)
    assert np.abs(xm - xf).max() <= 1e-7 * np.abs(xf).max()
    assert its_m <= 1.5 * its_f + 5
