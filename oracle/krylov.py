"""Outer Stokes solve (Section 2.2): block-triangular preconditioner and FGMRES; the
memory-light alternatives of Section 3.4 (GMRES with a fixed preconditioner, IDR(s)); MINRES with
the block-diagonal preconditioner (method (ii)(b) of Section 2.2).

P = [[A, B^T], [0, -S]] (eq. stokes_precond); applying P^-1 to r = [r_u; r_p]:
    z_p = -S_hat^-1 r_p,   z_u = A_hat^-1 (r_u - B^T z_p),
with A_hat^-1 one GMG V-cycle and S_hat^-1 a Jacobi-Chebyshev iteration on the
1/mu-weighted pressure mass matrix M_p (Section 2.2.2). Because S_hat^-1 is an
inner iteration the outer method is flexible GMRES, restart 50 (Section 2.2.2,
Section 3.4). Readings: S_hat^-1 is degree 5 (5 updates, zero initial guess)
on the fixed interval [1/8, 27/8] that bounds the spectrum of diag(M_p)^-1 M_p
for trilinear hexahedra (A. J. Wathen, IMA J. Numer. Anal. 7 (1987), element
eigenvalue bound: 1D element mass [[2,1],[1,2]] h/6 scaled by its diagonal has
eigenvalues 1/2 and 3/2; the tensor product gives [1/8, 27/8]).
"""
from __future__ import annotations

import numpy as np

from .gmg import chebyshev_smooth


class StokesPreconditioner:
    """kind "triangular": P^-1 of eq. stokes_precond (z_p = -S_hat^-1 r_p, z_u = A_hat^-1 (r_u - B^T z_p)).
    kind "diagonal": the block-diagonal P_D = diag(A, S) of Section 2.2 / Table 1
    (z_u = A_hat^-1 r_u, z_p = S_hat^-1 r_p)."""

    def __init__(self, ops_fine, gmg, schur_degree=5, exact_A=None, exact_S=None, kind="triangular"):
        self.ops = ops_fine
        self.gmg = gmg
        self.schur_degree = schur_degree
        self.kind = kind
        self.Mp_dinv = 1.0 / ops_fine.diag_Mp()
        self.exact_A = exact_A        # optional callables replacing the approximations
        self.exact_S = exact_S

    def schur_inverse(self, r_p):
        """S_hat^-1 r_p: Jacobi-Chebyshev on M_p, interval [1/8, 27/8], zero guess; degree 0 is
        S_hat = diag(M_p) itself, the fixed approximation Section 3.4 names for non-flexible GMRES."""
        if self.exact_S is not None:
            return self.exact_S(r_p)
        if self.schur_degree == 0:
            return self.Mp_dinv * r_p
        return chebyshev_smooth(self.ops.apply_Mp, self.Mp_dinv, r_p, None,
                                self.schur_degree, 1.0 / 8.0, 27.0 / 8.0, True)

    def velocity_inverse(self, t):
        if self.exact_A is not None:
            return self.exact_A(t)
        return self.gmg.vcycle(t)

    def apply(self, r):
        n_u = self.ops.mesh.n_u
        r_u, r_p = r[:n_u], r[n_u:]
        if self.kind == "diagonal":
            return np.concatenate([self.velocity_inverse(r_u), self.schur_inverse(r_p)])
        z_p = -self.schur_inverse(r_p)
        t = r_u - self.ops.apply_BT(z_p)
        z_u = self.velocity_inverse(t)
        return np.concatenate([z_u, z_p])


def fgmres(apply_K, apply_Pinv, b, rtol=1e-8, restart=50, max_it=1000, x0=None):
    """Right-preconditioned flexible GMRES (Y. Saad, SIAM J. Sci. Comput. 14 (1993);
    Iterative Methods, Alg. 9.6) with modified Gram-Schmidt and Givens rotations.
    A cycle ends when the recurrence residual |g_{j+1}| <= rtol * ||b||; the solve ends when the
    true residual b - K x, recomputed after the cycle, meets the tolerance too (else a new cycle
    starts from it). Returns (x, iterations, list of relative residual estimates)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    history = []
    its = 0
    if bnorm == 0.0:
        return x, 0, [0.0]
    while its < max_it:
        r = b - apply_K(x)
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= rtol * bnorm:
            break
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = apply_Pinv(V[j])
            w = apply_K(Z[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            denom = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / denom
            sn[j] = H[j + 1, j] / denom
            H[j, j] = denom
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or its >= max_it:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Z[:k].T @ y
        # the loop head recomputes b - K x: the solve ends when the true residual meets rtol
    return x, its, history


def gmres(apply_K, apply_Pinv, b, rtol=1e-8, restart=50, max_it=1000, x0=None):
    """Right-preconditioned GMRES(restart) (Y. Saad, Iterative Methods for Sparse Linear Systems,
    2nd ed., Alg. 9.5) with modified Gram-Schmidt and Givens rotations: the Arnoldi basis V of
    K P^-1 is kept, the preconditioned vectors are not, and a cycle ends with x += P^-1 (V y).
    This needs P^-1 to be one fixed linear map, which holds for the block-triangular P with a
    V-cycle (Chebyshev smoothing on fixed intervals, exact coarse solve) and a fixed-degree
    Chebyshev S_hat^-1; it halves the Krylov memory of flexible GMRES (Section 3.4).
    A cycle ends when the recurrence residual |g_{j+1}| <= rtol ||b||; the next cycle starts
    from the true residual b - K x and the solve stops only when that meets the tolerance (a
    P^-1 in lower precision makes the final update differ slightly from the combination the
    recurrence assumed). Returns (x, Arnoldi iterations, list of relative residual estimates)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    history = []
    its = 0
    if bnorm == 0.0:
        return x, 0, [0.0]
    while True:
        r = b - apply_K(x)
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= rtol * bnorm or its >= max_it:
            break
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = apply_K(apply_Pinv(V[j]))
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            its += 1
            k = j + 1
            # least-squares residual of the (j+2) x (j+1) Hessenberg problem, by Givens rotations
            R, gk = _givens_triangularise(H[:k + 1, :k], g[:k + 1])
            history.append(abs(gk[k]) / bnorm)
            if abs(gk[k]) <= rtol * bnorm or H[j + 1, j] == 0.0 or its >= max_it:
                break
        R, gk = _givens_triangularise(H[:k + 1, :k], g[:k + 1])
        y = np.linalg.solve(np.triu(R[:k, :k]), gk[:k])
        x = x + apply_Pinv(V[:k].T @ y)
    return x, its, history


def _givens_triangularise(H, g):
    """Applies the Givens rotations that make the (k+1) x k upper Hessenberg H upper triangular
    to H and g; returns the rotated copies (the last entry of g is the least-squares residual)."""
    R = H.copy()
    g = g.copy()
    k = R.shape[1]
    for j in range(k):
        d = np.hypot(R[j, j], R[j + 1, j])
        c, s = R[j, j] / d, R[j + 1, j] / d
        top = c * R[j, :] + s * R[j + 1, :]
        R[j + 1, :] = -s * R[j, :] + c * R[j + 1, :]
        R[j, :] = top
        g[j], g[j + 1] = c * g[j], -s * g[j]
    return R, g


def minres(apply_K, apply_Pinv, b, rtol=1e-8, max_it=1000, x0=None):
    """Preconditioned MINRES (C. C. Paige, M. A. Saunders, SIAM J. Numer. Anal. 12 (1975)) for a
    symmetric K with a symmetric positive definite preconditioner P (here P_D = diag(A_hat, S_hat),
    method (ii)(b) of Section 2.2): the Lanczos process of P^-1 K in the P-inner product, its
    tridiagonal matrix reduced by Givens rotations, x updated every step along directions w
    (three-term recurrence). Short recurrences: a fixed number of vectors.
    MINRES minimises the P^-1-norm of the residual; the 2-norm residual r = b - K x is carried
    along by the same recurrences (K w from K z) and the solve stops when ||r|| <= rtol ||b||, then
    verifies it against b - K x; if the carried residual drifted, MINRES restarts from x (at most
    10 times). Returns (x, iterations, list of relative residuals)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    hist = []
    its = 0
    if bnorm == 0.0:
        return x, 0, [0.0]
    tol = rtol * bnorm
    for _ in range(11):
        r = b - apply_K(x)
        hist.append(np.linalg.norm(r) / bnorm)
        if np.linalg.norm(r) <= tol or its >= max_it:
            break
        x, its = _minres_cycle(apply_K, apply_Pinv, x, r, tol, its, max_it, hist, bnorm)
    return x, its, hist


def _minres_cycle(apply_K, apply_Pinv, x, r, tol, its, max_it, hist, bnorm):
    """MINRES from (x, r = b - K x) until the carried residual meets tol or max_it is reached."""
    n = x.shape[0]
    v_old = np.zeros(n)                 # Lanczos vectors of the unpreconditioned space, scaled by gamma
    v = r.copy()
    z = apply_Pinv(v)
    gamma_old, gamma = 1.0, np.sqrt(v @ z)
    eta = gamma                         # P^-1-norm of the residual, with sign
    c_old, c, s_old, s = 1.0, 1.0, 0.0, 0.0
    w_old, w = np.zeros(n), np.zeros(n)     # search directions
    Kw_old, Kw = np.zeros(n), np.zeros(n)   # K times them
    r = r.copy()
    while its < max_it:
        z = z / gamma
        q = apply_K(z)
        delta = q @ z
        v_new = q - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = apply_Pinv(v_new)
        gamma_new = np.sqrt(v_new @ z_new)
        # new column of the tridiagonal matrix: rotate by the two previous rotations, then
        # annihilate gamma_new with a new one
        a0 = c * delta - c_old * s * gamma
        a1 = np.hypot(a0, gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_old, s_old = c, s
        c, s = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        Kw_new = (q - a3 * Kw_old - a2 * Kw) / a1
        x = x + (c * eta) * w_new
        r = r - (c * eta) * Kw_new
        eta = -s * eta
        its += 1
        v_old, v = v, v_new
        z = z_new
        gamma_old, gamma = gamma, gamma_new
        w_old, w = w, w_new
        Kw_old, Kw = Kw, Kw_new
        rn = np.linalg.norm(r)
        hist.append(rn / bnorm)
        if rn <= tol or gamma == 0.0:
            break
    return x, its


def zero_mean_pressure(ops, up):
    """Subtract the integral mean of the pressure (the constant pressure is the
    null space of the all-Dirichlet Stokes operator)."""
    n_u = ops.mesh.n_u
    w = ops.pressure_weights()
    out = up.copy()
    out[n_u:] -= (w @ up[n_u:]) / w.sum()
    return out


def dense_stokes_solve(ops, F):
    """Direct solve of [[A_c, B^T], [B, 0]] [u; p] = [F; 0] with the pressure mean
    fixed to zero by a bordering row (small meshes only)."""
    A = ops.csr_A().toarray()
    B = ops.csr_B().toarray()
    w = ops.pressure_weights()
    n_u, n_p = A.shape[0], B.shape[0]
    K = np.zeros((n_u + n_p + 1, n_u + n_p + 1))
    K[:n_u, :n_u] = A
    K[:n_u, n_u:n_u + n_p] = B.T
    K[n_u:n_u + n_p, :n_u] = B
    K[n_u + n_p, n_u:n_u + n_p] = w
    K[n_u:n_u + n_p, n_u + n_p] = w
    rhs = np.zeros(n_u + n_p + 1)
    rhs[:n_u] = F
    sol = np.linalg.solve(K, rhs)
    return sol[:n_u + n_p]


def idr_shadow_space(n, s, seed=1907100):
    """The s shadow vectors of IDR(s): splitmix64 uniforms u01 - 1/2 (seed + i for column i),
    orthonormalised by Gram-Schmidt, as columns of an (n, s) array."""
    import sinker_inputs
    P = np.stack([sinker_inputs.uniform01(seed + i, n) - 0.5 for i in range(s)], axis=1)
    for i in range(s):
        for j in range(i):
            P[:, i] -= (P[:, j] @ P[:, i]) * P[:, j]
        P[:, i] /= np.linalg.norm(P[:, i])
    return P


def idr_s(apply_K, apply_Pinv, b, s=2, rtol=1e-8, max_it=1000, x0=None, P=None, kappa=0.7):
    """IDR(s) with bi-orthogonalisation and a preconditioner (M. B. van Gijzen, P. Sonneveld,
    "Algorithm 913: an elegant IDR(s) variant that efficiently exploits bi-orthogonality
    properties", ACM TOMS 38 (2011)); the residual-smoothing-free variant with the "maintain the
    convergence" choice of omega (|cos| of the angle below kappa is lifted to kappa).
    The memory-light alternative to FGMRES of Section 3.4: 3s + 4 vectors.
    Stops when the recursively updated residual satisfies ||r|| <= rtol ||b||; if the true
    residual b - K x is then still above the tolerance (the recursion drifts from it, more so
    with an inexact preconditioner), IDR restarts from x with r = b - K x (at most 10 times).
    Returns (x, preconditioned operator applications, list of relative residuals)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if P is None:
        P = idr_shadow_space(n, s)
    its = 0
    hist = []
    tol = rtol * bnorm
    for _ in range(11):
        r = b - apply_K(x)
        hist.append(np.linalg.norm(r) / bnorm)
        if np.linalg.norm(r) <= tol or its >= max_it:
            break
        x, its = _idr_cycle(apply_K, apply_Pinv, b, x, r, P, s, tol, its, max_it, kappa, hist)
    return x, its, hist


def _idr_cycle(apply_K, apply_Pinv, b, x, r, P, s, tol, its, max_it, kappa, hist):
    """IDR(s) from (x, r) until the recursive residual meets tol or max_it is reached."""
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    G = np.zeros((n, s))
    U = np.zeros((n, s))
    Ms = np.eye(s)
    om = 1.0
    while np.linalg.norm(r) > tol and its < max_it:
        f = P.T @ r
        for k in range(s):
            # v = r - G[:, k:] c with M[k:, k:] c = f[k:] (lower triangular)
            c = np.linalg.solve(Ms[k:, k:], f[k:])
            v = r - G[:, k:] @ c
            v = apply_Pinv(v)
            U[:, k] = U[:, k:] @ c + om * v
            G[:, k] = apply_K(U[:, k])
            its += 1
            for i in range(k):                       # G_k orthogonal to p_0 .. p_{k-1}
                alpha = (P[:, i] @ G[:, k]) / Ms[i, i]
                G[:, k] -= alpha * G[:, i]
                U[:, k] -= alpha * U[:, i]
            Ms[k:, k] = P[:, k:].T @ G[:, k]
            beta = f[k] / Ms[k, k]
            r = r - beta * G[:, k]
            x = x + beta * U[:, k]
            hist.append(np.linalg.norm(r) / bnorm)
            if np.linalg.norm(r) <= tol or its >= max_it:
                break
            if k + 1 < s:
                f[k + 1:] = f[k + 1:] - beta * Ms[k + 1:, k]
        if np.linalg.norm(r) <= tol or its >= max_it:
            break
        # dimension-reduction step
        v = apply_Pinv(r)
        t = apply_K(v)
        its += 1
        tt, tr = t @ t, t @ r
        om = tr / tt
        rho = abs(tr) / (np.sqrt(tt) * np.linalg.norm(r))
        if rho < kappa:
            om = om * kappa / rho
        x = x + om * v
        r = r - om * t
        hist.append(np.linalg.norm(r) / bnorm)
    return x, its
