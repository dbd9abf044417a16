// pressure.cuh -- per-thread bodies of the pressure-side gathers of the preconditioner on uniform
// meshes (ops.cu kernels k_bt_gather and k_schur_cheb): B^T p as a tensor product of assembled 1D
// moment operators (Section 2.1, definition of B), and one Jacobi-Chebyshev step of S_hat^-1 on
// the 1/mu-weighted pressure mass matrix (Section 2.2.2) with M_p gathered per vertex. Both run
// their products in double-float on the FP32 pipes. Plain functions of the thread's indices, so
// that a host program can run them node by node and vertex by vertex.
#pragma once

#include "df64.cuh"
#include "q2_basis.cuh"

namespace stk {

// ---- B^T. B^T carries no viscosity, so component c of B^T p is -h^2 (X_2 x X_1 x X_0) p with X_d
// the 1D moment operator assembled over the cells along axis d (DP, the moments of the Q2 basis
// derivatives against the Q1 basis, along axis c; VP, those of the basis itself, along the other
// two). An interior Q2 node 2e (a vertex) has the row (XP(2,0), XP(2,1) + XP(0,0), XP(0,1)) at
// vertices e-1, e, e+1, an interior node 2e+1 the row (XP(1,0), XP(1,1)) at e, e+1. For the line
// (J, K) of component C: t_e = sum X_1[J][b] X_2[K][k] p(e, b, k), then the x-nodes 2e and 2e+1
// from t_{e-1}, t_e, t_{e+1}; boundary nodes get 0, as in the cell kernels.

// entry of X_0 (axis 0) in row i at vertex a, for the rows of vertex e (i = 2e, 2e + 1)
template <int C>
__host__ __device__ __forceinline__ double bt_x_row(int i, int a, int e) {
    constexpr bool D = C == 0;
    auto xp = [](int m, int v) { return D ? q2::DP(m, v) : q2::VP(m, v); };
    if (i & 1) return a == e ? xp(1, 0) : (a == e + 1 ? xp(1, 1) : 0.0);
    return a == e - 1 ? xp(2, 0) : (a == e ? xp(2, 1) + xp(0, 0) : (a == e + 1 ? xp(0, 1) : 0.0));
}

// row i of X_AX (interior i) over the vertices i/2 - 1, i/2, i/2 + 1
template <int C, int AX>
__host__ __device__ __forceinline__ void bt_row(int i, double (&w)[3]) {
    constexpr bool D = C == AX;
    auto xp = [](int m, int v) { return D ? q2::DP(m, v) : q2::VP(m, v); };
    if (i & 1) {   // vertices i/2, i/2 + 1
        w[0] = 0.0;
        w[1] = xp(1, 0);
        w[2] = xp(1, 1);
    } else {
        w[0] = xp(2, 0);
        w[1] = xp(2, 1) + xp(0, 0);
        w[2] = xp(0, 1);
    }
}

// weight q (= b-slot + 3 k-slot) of the interior line (J, K)
template <int C>
__host__ __device__ __forceinline__ q2::df64 bt_weight(int J, int K, int q) {
    double wy[3], wz[3];
    bt_row<C, 1>(J, wy);
    bt_row<C, 2>(K, wz);
    return q2::split_double(wy[q % 3] * wz[q / 3]);
}

// t_e of the interior line (J, K) from the line's 9 weights w
template <int C>
__host__ __device__ __forceinline__ q2::df64 bt_t(int n, const double* __restrict__ p, int J, int K, int e,
                                                   const q2::df64* w) {
    const int P = n + 1;
    const int by = J / 2 - 1, bz = K / 2 - 1;
    q2::df64 acc;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int b = by + q % 3, k = bz + q / 3;
        if (b < 0 || b >= P || k < 0 || k >= P) continue;   // zero weights only
        q2::mac(acc, w[q], q2::split_double(p[size_t(e) + size_t(P) * (b + size_t(P) * k)]));
    }
    q2::renorm(acc);
    return acc;
}

// the x-nodes 2e and 2e + 1 (e < n) of the interior line whose first node is o, times s = -h^2
template <int C>
__host__ __device__ __forceinline__ void bt_out(int n, double s, double* __restrict__ o, int e, const q2::df64* t) {
    using q2::df64;
    const int M = 2 * n + 1;
    const int i0 = 2 * e;
    if (i0 == 0 || i0 == M - 1) {
        o[i0] = 0.0;
    } else {
        df64 v;
        q2::mac(v, df64(bt_x_row<C>(i0, e - 1, e)), t[e - 1]);
        q2::mac(v, df64(bt_x_row<C>(i0, e, e)), t[e]);
        q2::mac(v, df64(bt_x_row<C>(i0, e + 1, e)), t[e + 1]);
        q2::renorm(v);
        o[i0] = s * v.to_double();
    }
    if (e < n) {
        df64 v;
        q2::mac(v, df64(bt_x_row<C>(i0 + 1, e, e)), t[e]);
        q2::mac(v, df64(bt_x_row<C>(i0 + 1, e + 1, e)), t[e + 1]);
        q2::renorm(v);
        o[i0 + 1] = s * v.to_double();
    }
}

// ---- S_hat^-1 step at pressure vertex vtx:
//   d' = c1 d + c2 D^-1 (r - M_p z),  z' = z + d'   (into the other buffers of the pairs).
// (M_p z)_v sums the element products of the up to 8 cells around v, s_K sum_w m(v, w) z_w with
// s_K = h^3 / mu_K and m = M1 x M1 x M1 (M1 the 1D Q1 mass matrix on [0,1]); the 27 neighbouring
// values are split once. In FP64 the 64 multiply-adds per vertex would bind the kernel to the FP64
// pipe (1/72 of the FP32 rate).
__host__ __device__ __forceinline__ void schur_vertex(int n, const double* __restrict__ scale,
                                                      const double* __restrict__ r, const double* __restrict__ dinv,
                                                      const double* __restrict__ z, const double* __restrict__ d,
                                                      double* __restrict__ z_new, double* __restrict__ d_new,
                                                      double c1, double c2, size_t vtx) {
    using q2::df64;
    const int P = n + 1;
    const int vi = int(vtx % P), vj = int((vtx / P) % P), vk = int(vtx / (size_t(P) * P));
    df64 zz[3][3][3];   // [k][j][i], the vertex (vi + i - 1, vj + j - 1, vk + k - 1)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int wi = vi + i - 1, wj = vj + j - 1, wk = vk + k - 1;
                const bool in = wi >= 0 && wj >= 0 && wk >= 0 && wi < P && wj < P && wk < P;
                zz[k][j][i] = in ? q2::split_double(z[size_t(wi) + size_t(P) * (wj + size_t(P) * wk)]) : df64();
            }
    df64 acc;
#pragma unroll
    for (int ck = 0; ck < 2; ++ck)
#pragma unroll
        for (int cj = 0; cj < 2; ++cj)
#pragma unroll
            for (int ci = 0; ci < 2; ++ci) {
                // cell (vi - 1 + ci, ...): v is its local corner (1 - ci, 1 - cj, 1 - ck)
                const int gi = vi - 1 + ci, gj = vj - 1 + cj, gk = vk - 1 + ck;
                if (gi < 0 || gj < 0 || gk < 0 || gi >= n || gj >= n || gk >= n) continue;
                df64 inner;
#pragma unroll
                for (int wk = 0; wk < 2; ++wk)
#pragma unroll
                    for (int wj = 0; wj < 2; ++wj)
#pragma unroll
                        for (int wi = 0; wi < 2; ++wi) {
                            const double m = q2::M1(1 - ci, wi) * q2::M1(1 - cj, wj) * q2::M1(1 - ck, wk);
                            q2::mac(inner, df64(m), zz[ck + wk][cj + wj][ci + wi]);
                        }
                q2::renorm(inner);
                acc = acc + q2::split_double(scale[size_t(gi) + size_t(n) * (gj + size_t(n) * gk)]) * inner;
            }
    const double mz = acc.to_double();
    const double dn = (c1 != 0.0 ? c1 * d[vtx] : 0.0) + c2 * (dinv[vtx] * (r[vtx] - mz));
    d_new[vtx] = dn;
    z_new[vtx] = z[vtx] + dn;
}

}  // namespace stk
