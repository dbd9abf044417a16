// q2_basis.cuh -- reference-cell tables and the sum-factorised cell kernels
// of the Q2-Q1 Stokes operators (Section 2.1, definitions of A, B, B^T, F;
// Section 2.2.2, weighted pressure mass matrix).
//
// Reference cell [0,1]^3. Q2 node (i,j,k) at (i/2, j/2, k/2), local index
// i + 3j + 9k. Gauss point (qx,qy,qz) of the 3-point Gauss-Legendre rule,
// local index qx + 3qy + 9qz. Q1 vertex (i,j,k) in {0,1}^3, index i + 2j + 4k.
//
// The velocity operator of one cube cell of side h with cell viscosity mu is
//   (A u)_(a,c) = mu h sum_q w_q sum_d sigma_cd(q) d_d phi_a(q),
//   sigma = grad_ref u + grad_ref u^T   (= 2 eps in reference coordinates),
// evaluated by sum factorisation in the Gauss-point collocation basis:
// U = (V x V x V) u interpolates the nodal values to the Gauss points, the
// reference gradient along axis d is then the 1D collocation derivative DC
// applied along d, and the transposed sweeps bring the quadrature sums back
// to the nodes. All 1D tables are compile-time constants computed from the
// closed-form Lagrange polynomials and Gauss points, and every loop is fully
// unrolled, so each coefficient (including the quadrature weight of the
// line) is an immediate operand of one FMA.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"

namespace q2 {

// ---------------------------------------------------------------- constants
__host__ __device__ constexpr double csqrt_newton(double x, double g, int it) {
    return it == 0 ? g : csqrt_newton(x, 0.5 * (g + x / g), it - 1);
}
__host__ __device__ constexpr double csqrt(double x) { return csqrt_newton(x, x > 1.0 ? x : 1.0, 64); }

// 3-point Gauss-Legendre on [0,1]: 1/2 -+ sqrt(15)/10, 1/2; weights 5/18, 8/18, 5/18.
__host__ __device__ constexpr double goff() { return csqrt(15.0) / 10.0; }
__host__ __device__ constexpr double gp(int q) { return q == 0 ? 0.5 - goff() : (q == 1 ? 0.5 : 0.5 + goff()); }
__host__ __device__ constexpr double gw(int q) { return q == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }

// Quadratic Lagrange basis on {0, 1/2, 1} and its derivative.
__host__ __device__ constexpr double lag(int m, double x) {
    return m == 0 ? (2.0 * x - 1.0) * (x - 1.0) : (m == 1 ? 4.0 * x * (1.0 - x) : x * (2.0 * x - 1.0));
}
__host__ __device__ constexpr double dlag(int m, double x) {
    return m == 0 ? 4.0 * x - 3.0 : (m == 1 ? 4.0 - 8.0 * x : 4.0 * x - 1.0);
}
// V[q][m] = l_m(g_q): nodal values -> Gauss-point values.
__host__ __device__ constexpr double Vq(int q, int m) { return lag(m, gp(q)); }
// Derivative of the Lagrange polynomials through the Gauss points, at the Gauss points.
__host__ __device__ constexpr double DC(int q, int m) {
    // L_m(x) = prod_{k != m} (x - g_k) / (g_m - g_k)
    return q == m
        ? (m == 0 ? 1.0 / (gp(0) - gp(1)) + 1.0 / (gp(0) - gp(2))
                  : (m == 1 ? 1.0 / (gp(1) - gp(0)) + 1.0 / (gp(1) - gp(2))
                            : 1.0 / (gp(2) - gp(0)) + 1.0 / (gp(2) - gp(1))))
        : ((gp(q) - gp(3 - q - m)) /
           ((gp(m) - gp(q)) * (gp(m) - gp(3 - q - m))));
}
// Q1 basis on [0,1] at Gauss point q.
__host__ __device__ constexpr double Pq(int q, int v) { return v == 0 ? 1.0 - gp(q) : gp(q); }
// 1D Q1 mass matrix on [0,1] by the same quadrature.
__host__ __device__ constexpr double M1(int a, int b) {
    return gw(0) * Pq(0, a) * Pq(0, b) + gw(1) * Pq(1, a) * Pq(1, b) + gw(2) * Pq(2, a) * Pq(2, b);
}

// Linear index of (axis index a, other indices o1 < o2 in axis order).
template <int AX>
__host__ __device__ constexpr int lin(int a, int o1, int o2) {
    return AX == 0 ? a + 3 * o1 + 9 * o2 : (AX == 1 ? o1 + 3 * a + 9 * o2 : o1 + 3 * o2 + 9 * a);
}

// ---------------------------------------------------------------- 1D sweeps
// x <- V x along AX, in place (nodes -> Gauss points).
template <int AX, typename T>
__host__ __device__ __forceinline__ void interp(T* x) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const T a0 = x[lin<AX>(0, o1, o2)], a1 = x[lin<AX>(1, o1, o2)], a2 = x[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int q = 0; q < 3; ++q)
                x[lin<AX>(q, o1, o2)] = T(Vq(q, 0)) * a0 + T(Vq(q, 1)) * a1 + T(Vq(q, 2)) * a2;
        }
}

// x <- V^T x along AX, in place (Gauss-point sums -> nodes).
template <int AX, typename T>
__host__ __device__ __forceinline__ void interpT(T* x) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const T a0 = x[lin<AX>(0, o1, o2)], a1 = x[lin<AX>(1, o1, o2)], a2 = x[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int m = 0; m < 3; ++m)
                x[lin<AX>(m, o1, o2)] = T(Vq(0, m)) * a0 + T(Vq(1, m)) * a1 + T(Vq(2, m)) * a2;
        }
}

// The Gauss points are symmetric about 1/2, so DC(2-q, 2-m) = -DC(q, m): the middle row and
// column of DC are DC(1,0) (1, 0, -1) and DC(0,1) (1, 0, -1) (DC(1,1) = 0), and gw(0) = gw(2).
// The sweeps use that for the middle output (two operations instead of three multiply-adds).

// g (+)= DC x along AX (collocation derivative at the Gauss points).
template <int AX, bool ADD, typename T>
__host__ __device__ __forceinline__ void deriv(const T* x, T* g) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const T a0 = x[lin<AX>(0, o1, o2)], a1 = x[lin<AX>(1, o1, o2)], a2 = x[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const T v = q == 1 ? T(DC(1, 0)) * (a0 - a2)
                                   : T(DC(q, 0)) * a0 + T(DC(q, 1)) * a1 + T(DC(q, 2)) * a2;
                if (ADD) g[lin<AX>(q, o1, o2)] += v; else g[lin<AX>(q, o1, o2)] = v;
            }
        }
}

// w += S * DC^T (W3 .* g) along AX, W3 the 3D quadrature weight of each Gauss point.
template <int AX, int S, typename T>
__host__ __device__ __forceinline__ void derivT_w(const T* g, T* w) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const T a0 = g[lin<AX>(0, o1, o2)], a1 = g[lin<AX>(1, o1, o2)], a2 = g[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const double wl = gw(o1) * gw(o2) * double(S);
                if (m == 1)
                    w[lin<AX>(1, o1, o2)] += T(DC(0, 1) * gw(0) * wl) * (a0 - a2);
                else
                    w[lin<AX>(m, o1, o2)] += T(DC(0, m) * gw(0) * wl) * a0 + T(DC(1, m) * gw(1) * wl) * a1 +
                                             T(DC(2, m) * gw(2) * wl) * a2;
            }
        }
}

// ---------------------------------------------------------------- double-float sweeps
// The same four sweeps for double-float values, each output formed by dot3 / dot3_acc
// (one renormalisation per output instead of one per operation).
template <int AX>
__host__ __device__ __forceinline__ void interp(df64* x) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const df64 a0 = x[lin<AX>(0, o1, o2)], a1 = x[lin<AX>(1, o1, o2)], a2 = x[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int q = 0; q < 3; ++q)
                x[lin<AX>(q, o1, o2)] = dot3(df64(Vq(q, 0)), a0, df64(Vq(q, 1)), a1, df64(Vq(q, 2)), a2);
        }
}
template <int AX>
__host__ __device__ __forceinline__ void interpT(df64* x) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const df64 a0 = x[lin<AX>(0, o1, o2)], a1 = x[lin<AX>(1, o1, o2)], a2 = x[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int m = 0; m < 3; ++m)
                x[lin<AX>(m, o1, o2)] = dot3(df64(Vq(0, m)), a0, df64(Vq(1, m)), a1, df64(Vq(2, m)), a2);
        }
}
template <int AX, bool ADD>
__host__ __device__ __forceinline__ void deriv(const df64* x, df64* g) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const df64 a0 = x[lin<AX>(0, o1, o2)], a1 = x[lin<AX>(1, o1, o2)], a2 = x[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                df64& out = g[lin<AX>(q, o1, o2)];
                if (q == 1)
                    out = ADD ? out + df64(DC(1, 0)) * (a0 - a2) : df64(DC(1, 0)) * (a0 - a2);
                else
                    out = ADD ? dot3_acc(out, df64(DC(q, 0)), a0, df64(DC(q, 1)), a1, df64(DC(q, 2)), a2)
                              : dot3(df64(DC(q, 0)), a0, df64(DC(q, 1)), a1, df64(DC(q, 2)), a2);
            }
        }
}
template <int AX, int S>
__host__ __device__ __forceinline__ void derivT_w(const df64* g, df64* w) {
#pragma unroll
    for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
        for (int o1 = 0; o1 < 3; ++o1) {
            const df64 a0 = g[lin<AX>(0, o1, o2)], a1 = g[lin<AX>(1, o1, o2)], a2 = g[lin<AX>(2, o1, o2)];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const double wl = gw(o1) * gw(o2) * double(S);
                df64& out = w[lin<AX>(m, o1, o2)];
                if (m == 1)
                    out = out + df64(DC(0, 1) * gw(0) * wl) * (a0 - a2);
                else
                    out = dot3_acc(out, df64(DC(0, m) * gw(0) * wl), a0, df64(DC(1, m) * gw(1) * wl), a1,
                                   df64(DC(2, m) * gw(2) * wl), a2);
            }
        }
}

// ---------------------------------------------------------------- cell kernels
// Velocity operator of one reference cell, without the factor mu h:
// in: u[c][a] nodal values (overwritten by their Gauss-point values);
// out: w[c][a] = sum_q w_q sum_d sigma_cd d_d phi_a.
template <typename T>
__host__ __device__ __forceinline__ void cell_A(T (&u)[3][27], T (&w)[3][27]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        interp<0>(u[c]); interp<1>(u[c]); interp<2>(u[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 27; ++a) w[c][a] = T(0);
    T g[27];
    // sigma_cc = 2 d_c U_c
    deriv<0, false>(u[0], g); derivT_w<0, 2>(g, w[0]);
    deriv<1, false>(u[1], g); derivT_w<1, 2>(g, w[1]);
    deriv<2, false>(u[2], g); derivT_w<2, 2>(g, w[2]);
    // sigma_cd = d_d U_c + d_c U_d, c < d, added to rows (c, d) and (d, c)
    deriv<1, false>(u[0], g); deriv<0, true>(u[1], g); derivT_w<1, 1>(g, w[0]); derivT_w<0, 1>(g, w[1]);
    deriv<2, false>(u[0], g); deriv<0, true>(u[2], g); derivT_w<2, 1>(g, w[0]); derivT_w<0, 1>(g, w[2]);
    deriv<2, false>(u[1], g); deriv<1, true>(u[2], g); derivT_w<2, 1>(g, w[1]); derivT_w<1, 1>(g, w[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        interpT<0>(w[c]); interpT<1>(w[c]); interpT<2>(w[c]);
    }
}

// 1D moments of the Q2 basis against the Q1 basis on [0,1], exact by the same
// quadrature: VP(m,v) = int l_m psi_v, DP(m,v) = int l_m' psi_v.
__host__ __device__ constexpr double VP(int m, int v) {
    return gw(0) * lag(m, gp(0)) * Pq(0, v) + gw(1) * lag(m, gp(1)) * Pq(1, v) + gw(2) * lag(m, gp(2)) * Pq(2, v);
}
__host__ __device__ constexpr double DP(int m, int v) {
    return gw(0) * dlag(m, gp(0)) * Pq(0, v) + gw(1) * dlag(m, gp(1)) * Pq(1, v) + gw(2) * dlag(m, gp(2)) * Pq(2, v);
}
// 1D factor of int d_c(phi_m) psi_v along axis AX for velocity component C.
template <int C, int AX>
__host__ __device__ constexpr double XP(int m, int v) { return C == AX ? DP(m, v) : VP(m, v); }

// out_c(i,j,k) (+)= sum_v [int d_c(phi_ijk) psi_v] p_v on the reference cell: the
// tensor product of three 3x2 moment matrices, applied axis by axis (B^T without h).
template <int C, typename T>
__host__ __device__ __forceinline__ void bt_component(const T (&p)[8], T* out) {
    T s1[3][2][2], s2[3][3][2];
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                s1[i][b][d] = T(XP<C, 0>(i, 0)) * p[0 + 2 * b + 4 * d] + T(XP<C, 0>(i, 1)) * p[1 + 2 * b + 4 * d];
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                s2[i][j][d] = T(XP<C, 1>(j, 0)) * s1[i][0][d] + T(XP<C, 1>(j, 1)) * s1[i][1][d];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                out[i + 3 * j + 9 * k] += T(XP<C, 2>(k, 0)) * s2[i][j][0] + T(XP<C, 2>(k, 1)) * s2[i][j][1];
}

// out_v += sum_(c,m) [int d_c(phi_m) psi_v] u_c(m): the transpose (B without h).
template <int C, typename T>
__host__ __device__ __forceinline__ void b_component(const T* u, T (&out)[8]) {
    T t1[3][3][2], t2[3][2][2];
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                t1[i][j][d] = T(XP<C, 2>(0, d)) * u[i + 3 * j] + T(XP<C, 2>(1, d)) * u[i + 3 * j + 9] +
                              T(XP<C, 2>(2, d)) * u[i + 3 * j + 18];
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                t2[i][b][d] = T(XP<C, 1>(0, b)) * t1[i][0][d] + T(XP<C, 1>(1, b)) * t1[i][1][d] +
                              T(XP<C, 1>(2, b)) * t1[i][2][d];
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                out[a + 2 * b + 4 * d] += T(XP<C, 0>(0, a)) * t2[0][b][d] + T(XP<C, 0>(1, a)) * t2[1][b][d] +
                                          T(XP<C, 0>(2, a)) * t2[2][b][d];
}

}  // namespace q2
