// outer.cuh -- the FP64-interface outer Stokes blocks [A, B^T; B, 0]
// (Section 2.1, eq. stokes_linear_system) in double-float arithmetic with one
// velocity component per thread.
//
// A CTA holds 32 cells and 96 threads; warp c owns velocity component c of
// the 32 cells (lane g = cell g). Per thread, with U_c the Gauss-point values
// of component c and DC_d the collocation derivative along axis d:
//   W_c  = 2 DC_c^T (w .* DC_c U_c)                          (diagonal term)
//        + sum_{d != c} DC_d^T (w .* (DC_d U_c + DC_c U_d))   (symmetric pairs)
// The products DC_d U_c (d != c) are exchanged through shared memory so
// that each thread only keeps its own component: three 27-vectors of
// double-floats. Then out_c = mu h V^T W_c - h^2 (moments of B^T) p, and B's
// moments of u_c are added into the pressure output per component.
// The phases are plain functions of the thread index so that a host program
// can run them and compare with the FP64 kernel.
#pragma once

#include "df64.cuh"
#include "q2_basis.cuh"

namespace stk {

constexpr int kOuterCells = 32;       // cells per CTA
constexpr int kOuterThreads = 96;     // 3 components x 32 cells

struct OuterArgs {
    int n, M;
    size_t nodes;
    double h;
    const double* mu;
    const double* src_u;
    const double* src_p;
    double* dst_u;
    double* dst_p;
};

// Shared exchange buffer: X[pair(c,d)][q][g], pair over the 6 ordered pairs c != d.
struct OuterShared {
    q2::df64 X[6][27][kOuterCells];
};

__host__ __device__ __forceinline__ constexpr int outer_pair(int c, int d) { return 2 * c + (d > c ? d - 1 : d); }

__host__ __device__ __forceinline__ bool outer_bnd(int g, int M) { return g == 0 || g == M - 1; }

template <int C>
__host__ __device__ __forceinline__ void outer_atomic_add(double* p, double v) {
#ifdef __CUDA_ARCH__
    atomicAdd(p, v);
#else
    *p += v;
#endif
}

// Phase 1 of thread (C, g): gather, B moments, interpolation, diagonal term, and the two
// cross products DC_d U_C for d != C into shared memory. U and W stay in registers
// (passed back to phase 2 by reference).
template <int C, bool DO_A, bool DO_B>
__host__ __device__ __forceinline__ void outer_phase1(const OuterArgs& a, int blk, int g, OuterShared& sh,
                                                      q2::df64 (&U)[27], q2::df64 (&W)[27]) {
    using q2::df64;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const size_t cell = size_t(blk) * kOuterCells + g;
    const bool valid = cell < cells;
#pragma unroll
    for (int m = 0; m < 27; ++m) { U[m] = df64(0); W[m] = df64(0); }
    if (!(DO_A || DO_B)) return;
    if (valid) {
        const int ci = int(cell % a.n), cj = int((cell / a.n) % a.n), ck = int(cell / (size_t(a.n) * a.n));
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                    if (!(outer_bnd(gi, a.M) || outer_bnd(gj, a.M) || outer_bnd(gk, a.M)))
                        U[i + 3 * j + 9 * k] =
                            q2::from_double(a.src_u[C * a.nodes + size_t(gi) + size_t(a.M) * (gj + size_t(a.M) * gk)]);
                }
        if (DO_B) {
            df64 bp[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) bp[v] = df64(0);
            q2::b_component<C>(U, bp);
            const int P = a.n + 1;
            const double s = -a.h * a.h;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const size_t vert =
                    size_t(ci + (v & 1)) + size_t(P) * (cj + ((v >> 1) & 1) + size_t(P) * (ck + (v >> 2)));
                outer_atomic_add<C>(a.dst_p + vert, s * bp[v].to_double());
            }
        }
    }
    if (!DO_A) return;
    q2::interp<0>(U);
    q2::interp<1>(U);
    q2::interp<2>(U);
    df64 T[27];
    q2::deriv<C, false>(U, T);
    q2::derivT_w<C, 2>(T, W);
    constexpr int D0 = C == 0 ? 1 : 0, D1 = C == 2 ? 1 : 2;
    q2::deriv<D0, false>(U, T);
#pragma unroll
    for (int q = 0; q < 27; ++q) sh.X[outer_pair(C, D0)][q][g] = T[q];
    q2::deriv<D1, false>(U, T);
#pragma unroll
    for (int q = 0; q < 27; ++q) sh.X[outer_pair(C, D1)][q][g] = T[q];
}

// Phase 2 (after a barrier): finish the symmetric pairs, transposed interpolation,
// B^T moments, scatter into the velocity output.
template <int C, bool DO_A, bool DO_BT>
__host__ __device__ __forceinline__ void outer_phase2(const OuterArgs& a, int blk, int g, const OuterShared& sh,
                                                      q2::df64 (&W)[27]) {
    using q2::df64;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const size_t cell = size_t(blk) * kOuterCells + g;
    if (cell >= cells || !(DO_A || DO_BT)) return;
    const int ci = int(cell % a.n), cj = int((cell / a.n) % a.n), ck = int(cell / (size_t(a.n) * a.n));
    if (DO_A) {
        constexpr int D0 = C == 0 ? 1 : 0, D1 = C == 2 ? 1 : 2;
        df64 T[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) T[q] = sh.X[outer_pair(C, D0)][q][g] + sh.X[outer_pair(D0, C)][q][g];
        q2::derivT_w<D0, 1>(T, W);
#pragma unroll
        for (int q = 0; q < 27; ++q) T[q] = sh.X[outer_pair(C, D1)][q][g] + sh.X[outer_pair(D1, C)][q][g];
        q2::derivT_w<D1, 1>(T, W);
        q2::interpT<0>(W);
        q2::interpT<1>(W);
        q2::interpT<2>(W);
        const df64 sA = q2::from_double(a.mu[cell] * a.h);
#pragma unroll
        for (int m = 0; m < 27; ++m) W[m] *= sA;
    }
    if (DO_BT) {
        const int P = a.n + 1;
        const double s = -a.h * a.h;
        df64 p8[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const size_t vert = size_t(ci + (v & 1)) + size_t(P) * (cj + ((v >> 1) & 1) + size_t(P) * (ck + (v >> 2)));
            p8[v] = q2::from_double(s * a.src_p[vert]);
        }
        q2::bt_component<C>(p8, W);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                if (outer_bnd(gi, a.M) || outer_bnd(gj, a.M) || outer_bnd(gk, a.M)) continue;
                outer_atomic_add<C>(a.dst_u + C * a.nodes + size_t(gi) + size_t(a.M) * (gj + size_t(a.M) * gk),
                                    W[i + 3 * j + 9 * k].to_double());
            }
}

}  // namespace stk
