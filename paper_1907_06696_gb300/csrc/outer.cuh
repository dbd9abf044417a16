// outer.cuh -- the FP64-interface outer Stokes blocks [A, B^T; B, 0]
// (Section 2.1, eq. stokes_linear_system) in double-float arithmetic with one
// velocity component per thread.
//
// A CTA holds 32 cells and 96 threads; warp c owns velocity component c of
// the 32 cells (lane g = cell g). Per thread, with U_c the Gauss-point values
// of component c and DC_d the collocation derivative along axis d:
//   W_c  = 2 DC_c^T (w .* DC_c U_c)                          (diagonal term)
//        + sum_{d != c} DC_d^T (w .* (DC_d U_c + DC_c U_d))   (symmetric pairs)
// The products DC_d U_c (d != c) and DC_c U_c are exchanged through shared
// memory so that each thread only keeps its own component: the symmetric pair of
// components c and c+1 (mod 3) has one slot, which warp c writes and warp c+1 adds to
// after a barrier (three pair slots instead of six ordered ones: 41.5 KB of shared memory
// per CTA, four CTAs per SM). Then
// out_c = mu h V^T W_c - h^2 (moments of B^T) p, and B's moments of u_c are
// added into the pressure output per component.
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

// Shared exchange buffer: X[c][q][g] = DC_{c+1} U_c + DC_c U_{c+1} (indices mod 3), the
// symmetric pair of components c and c+1, and the diagonal term Dg[c][q][g] = DC_c U_c.
struct OuterShared {
    q2::df64 X[3][27][kOuterCells];
    q2::df64 Dg[3][27][kOuterCells];
};

__host__ __device__ __forceinline__ bool outer_bnd(int g, int M) { return g == 0 || g == M - 1; }

template <int C>
__host__ __device__ __forceinline__ void outer_atomic_add(double* p, double v) {
#ifdef __CUDA_ARCH__
    atomicAdd(p, v);
#else
    *p += v;
#endif
}

// Every thread runs the same code: in its local frame the axes are rotated cyclically so that
// its own velocity component C lies along local axis 0 (local axes = global axes C, C+1, C+2
// mod 3). The operator is invariant under this relabelling (same 1D matrices and weights on every
// axis), so only the addressing differs between the three warps: gathers, scatters and the
// shared-memory exchange map local indices to global ones at run time. This keeps one copy of
// the unrolled double-float code (three copies overflow the instruction cache).
struct OuterFrame {
    int C;            // velocity component of this thread
    int D1, D2;       // global axes of local axes 1 and 2
    size_t sn[3];     // global node strides of local axes 0, 1, 2
    int sq[3];        // global Gauss-point strides (1, 3, 9 rotated)
    int sv[3];        // global Q1-vertex bits (1, 2, 4 rotated)
    int cl[3];        // cell coordinates along the local axes
    int ci, cj, ck;   // global cell coordinates
};

__host__ __device__ __forceinline__ OuterFrame outer_frame(const OuterArgs& a, int C, size_t cell) {
    OuterFrame f;
    f.C = C;
    f.D1 = (C + 1) % 3;
    f.D2 = (C + 2) % 3;
    f.ci = int(cell % a.n);
    f.cj = int((cell / a.n) % a.n);
    f.ck = int(cell / (size_t(a.n) * a.n));
    const size_t ns[3] = {1, size_t(a.M), size_t(a.M) * a.M};
    const int qs[3] = {1, 3, 9}, vs[3] = {1, 2, 4};
    const int cc[3] = {f.ci, f.cj, f.ck};
    const int ax[3] = {C, f.D1, f.D2};
    for (int d = 0; d < 3; ++d) {
        f.sn[d] = ns[ax[d]];
        f.sq[d] = qs[ax[d]];
        f.sv[d] = vs[ax[d]];
        f.cl[d] = cc[ax[d]];
    }
    return f;
}

// Global Gauss-point index of local index q (= qa + 3 qb + 9 qc).
__host__ __device__ __forceinline__ int outer_gq(const OuterFrame& f, int q) {
    return (q % 3) * f.sq[0] + ((q / 3) % 3) * f.sq[1] + (q / 9) * f.sq[2];
}

// Phase 1: gather own component, B moments, interpolation, and the diagonal derivative
// DC_0 U and the cross product DC_1 U (local axes) into shared memory; the other cross product
// DC_2 U is left in T2 for phase 1b.
template <bool DO_A, bool DO_B>
__host__ __device__ __forceinline__ void outer_phase1(const OuterArgs& a, int C, int blk, int g, OuterShared& sh,
                                                      q2::df64 (&U)[27], q2::df64 (&T2)[27]) {
    using q2::df64;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const size_t cell = size_t(blk) * kOuterCells + g;
    const bool valid = cell < cells;
#pragma unroll
    for (int m = 0; m < 27; ++m) U[m] = df64(0);
    if (!(DO_A || DO_B)) return;
    if (valid) {
        const OuterFrame f = outer_frame(a, C, cell);
        const double* src = a.src_u + size_t(C) * a.nodes +
                            (size_t(2 * f.ci) + size_t(a.M) * (size_t(2 * f.cj) + size_t(a.M) * size_t(2 * f.ck)));
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) {
                    const int g0 = 2 * f.cl[0] + aa, g1 = 2 * f.cl[1] + b, g2 = 2 * f.cl[2] + c;
                    if (!(outer_bnd(g0, a.M) || outer_bnd(g1, a.M) || outer_bnd(g2, a.M)))
                        U[aa + 3 * b + 9 * c] = q2::split_double(src[aa * f.sn[0] + b * f.sn[1] + c * f.sn[2]]);
                }
        if (DO_B) {
            df64 bp[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) bp[v] = df64(0);
            q2::b_component<0>(U, bp);
            const int P = a.n + 1;
            const double s = -a.h * a.h;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const int gv = (v & 1) * f.sv[0] + ((v >> 1) & 1) * f.sv[1] + (v >> 2) * f.sv[2];
                const size_t vert = size_t(f.ci + (gv & 1)) +
                                    size_t(P) * (f.cj + ((gv >> 1) & 1) + size_t(P) * (f.ck + (gv >> 2)));
                outer_atomic_add<0>(a.dst_p + vert, s * bp[v].to_double());
            }
        }
    }
    if (!DO_A) return;
    const int D1 = (C + 1) % 3, D2 = (C + 2) % 3;
    const OuterFrame f = outer_frame(a, C, valid ? cell : 0);
    q2::interp<0>(U);
    q2::interp<1>(U);
    q2::interp<2>(U);
    df64 T[27];
    q2::deriv<0, false>(U, T);
#pragma unroll
    for (int q = 0; q < 27; ++q) sh.Dg[C][outer_gq(f, q)][g] = T[q];
    q2::deriv<1, false>(U, T);
#pragma unroll
    for (int q = 0; q < 27; ++q) sh.X[C][outer_gq(f, q)][g] = T[q];     // pair (C, D1): writer
    q2::deriv<2, false>(U, T2);
    (void)D1;
    (void)D2;
}

// Phase 1b (after a barrier): add this thread's DC_2 U (local axis 2 = global axis D2), i.e.
// DC_{D2} U_C, into the slot of the pair (D2, C), which warp D2 wrote with DC_C U_{D2}.
template <bool DO_A>
__host__ __device__ __forceinline__ void outer_phase1b(const OuterArgs& a, int C, int blk, int g, OuterShared& sh,
                                                       const q2::df64 (&T2)[27]) {
    if (!DO_A) return;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const size_t cell = size_t(blk) * kOuterCells + g;
    const OuterFrame f = outer_frame(a, C, cell < cells ? cell : 0);
    const int D2 = f.D2;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        q2::df64& x = sh.X[D2][outer_gq(f, q)][g];
        x = x + T2[q];
    }
}

// Phase 2 (after a barrier): diagonal and symmetric pairs, transposed interpolation,
// B^T moments, scatter into the velocity output.
template <bool DO_A, bool DO_BT>
__host__ __device__ __forceinline__ void outer_phase2(const OuterArgs& a, int C, int blk, int g, const OuterShared& sh,
                                                      q2::df64 (&W)[27]) {
    using q2::df64;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const size_t cell = size_t(blk) * kOuterCells + g;
    if (cell >= cells || !(DO_A || DO_BT)) return;
    const OuterFrame f = outer_frame(a, C, cell);
#pragma unroll
    for (int m = 0; m < 27; ++m) W[m] = df64(0);
    if (DO_A) {
        const int D1 = f.D1, D2 = f.D2;
        df64 T[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) T[q] = sh.Dg[C][outer_gq(f, q)][g];
        q2::derivT_w<0, 2>(T, W);
#pragma unroll
        for (int q = 0; q < 27; ++q) T[q] = sh.X[C][outer_gq(f, q)][g];    // pair (C, D1)
        q2::derivT_w<1, 1>(T, W);
#pragma unroll
        for (int q = 0; q < 27; ++q) T[q] = sh.X[D2][outer_gq(f, q)][g];   // pair (D2, C)
        q2::derivT_w<2, 1>(T, W);
        (void)D1;
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
            const int gv = (v & 1) * f.sv[0] + ((v >> 1) & 1) * f.sv[1] + (v >> 2) * f.sv[2];
            const size_t vert = size_t(f.ci + (gv & 1)) +
                                size_t(P) * (f.cj + ((gv >> 1) & 1) + size_t(P) * (f.ck + (gv >> 2)));
            p8[v] = q2::split_double(s * a.src_p[vert]);
        }
        q2::bt_component<0>(p8, W);
    }
    double* dst = a.dst_u + size_t(C) * a.nodes +
                  (size_t(2 * f.ci) + size_t(a.M) * (size_t(2 * f.cj) + size_t(a.M) * size_t(2 * f.ck)));
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
                const int g0 = 2 * f.cl[0] + aa, g1 = 2 * f.cl[1] + b, g2 = 2 * f.cl[2] + c;
                if (outer_bnd(g0, a.M) || outer_bnd(g1, a.M) || outer_bnd(g2, a.M)) continue;
                outer_atomic_add<0>(dst + aa * f.sn[0] + b * f.sn[1] + c * f.sn[2], W[aa + 3 * b + 9 * c].to_double());
            }
}

}  // namespace stk
