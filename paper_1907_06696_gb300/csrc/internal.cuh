// internal.cuh -- launchers shared by the translation units of the library.
// Not part of the public ABI (include/stokes.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace stk {

// Geometry of one uniform level: n cells per axis, Q2 lattice M = 2n+1.
struct LevelGeom {
    int n;
    int M;
    size_t nodes;    // M^3
    size_t n_u;      // 3 M^3
    size_t cells;    // n^3
    size_t n_p;      // (n+1)^3
    double h;
};

inline LevelGeom make_geom(int n) {
    LevelGeom g;
    g.n = n;
    g.M = 2 * n + 1;
    g.nodes = size_t(g.M) * g.M * g.M;
    g.n_u = 3 * g.nodes;
    g.cells = size_t(n) * n * n;
    g.n_p = size_t(n + 1) * (n + 1) * (n + 1);
    g.h = 1.0 / n;
    return g;
}

// ---- operators (ops.cu) ----
// Finest-level FP64 blocks. Flags select the parts of [[A, B^T], [B, 0]]:
// the u-part of dst gets A u (DO_A) + B^T p (DO_BT), the p-part gets B u (DO_B).
// src_u / src_p may be null when unused; dst parts are overwritten.
// df64 selects double-float arithmetic on the FP32 pipes (q2::df64) instead of native FP64.
cudaError_t launch_stokes_blocks(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                                 double* dst_u, double* dst_p, bool do_a, bool do_bt, bool do_b, bool df64,
                                 cudaStream_t s);
// The same blocks in double-float arithmetic, one velocity component per thread (outer.cu).
cudaError_t launch_outer_df64(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                              double* dst_u, double* dst_p, bool do_a, bool do_bt, bool do_b, cudaStream_t s);
// The whole outer operator [A B^T; B 0] to FP64 accuracy on the tensor cores, by exact integer
// products with fixed-point digit slices (outer_tc.cu; the caller clears dst_u and dst_p and copies
// the constrained rows afterwards). outer_tc_setup builds the f16 table (outer_tc_table_bytes()
// bytes) and sets the kernel's shared-memory size; flag != 0 afterwards if an entry is not exact.
size_t outer_tc_table_bytes();
cudaError_t outer_tc_setup(void* table, int* flag, cudaStream_t s);
cudaError_t launch_outer_tc(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                            double* dst_u, double* dst_p, const void* table, unsigned* status,
                            unsigned long long wait_ns, cudaStream_t s);
// dst = M_p src (weighted pressure mass, FP64).
cudaError_t launch_mass_p(const LevelGeom& g, const double* mu, const double* src, double* dst, cudaStream_t s);
// out = B^T p on the uniform mesh (velocity boundary nodes 0), gathered per node pair; no atomics
cudaError_t launch_bt_gather(const LevelGeom& g, const double* p, double* out, cudaStream_t s);
// scale[cell] = h^3 / mu[cell]
cudaError_t launch_mass_scale(const LevelGeom& g, const double* mu, double* scale, cudaStream_t s);
// One Chebyshev step of S_hat^-1 with M_p gathered per vertex (double-float products):
// d_new = c1 d + c2 dinv (r - M_p z), z_new = z + d_new; z_new, d_new must not alias z, d.
cudaError_t launch_schur_cheb(const LevelGeom& g, const double* scale, const double* r, const double* dinv,
                              const double* z, const double* d, double* z_new, double* d_new, double c1, double c2,
                              cudaStream_t s);
// diag(M_p) and int psi_l (pressure weights), FP64.
cudaError_t launch_mass_p_diag(const LevelGeom& g, const double* mu, double* diag, double* weights,
                               cudaStream_t s);
// Diagonal of the reference cell operator (81 values, mu = h = 1).
cudaError_t launch_ref_diag(double* ref_diag81, cudaStream_t s);
// dinv = 1 / diag(A_c) on free DoFs, 0 on constrained ones.
cudaError_t launch_inv_diag(const LevelGeom& g, const double* mu, const double* ref_diag81, double* dinv,
                            cudaStream_t s);
// Cell viscosity on the finest level from the sinker formula (harmonic average).
cudaError_t launch_mu_sinker(const LevelGeom& g, const double* centres, int n_sinkers, double mu_min,
                             double mu_max, double delta, double omega, double* mu, cudaStream_t s);
// Cell viscosity from values at the quadrature points (harmonic average).
cudaError_t launch_mu_from_q(const LevelGeom& g, const double* mu_q, double* mu, cudaStream_t s);
// Parent viscosity = mean of 8 children.
cudaError_t launch_mu_restrict(const LevelGeom& coarse, const double* mu_fine, double* mu_coarse, cudaStream_t s);
// F = int phi . f, f = (0,0,beta(X-1)) at the Gauss points (accumulates into zeroed F).
cudaError_t launch_rhs_sinker(const LevelGeom& g, const double* centres, int n_sinkers, double delta,
                              double omega, double beta, double* F, cudaStream_t s);

// ---- vectors and transfers (vec.cu) ----
template <typename T>
cudaError_t launch_prolongate(const LevelGeom& fine, const T* coarse, T* finev, bool add, cudaStream_t s);
// coarse = P^T fine; deterministic: a gather per coarse node (fixed summation order), else per
// coarse cell with atomic adds.
template <typename T>
cudaError_t launch_restrict(const LevelGeom& fine, const T* finev, T* coarse, cudaStream_t s, bool deterministic = false);

// Chebyshev update: r = Dinv (b - Ax) (Ax may be null = 0); d = c1 d + c2 r; x = (x_valid ? x : 0) + d.
template <typename T>
cudaError_t launch_cheb_update(size_t n, const T* b, const T* Ax, const T* dinv, T* d, T* x, double c1, double c2,
                               bool x_valid, cudaStream_t s);
// r = b - Ax
template <typename T>
cudaError_t launch_residual(size_t n, const T* b, const T* Ax, T* r, cudaStream_t s);
// Zero the velocity entries on boundary nodes of a level vector.
template <typename T>
cudaError_t launch_zero_boundary(const LevelGeom& g, T* x, cudaStream_t s);
// out = in on boundary nodes (identity rows).
template <typename T>
cudaError_t launch_copy_boundary(const LevelGeom& g, const T* in, T* out, cudaStream_t s);
// Casts with the boundary entries zeroed (to_boundary_zero) or kept.
cudaError_t launch_cast_d2f(size_t n, const double* in, float* out, cudaStream_t s);
cudaError_t launch_cast_f2d(size_t n, const float* in, double* out, cudaStream_t s);
// Coarse solve: x[free[i]] = sum_j Ainv[i][j] b[free[j]], FP64 arithmetic; x elsewhere untouched.
template <typename T>
cudaError_t launch_coarse_solve(int nf, const int* free_idx, const double* Ainv, const T* b, T* x, cudaStream_t s);

// FP64 vector ops.
cudaError_t launch_axpby(size_t n, double a, const double* x, double b, double* y, cudaStream_t s);   // y = a x + b y
cudaError_t launch_mul(size_t n, const double* a, const double* x, double* y, cudaStream_t s);         // y = a .* x
cudaError_t launch_axpby_f(size_t n, float a, const float* x, float b, float* y, cudaStream_t s);      // FP32
cudaError_t launch_sqrt_vec(size_t n, const double* a, double* y, cudaStream_t s);                     // y = sqrt(a)
cudaError_t launch_fill(size_t n, double v, double* y, cudaStream_t s);
cudaError_t launch_recip(size_t n, const double* a, double* y, cudaStream_t s);                       // y = 1 / a
cudaError_t launch_add_scalar(size_t n, double v, double* y, cudaStream_t s);                          // y += v
cudaError_t launch_splitmix_vector(size_t n, uint64_t seed, const double* mask, double* y, cudaStream_t s);
// Multi-dot: out[i] = sum_e V[i*ld + e] * w[e], i < k, and out[k] = w . w when self; deterministic
// two-pass reduction through `partials` (multidot_blocks() * (k + 1) doubles).
cudaError_t launch_multidot(size_t n, int k, const double* V, size_t ld, const double* w, double* partials,
                            double* out, cudaStream_t s, bool self = false);
int multidot_blocks();
// w -= sum_i h[i] V[i*ld + :], i < k (h on device); with sign = +1 adds instead.
cudaError_t launch_multiaxpy(size_t n, int k, const double* V, size_t ld, const double* h, double* w, double sign,
                             cudaStream_t s);
// Fused vector passes of IDR(s) and MINRES (FP64). out non-null: out[0] (out[0..1] for dot2) on the
// device from the partials, as launch_multidot.
// y1 += a1 x1, y2 += a2 x2 (x2 null: no second update); out: y1 . y1 of the updated y1
cudaError_t launch_axpy2(size_t n, double a1, const double* x1, double* y1, double a2, const double* x2, double* y2,
                         double* partials, double* out, cudaStream_t s);
// out[0] = x . y1, out[1] = x . y2
cudaError_t launch_dot2(size_t n, const double* x, const double* y1, const double* y2, double* partials, double* out,
                        cudaStream_t s);
// w = a src + sign sum_{i<k} h_i V_i (h on the device; w may alias src or a row of V)
cudaError_t launch_lincomb(size_t n, int k, const double* V, size_t ld, const double* h, double a, const double* src,
                           double* w, double sign, cudaStream_t s);
// vo = q + bv vo + cv v, kwo = q + bk kwo + ck kw, wo = z + bw wo + cw w
cudaError_t launch_minres_dirs(size_t n, const double* q, const double* z, double* vo, const double* v, double bv,
                               double cv, double* kwo, const double* kw, double bk, double ck, double* wo,
                               const double* w, double bw, double cw, cudaStream_t s);
// w *= f, kw *= f, x += e w, r -= e kw; out[0] = r . r
cudaError_t launch_minres_update(size_t n, double f, double* w, double* kw, double e, double* x, double* r,
                                 double* partials, double* out, cudaStream_t s);

// Fused Gram-Schmidt passes (krylov.cu), all results on the device; `partials` holds
// gs_partials_blocks() * (k + 1) doubles at least. df = double-float arithmetic with V stored
// as double-float pairs (k <= 64); otherwise native FP64 kernels with V in FP64.
//   launch_gs_dot:           out[i] = V_i . w, i < k
//   launch_gs_project_dot:   w -= V h; out[i] = V_i . w (i < k), out[k] = w . w,
//                            out[k+1] = hn = sqrt(max(out[k] - sum_i out[i]^2, 0)), out[k+2] = 1 / hn
//   launch_gs_project_scale: y = (w - V h) * scale[0]
cudaError_t gs_configure();
int gs_partials_blocks();
int gs_max_k();   // restart lengths above this use the native FP64 passes
cudaError_t launch_gs_dot(size_t n, int k, const double* V, size_t ld, const double* w, double* partials,
                          double* out, bool df, cudaStream_t s);
cudaError_t launch_gs_project_dot(size_t n, int k, const double* V, size_t ld, const double* h, double* w,
                                  double* partials, double* out, bool df, cudaStream_t s);
cudaError_t launch_gs_project_scale(size_t n, int k, const double* V, size_t ld, const double* h, const double* w,
                                    const double* scale, double* y, bool df, cudaStream_t s);
// y = w * scale stored as double-float pairs; x = double-float pairs v as FP64.
cudaError_t launch_df_store_scaled(size_t n, const double* w, double scale, double* y, cudaStream_t s);
cudaError_t launch_df_to_double(size_t n, const double* v, double* x, cudaStream_t s, double scale = 1.0);
// FGMRES with delayed re-orthogonalisation (two passes over the basis per step instead of three):
//   launch_gs_dot_lag:     out[i] = V_i . w, i < k; with lag (the record below of the previous step,
//                          j = k - 1, row j holding u_j): out[j] = v_j . w for the corrected v_j
//   launch_gs_lag_project: v_j = (u_j - V_{<j} c) / alpha over row j (lag null: row j is final);
//                          w1 = w - V_{<=j} h into row j + 1 (double-float); record of this step:
//                          out[0..j] = V_{<=j}^T w1 (= c of the next), out[j+1] = |w1|^2,
//                          out[j+2] = alpha = sqrt(|w1|^2 - |c|^2), out[j+3] = 1 / alpha
cudaError_t launch_gs_dot_lag(size_t n, int k, const double* V, size_t ld, const double* w, double* partials,
                              double* out, const double* lag, cudaStream_t s);
cudaError_t launch_gs_lag_project(size_t n, int k, double* V, size_t ld, const double* h, const double* lag,
                                  const double* w, double* partials, double* out, cudaStream_t s);

}  // namespace stk
