// ops.cu -- matrix-free Q2-Q1 operators and the set-up kernels.
//
// The FP64 outer operator [A, B^T; B, 0] (Section 2.1): one thread per cube
//   cell, sum-factorised A (q2::cell_A) and the 1D-moment tensor products of
//   B and B^T; contributions are accumulated into the zeroed outputs with
//   atomic adds and constrained (boundary-node) rows then get src. (The level
//   operators of the V-cycle use the brick-tiled kernel of brick.cuh.)
// M_p (Section 2.2.2): Q1 mass matrix weighted by 1/mu per cell.
// Set-up: viscosity at the Gauss points and its harmonic cell average
//   (Section 2.3), Q0 restriction (parent = mean of children, Section 2.3),
//   the sinker right-hand side (Section 3.2), diagonals.
#include "internal.cuh"
#include "q2_basis.cuh"
#include "df64.cuh"
#include "prof.cuh"
#include "pressure.cuh"

#define LAUNCH(cls, s, ...)              \
    do {                                \
        prof_begin((cls), (s));         \
        __VA_ARGS__;                    \
        prof_end((cls), (s));           \
        prof_count(1);                  \
    } while (0)

namespace stk {

namespace {

constexpr int kCellThreads = 128;

__device__ __forceinline__ bool on_bnd(int gi, int M) { return gi == 0 || gi == M - 1; }

template <typename T>
__device__ __forceinline__ void gather_u(const T* __restrict__ src, size_t nodes, int M, int ci, int cj, int ck,
                                         T (&u)[3][27]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                const bool b = on_bnd(gi, M) || on_bnd(gj, M) || on_bnd(gk, M);
                const size_t node = size_t(gi) + size_t(M) * (gj + size_t(M) * gk);
#pragma unroll
                for (int c = 0; c < 3; ++c) u[c][i + 3 * j + 9 * k] = b ? T(0) : src[c * nodes + node];
            }
}

__device__ __forceinline__ double to_io(double v) { return v; }
__device__ __forceinline__ double to_io(const q2::df64& v) { return double(v.hi) + double(v.lo); }
template <typename CT> __device__ __forceinline__ CT from_io(double v);
template <> __device__ __forceinline__ double from_io<double>(double v) { return v; }
template <> __device__ __forceinline__ q2::df64 from_io<q2::df64>(double v) { return q2::from_double(v); }

// dst += w (converted to FP64) on the free nodes of one cell.
template <typename CT>
__device__ __forceinline__ void scatter_io(double* __restrict__ dst, size_t nodes, int M, int ci, int cj, int ck,
                                           const CT (&w)[3][27]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                if (on_bnd(gi, M) || on_bnd(gj, M) || on_bnd(gk, M)) continue;
                const size_t node = size_t(gi) + size_t(M) * (gj + size_t(M) * gk);
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(dst + c * nodes + node, to_io(w[c][i + 3 * j + 9 * k]));
            }
}

// u = src on the free nodes of one cell, 0 on constrained ones, converted to the compute type.
template <typename CT>
__device__ __forceinline__ void gather_io(const double* __restrict__ src, size_t nodes, int M, int ci, int cj, int ck,
                                          CT (&u)[3][27]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                const bool b = on_bnd(gi, M) || on_bnd(gj, M) || on_bnd(gk, M);
                const size_t node = size_t(gi) + size_t(M) * (gj + size_t(M) * gk);
#pragma unroll
                for (int c = 0; c < 3; ++c) u[c][i + 3 * j + 9 * k] = b ? CT(0) : from_io<CT>(src[c * nodes + node]);
            }
}

template <typename T>
__device__ __forceinline__ void scatter_u(T* __restrict__ dst, size_t nodes, int M, int ci, int cj, int ck,
                                          const T (&w)[3][27], T scale) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                const bool b = on_bnd(gi, M) || on_bnd(gj, M) || on_bnd(gk, M);
                if (b) continue;
                const size_t node = size_t(gi) + size_t(M) * (gj + size_t(M) * gk);
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(dst + c * nodes + node, scale * w[c][i + 3 * j + 9 * k]);
            }
}

// Boundary nodes of an M^3 lattice: 6 faces of M*M nodes (edges repeated; writes are identical).
template <typename T>
__global__ void k_copy_boundary(int M, const T* __restrict__ in, T* __restrict__ out) {
    const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t face = size_t(M) * M;
    if (t >= 6 * face) return;
    const int f = int(t / face);
    const int a = int((t % face) % M), b = int((t % face) / M);
    const int fixed = (f & 1) ? M - 1 : 0;
    int i, j, k;
    if (f < 2) { i = fixed; j = a; k = b; } else if (f < 4) { i = a; j = fixed; k = b; } else { i = a; j = b; k = fixed; }
    const size_t nodes = size_t(M) * M * M;
    const size_t node = size_t(i) + size_t(M) * (j + size_t(M) * k);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * nodes + node] = in ? in[c * nodes + node] : T(0);
}

// ---------------------------------------------------------------- Stokes blocks (FP64 in/out)
// Native FP64, one thread per cell (CT = double). The double-float variant is the
// component-split kernel of outer.cuh.
template <typename CT, bool DO_A, bool DO_BT, bool DO_B>
__global__ void __launch_bounds__(kCellThreads) k_stokes_blocks(int n, double h, const double* __restrict__ mu,
                                                                const double* __restrict__ src_u,
                                                                const double* __restrict__ src_p,
                                                                double* __restrict__ dst_u,
                                                                double* __restrict__ dst_p) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t cells = size_t(n) * n * n;
    if (cell >= cells) return;
    const int ci = int(cell % n), cj = int((cell / n) % n), ck = int(cell / (size_t(n) * n));
    const int M = 2 * n + 1;
    const size_t nodes = size_t(M) * M * M;
    const int P = n + 1;
    CT u[3][27], w[3][27];
    if (DO_A || DO_B) gather_io<CT>(src_u, nodes, M, ci, cj, ck, u);
    if (DO_B) {
        // (B u)_v = -int div(u_h) psi_v = -h^2 sum_c (moments along each axis) . u_c
        CT bp[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) bp[v] = CT(0);
        q2::b_component<0>(u[0], bp);
        q2::b_component<1>(u[1], bp);
        q2::b_component<2>(u[2], bp);
        const double s = -h * h;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const size_t vert = size_t(ci + (v & 1)) + size_t(P) * (cj + ((v >> 1) & 1) + size_t(P) * (ck + (v >> 2)));
            atomicAdd(dst_p + vert, s * to_io(bp[v]));
        }
    }
    if (DO_A || DO_BT) {
        if (DO_A) {
            q2::cell_A(u, w);
            const CT sA = from_io<CT>(mu[cell] * h);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int a = 0; a < 27; ++a) w[c][a] *= sA;
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int a = 0; a < 27; ++a) w[c][a] = CT(0);
        }
        if (DO_BT) {
            // (B^T p)_(c,m) = -int d_c(phi_m) p_h = -h^2 sum_v (moments along each axis) p_v
            CT p8[8];
            const double s = -h * h;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const size_t vert =
                    size_t(ci + (v & 1)) + size_t(P) * (cj + ((v >> 1) & 1) + size_t(P) * (ck + (v >> 2)));
                p8[v] = from_io<CT>(s * src_p[vert]);
            }
            q2::bt_component<0>(p8, w[0]);
            q2::bt_component<1>(p8, w[1]);
            q2::bt_component<2>(p8, w[2]);
        }
        scatter_io<CT>(dst_u, nodes, M, ci, cj, ck, w);
    }
}

// ---------------------------------------------------------------- pressure mass
__global__ void k_mass_p(int n, double h, const double* __restrict__ mu, const double* __restrict__ src,
                         double* __restrict__ dst) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const size_t cells = size_t(n) * n * n;
    if (cell >= cells) return;
    const int ci = int(cell % n), cj = int((cell / n) % n), ck = int(cell / (size_t(n) * n));
    const int P = n + 1;
    size_t vert[8];
    double p[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        vert[v] = size_t(ci + (v & 1)) + size_t(P) * (cj + ((v >> 1) & 1) + size_t(P) * (ck + (v >> 2)));
        p[v] = src[vert[v]];
    }
    const double s = h * h * h / mu[cell];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc += q2::M1(a & 1, b & 1) * q2::M1((a >> 1) & 1, (b >> 1) & 1) * q2::M1(a >> 2, b >> 2) * p[b];
        atomicAdd(dst + vert[a], s * acc);
    }
}

// ---- B^T on the uniform mesh as a gather (pressure.cuh). Block (line (J, K), component c):
// threads 0..8 put the line's weights, thread e then t_e into shared memory; thread e writes the
// x-nodes 2e and 2e + 1. No atomics.
template <int C>
__device__ __forceinline__ void bt_line(int n, double s, const double* __restrict__ p, double* __restrict__ out,
                                        int J, int K, q2::df64* t, q2::df64* w) {
    const int P = n + 1, M = 2 * n + 1;
    const int e = int(threadIdx.x);
    double* o = out + size_t(C) * size_t(M) * M * M + size_t(M) * (J + size_t(M) * K);
    if (J == 0 || J == M - 1 || K == 0 || K == M - 1) {   // boundary rows
        for (int i = e; i < M; i += int(blockDim.x)) o[i] = 0.0;
        return;
    }
    if (e < 9) w[e] = bt_weight<C>(J, K, e);
    __syncthreads();
    if (e < P) t[e] = bt_t<C>(n, p, J, K, e, w);
    __syncthreads();
    if (e < P) bt_out<C>(n, s, o, e, t);
}

__global__ void k_bt_gather(int n, double h, const double* __restrict__ p, double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char bt_smem[];
    q2::df64* t = reinterpret_cast<q2::df64*>(bt_smem);   // n + 1 entries
    q2::df64* w = t + (n + 1);                             // 9 entries
    const int M = 2 * n + 1;
    const int J = int(blockIdx.x % unsigned(M)), K = int(blockIdx.x / unsigned(M)), c = int(blockIdx.y);
    const double s = -h * h;
    if (c == 0) bt_line<0>(n, s, p, out, J, K, t, w);
    else if (c == 1) bt_line<1>(n, s, p, out, J, K, t, w);
    else bt_line<2>(n, s, p, out, J, K, t, w);
}

// s_K = h^3 / mu_K per cell: the factor of the cell's pressure mass matrix (Section 2.2.2, the
// 1/mu-weighted mass matrix), as k_mass_p forms it.
__global__ void k_mass_scale(size_t cells, double h, const double* __restrict__ mu, double* __restrict__ scale) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell < cells) scale[cell] = h * h * h / mu[cell];
}

// One Jacobi-Chebyshev step of S_hat^-1 with the M_p product gathered per pressure vertex
// (pressure.cuh schur_vertex): one thread per vertex, no atomics.
__global__ void __launch_bounds__(128) k_schur_cheb(int n, const double* __restrict__ scale, const double* __restrict__ r,
                                                    const double* __restrict__ dinv, const double* __restrict__ z,
                                                    const double* __restrict__ d, double* __restrict__ z_new,
                                                    double* __restrict__ d_new, double c1, double c2) {
    const int P = n + 1;
    const size_t vtx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (vtx >= size_t(P) * P * P) return;
    schur_vertex(n, scale, r, dinv, z, d, z_new, d_new, c1, c2, vtx);
}

__global__ void k_mass_p_diag(int n, double h, const double* __restrict__ mu, double* __restrict__ diag,
                              double* __restrict__ weights) {
    const size_t vtx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int P = n + 1;
    if (vtx >= size_t(P) * P * P) return;
    const int vi = int(vtx % P), vj = int((vtx / P) % P), vk = int(vtx / (size_t(P) * P));
    const double h3 = h * h * h;
    // int psi over one cell for a vertex: product of 1D sum_q w_q psi(q) = 1/2 each
    const double int1 = q2::gw(0) * q2::Pq(0, 0) + q2::gw(1) * q2::Pq(1, 0) + q2::gw(2) * q2::Pq(2, 0);
    const double mii = q2::M1(0, 0) * q2::M1(0, 0) * q2::M1(0, 0);
    double d = 0.0, wsum = 0.0;
    for (int dk = -1; dk <= 0; ++dk)
        for (int dj = -1; dj <= 0; ++dj)
            for (int di = -1; di <= 0; ++di) {
                const int ci = vi + di, cj = vj + dj, ck = vk + dk;
                if (ci < 0 || cj < 0 || ck < 0 || ci >= n || cj >= n || ck >= n) continue;
                const size_t cell = size_t(ci) + size_t(n) * (cj + size_t(n) * ck);
                d += h3 * mii / mu[cell];
                wsum += h3 * int1 * int1 * int1;
            }
    diag[vtx] = d;
    if (weights) weights[vtx] = wsum;
}

// ---------------------------------------------------------------- diagonal of A
__global__ void k_ref_diag(double* out81) {
    const int t = threadIdx.x;
    if (t >= 81) return;
    double u[3][27], w[3][27];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 27; ++a) u[c][a] = (c * 27 + a == t) ? 1.0 : 0.0;
    q2::cell_A(u, w);
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 27; ++a)
            if (c * 27 + a == t) v = w[c][a];
    out81[t] = v;
}

__global__ void k_inv_diag(int n, double h, const double* __restrict__ mu, const double* __restrict__ ref,
                           double* __restrict__ dinv) {
    const size_t node = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int M = 2 * n + 1;
    const size_t nodes = size_t(M) * M * M;
    if (node >= nodes) return;
    const int gi = int(node % M), gj = int((node / M) % M), gk = int(node / (size_t(M) * M));
    if (on_bnd(gi, M) || on_bnd(gj, M) || on_bnd(gk, M)) {
        for (int c = 0; c < 3; ++c) dinv[c * nodes + node] = 0.0;
        return;
    }
    // cells containing the node along one axis: odd index -> one cell (local 1); even -> two (local 2, 0)
    int cx[2], lx[2], nx = 0, cy[2], ly[2], ny = 0, cz[2], lz[2], nz = 0;
    auto axis = [n](int g, int* cc, int* ll, int& cnt) {
        if (g & 1) { cc[0] = (g - 1) / 2; ll[0] = 1; cnt = 1; return; }
        cnt = 0;
        if (g / 2 - 1 >= 0) { cc[cnt] = g / 2 - 1; ll[cnt] = 2; ++cnt; }
        if (g / 2 < n) { cc[cnt] = g / 2; ll[cnt] = 0; ++cnt; }
    };
    axis(gi, cx, lx, nx); axis(gj, cy, ly, ny); axis(gk, cz, lz, nz);
    double d[3] = {0.0, 0.0, 0.0};
    for (int c3 = 0; c3 < nz; ++c3)
        for (int c2 = 0; c2 < ny; ++c2)
            for (int c1 = 0; c1 < nx; ++c1) {
                const size_t cell = size_t(cx[c1]) + size_t(n) * (cy[c2] + size_t(n) * cz[c3]);
                const int a = lx[c1] + 3 * ly[c2] + 9 * lz[c3];
                const double s = mu[cell] * h;
                for (int c = 0; c < 3; ++c) d[c] += s * ref[c * 27 + a];
            }
    for (int c = 0; c < 3; ++c) dinv[c * nodes + node] = 1.0 / d[c];
}

// ---------------------------------------------------------------- sinker coefficients
__device__ __forceinline__ double sinker_X(double x, double y, double z, const double* __restrict__ centres, int ns,
                                           double delta, double omega) {
    double X = 1.0;
    for (int s = 0; s < ns; ++s) {
        const double dx = x - centres[3 * s], dy = y - centres[3 * s + 1], dz = z - centres[3 * s + 2];
        const double dist = sqrt(dx * dx + dy * dy + dz * dz);
        const double e = fmax(0.0, dist - 0.5 * omega);
        X *= 1.0 - exp(-delta * e * e);
    }
    return X;
}

__global__ void k_mu_sinker(int n, double h, const double* __restrict__ centres, int ns, double mu_min,
                            double mu_max, double delta, double omega, double* __restrict__ mu) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= size_t(n) * n * n) return;
    const int ci = int(cell % n), cj = int((cell / n) % n), ck = int(cell / (size_t(n) * n));
    double inv = 0.0, wsum = 0.0;
    for (int qz = 0; qz < 3; ++qz)
        for (int qy = 0; qy < 3; ++qy)
            for (int qx = 0; qx < 3; ++qx) {
                const double x = (ci + q2::gp(qx)) * h, y = (cj + q2::gp(qy)) * h, z = (ck + q2::gp(qz)) * h;
                const double X = sinker_X(x, y, z, centres, ns, delta, omega);
                const double m = X * mu_min + (1.0 - X) * mu_max;
                const double wq = q2::gw(qx) * q2::gw(qy) * q2::gw(qz);
                inv += wq / m;
                wsum += wq;
            }
    mu[cell] = wsum / inv;
}

__global__ void k_mu_from_q(size_t cells, const double* __restrict__ mu_q, double* __restrict__ mu) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= cells) return;
    double inv = 0.0, wsum = 0.0;
    for (int q = 0; q < 27; ++q) {
        const double wq = q2::gw(q % 3) * q2::gw((q / 3) % 3) * q2::gw(q / 9);
        inv += wq / mu_q[cell * 27 + q];
        wsum += wq;
    }
    mu[cell] = wsum / inv;
}

__global__ void k_mu_restrict(int nc, const double* __restrict__ fine, double* __restrict__ coarse) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= size_t(nc) * nc * nc) return;
    const int ci = int(cell % nc), cj = int((cell / nc) % nc), ck = int(cell / (size_t(nc) * nc));
    const int nf = 2 * nc;
    double s = 0.0;
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) s += fine[size_t(2 * ci + i) + size_t(nf) * (2 * cj + j + size_t(nf) * (2 * ck + k))];
    coarse[cell] = s / 8.0;
}

__global__ void k_rhs_sinker(int n, double h, const double* __restrict__ centres, int ns, double delta,
                             double omega, double beta, double* __restrict__ F) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= size_t(n) * n * n) return;
    const int ci = int(cell % n), cj = int((cell / n) % n), ck = int(cell / (size_t(n) * n));
    const int M = 2 * n + 1;
    const size_t nodes = size_t(M) * M * M;
    double f[27];
    for (int qz = 0; qz < 3; ++qz)
        for (int qy = 0; qy < 3; ++qy)
            for (int qx = 0; qx < 3; ++qx) {
                const double x = (ci + q2::gp(qx)) * h, y = (cj + q2::gp(qy)) * h, z = (ck + q2::gp(qz)) * h;
                const double X = sinker_X(x, y, z, centres, ns, delta, omega);
                f[qx + 3 * qy + 9 * qz] = q2::gw(qx) * q2::gw(qy) * q2::gw(qz) * beta * (X - 1.0);
            }
    q2::interpT<0>(f); q2::interpT<1>(f); q2::interpT<2>(f);
    const double h3 = h * h * h;
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) {
                const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                if (on_bnd(gi, M) || on_bnd(gj, M) || on_bnd(gk, M)) continue;
                const size_t node = size_t(gi) + size_t(M) * (gj + size_t(M) * gk);
                atomicAdd(F + 2 * nodes + node, h3 * f[i + 3 * j + 9 * k]);
            }
}

inline unsigned blocks_for(size_t n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace

template <typename T>
cudaError_t launch_copy_boundary(const LevelGeom& g, const T* in, T* out, cudaStream_t s) {
    const size_t nb = 6 * size_t(g.M) * g.M;
    LAUNCH(PROF_SMOOTH_VEC, s, k_copy_boundary<T><<<blocks_for(nb, 256), 256, 0, s>>>(g.M, in, out));
    return cudaGetLastError();
}
template cudaError_t launch_copy_boundary<float>(const LevelGeom&, const float*, float*, cudaStream_t);
template cudaError_t launch_copy_boundary<double>(const LevelGeom&, const double*, double*, cudaStream_t);

template <typename T>
cudaError_t launch_zero_boundary(const LevelGeom& g, T* x, cudaStream_t s) {
    return launch_copy_boundary<T>(g, nullptr, x, s);
}
template cudaError_t launch_zero_boundary<float>(const LevelGeom&, float*, cudaStream_t);
template cudaError_t launch_zero_boundary<double>(const LevelGeom&, double*, cudaStream_t);

template <typename CT>
cudaError_t stokes_blocks_ct(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                             double* dst_u, double* dst_p, bool do_a, bool do_bt, bool do_b, cudaStream_t s) {
    const unsigned nb = blocks_for(g.cells, kCellThreads);
    const double h = g.h;
    if (do_a && do_bt && do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_stokes_blocks<CT, true, true, true><<<nb, kCellThreads, 0, s>>>(g.n, h, mu, src_u, src_p, dst_u, dst_p)));
    else if (do_a && !do_bt && !do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_stokes_blocks<CT, true, false, false><<<nb, kCellThreads, 0, s>>>(g.n, h, mu, src_u, src_p, dst_u, dst_p)));
    else if (!do_a && do_bt && !do_b)
        LAUNCH(PROF_BT_F64, s, (k_stokes_blocks<CT, false, true, false><<<nb, kCellThreads, 0, s>>>(g.n, h, mu, src_u, src_p, dst_u, dst_p)));
    else if (!do_a && !do_bt && do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_stokes_blocks<CT, false, false, true><<<nb, kCellThreads, 0, s>>>(g.n, h, mu, src_u, src_p, dst_u, dst_p)));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_stokes_blocks(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                                 double* dst_u, double* dst_p, bool do_a, bool do_bt, bool do_b, bool df64,
                                 cudaStream_t s) {
    cudaError_t e;
    // B^T alone (the preconditioner's): the gather writes every velocity entry, no clear needed;
    // its blocks hold one thread per vertex of a line (n + 1 <= 1024)
    if (df64 && !do_a && do_bt && !do_b && g.n + 1 <= 1024) return launch_bt_gather(g, src_p, dst_u, s);
    if (do_a || do_bt) {
        e = cudaMemsetAsync(dst_u, 0, g.n_u * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    if (do_b) {
        e = cudaMemsetAsync(dst_p, 0, g.n_p * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    // double-float on the FP32 pipes for every block (GB300's FP64 pipe retires 1/72 of the FP32
    // rate): B^T alone, the preconditioner's, takes 148 us at 64^3 against 221 us in native FP64
    e = df64 ? launch_outer_df64(g, mu, src_u, src_p, dst_u, dst_p, do_a, do_bt, do_b, s)
                       : stokes_blocks_ct<double>(g, mu, src_u, src_p, dst_u, dst_p, do_a, do_bt, do_b, s);
    if (e != cudaSuccess) return e;
    if (do_a) {
        const size_t nbd = 6 * size_t(g.M) * g.M;
        LAUNCH(PROF_SMOOTH_VEC, s, (k_copy_boundary<double><<<blocks_for(nbd, 256), 256, 0, s>>>(g.M, src_u, dst_u)));
    }
    return cudaGetLastError();
}

cudaError_t launch_mass_p(const LevelGeom& g, const double* mu, const double* src, double* dst, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(dst, 0, g.n_p * sizeof(double), s);
    if (e != cudaSuccess) return e;
    LAUNCH(PROF_MASS_P, s, k_mass_p<<<blocks_for(g.cells, 128), 128, 0, s>>>(g.n, g.h, mu, src, dst));
    return cudaGetLastError();
}

cudaError_t launch_bt_gather(const LevelGeom& g, const double* p, double* out, cudaStream_t s) {
    // one block per (line, component), one thread per vertex of the line (x-nodes 2e, 2e + 1)
    const unsigned threads = unsigned((g.n + 1 + 31) / 32 * 32);
    const size_t smem = size_t(g.n + 1 + 9) * sizeof(q2::df64);
    const dim3 grid(unsigned(size_t(g.M) * g.M), 3);
    LAUNCH(PROF_BT_F64, s, k_bt_gather<<<grid, threads, smem, s>>>(g.n, g.h, p, out));
    return cudaGetLastError();
}

cudaError_t launch_mass_scale(const LevelGeom& g, const double* mu, double* scale, cudaStream_t s) {
    LAUNCH(PROF_MASS_P, s, k_mass_scale<<<blocks_for(g.cells, 256), 256, 0, s>>>(g.cells, g.h, mu, scale));
    return cudaGetLastError();
}

cudaError_t launch_schur_cheb(const LevelGeom& g, const double* scale, const double* r, const double* dinv,
                              const double* z, const double* d, double* z_new, double* d_new, double c1, double c2,
                              cudaStream_t s) {
    LAUNCH(PROF_MASS_P, s, k_schur_cheb<<<blocks_for(g.n_p, 128), 128, 0, s>>>(g.n, scale, r, dinv, z, d, z_new, d_new,
                                                                             c1, c2));
    return cudaGetLastError();
}

cudaError_t launch_mass_p_diag(const LevelGeom& g, const double* mu, double* diag, double* weights,
                               cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_mass_p_diag<<<blocks_for(g.n_p, 256), 256, 0, s>>>(g.n, g.h, mu, diag, weights));
    return cudaGetLastError();
}

cudaError_t launch_ref_diag(double* ref_diag81, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_ref_diag<<<1, 96, 0, s>>>(ref_diag81));
    return cudaGetLastError();
}

cudaError_t launch_inv_diag(const LevelGeom& g, const double* mu, const double* ref_diag81, double* dinv,
                            cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_inv_diag<<<blocks_for(g.nodes, 256), 256, 0, s>>>(g.n, g.h, mu, ref_diag81, dinv));
    return cudaGetLastError();
}

cudaError_t launch_mu_sinker(const LevelGeom& g, const double* centres, int n_sinkers, double mu_min,
                             double mu_max, double delta, double omega, double* mu, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_mu_sinker<<<blocks_for(g.cells, 128), 128, 0, s>>>(g.n, g.h, centres, n_sinkers, mu_min, mu_max, delta,
                                                          omega, mu));
    return cudaGetLastError();
}

cudaError_t launch_mu_from_q(const LevelGeom& g, const double* mu_q, double* mu, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_mu_from_q<<<blocks_for(g.cells, 128), 128, 0, s>>>(g.cells, mu_q, mu));
    return cudaGetLastError();
}

cudaError_t launch_mu_restrict(const LevelGeom& coarse, const double* mu_fine, double* mu_coarse, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_mu_restrict<<<blocks_for(coarse.cells, 128), 128, 0, s>>>(coarse.n, mu_fine, mu_coarse));
    return cudaGetLastError();
}

cudaError_t launch_rhs_sinker(const LevelGeom& g, const double* centres, int n_sinkers, double delta,
                              double omega, double beta, double* F, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(F, 0, g.n_u * sizeof(double), s);
    if (e != cudaSuccess) return e;
    LAUNCH(PROF_SMOOTH_VEC, s, k_rhs_sinker<<<blocks_for(g.cells, 128), 128, 0, s>>>(g.n, g.h, centres, n_sinkers, delta, omega, beta, F));
    return cudaGetLastError();
}

}  // namespace stk
