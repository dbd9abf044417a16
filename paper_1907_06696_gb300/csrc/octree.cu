// octree.cu -- device kernels of the adaptive (octree) path: level operators on the cells of
// one level through an index map (local smoothing, Section 2.2.1 by citation), Q2 transfers
// between levels, copies between the active space and the levels, and the active Stokes
// blocks with hanging-node constraints resolved in the gather and the scatter (Section 2.1,
// with the constrained space of the adaptive meshes).
//
// Every kernel takes one cell (or one node) per thread. Level vectors are component-blocked
// [3][nn]; the active velocity vector is [3][nu] and the active pressure vector [np].
#include "octree.cuh"
#include "prof.cuh"
#include "q2_basis.cuh"

#define LAUNCH(cls, s, ...)              \
    do {                                \
        prof_begin((cls), (s));         \
        __VA_ARGS__;                    \
        prof_end((cls), (s));           \
        prof_count(1);                  \
    } while (0)

namespace stk {

namespace {

inline unsigned blocks_for(size_t n, int t) {
    const size_t b = (n + t - 1) / t;
    return unsigned(b == 0 ? 1 : b);
}

// Quadratic Lagrange basis on {0, 1/2, 1} at positions 0, 1/4, 1/2, 3/4, 1 of a parent cell.
__constant__ double c_q2_at[5][3] = {{1, 0, 0}, {0.375, 0.75, -0.125}, {0, 1, 0}, {-0.125, 0.75, 0.375}, {0, 0, 1}};
__device__ __forceinline__ double q2_at(int p, int m) { return c_q2_at[p][m]; }

// Is entry v, read at position `at` of table t, below `bound`? STOKES_DEBUG builds check and record
// the first failure (flag, table + 1, position); release builds return true without a test.
__device__ __forceinline__ bool idx_ok(const OctDebug& d, int t, long long v, long long bound, size_t at) {
#ifdef STOKES_DEBUG
    if (v >= 0 && v < bound - d.cut[t]) return true;
    if (d.status) {
        atomicOr(d.status, kStatusBadIndex);
        if (atomicCAS(d.status + 1, 0u, unsigned(t + 1)) == 0u) {
            d.status[2] = unsigned(uint64_t(at) & 0xffffffffu);
            d.status[3] = unsigned(uint64_t(at) >> 32);
        }
    }
    return false;
#else
    (void)d; (void)t; (void)v; (void)bound; (void)at;
    return true;
#endif
}

template <typename T>
__global__ void __launch_bounds__(128) k_oct_cells(OctLevelDev L, const T* __restrict__ mu, const T* __restrict__ src,
                                                   T* __restrict__ acc) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.n_cells) return;
    const int32_t* cn = L.cell_nodes + size_t(cell) * 27;
    T u[3][27], w[3][27];
    unsigned skip = 0;   // bit a: node a is a boundary node (or a bad table entry)
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        const int32_t node = cn[a];
        const bool b = !idx_ok(L.dbg, OCT_CELL_NODES, node, (long long)L.nn, size_t(cell) * 27 + a) ||
                       (L.flags[node] & 1) != 0;
        skip |= unsigned(b) << a;
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c][a] = b ? T(0) : src[c * L.nn + node];
    }
    q2::cell_A(u, w);
    const T s = mu[cell] * T(L.h);
#pragma unroll
    for (int a = 0; a < 27; ++a) {
        if ((skip >> a) & 1u) continue;
        const int32_t node = cn[a];
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(acc + c * L.nn + node, w[c][a] * s);
    }
}

template <typename T>
__global__ void k_oct_copy_boundary(OctLevelDev L, const T* __restrict__ src, T* __restrict__ dst) {
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= L.nn || !(L.flags[n] & 1)) return;
    for (int c = 0; c < 3; ++c) dst[c * L.nn + n] = src[c * L.nn + n];
}

__global__ void k_oct_diag(OctLevelDev L, const double* __restrict__ mu, const double* __restrict__ ref,
                           double* __restrict__ diag) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.n_cells) return;
    const double s = mu[cell] * L.h;
    for (int a = 0; a < 27; ++a) {
        const int32_t node = L.cell_nodes[size_t(cell) * 27 + a];
        if (!idx_ok(L.dbg, OCT_CELL_NODES, node, (long long)L.nn, size_t(cell) * 27 + a)) continue;
        for (int c = 0; c < 3; ++c) atomicAdd(diag + c * L.nn + node, s * ref[c * 27 + a]);
    }
}

__global__ void k_oct_dinv(OctLevelDev L, const double* __restrict__ diag, double* __restrict__ dinv) {
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= L.nn) return;
    const bool skip = L.flags[n] != 0;
    for (int c = 0; c < 3; ++c) dinv[c * L.nn + n] = skip ? 0.0 : 1.0 / diag[c * L.nn + n];
}

template <typename T>
__global__ void k_oct_prolongate(OctLevelDev F, OctLevelDev C, const T* __restrict__ coarse, T* __restrict__ fine,
                                 bool add) {
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= F.nn) return;
    if (F.flags[n] & 1) {
        if (!add)
            for (int c = 0; c < 3; ++c) fine[c * F.nn + n] = T(0);
        return;
    }
    const uint32_t par = F.parent[n];
    const int p = F.pos[n], px = p % 5, py = (p / 5) % 5, pz = p / 25;
    T v[3] = {T(0), T(0), T(0)};
    if (idx_ok(F.dbg, OCT_PARENT, par, C.n_cells, n) && idx_ok(F.dbg, OCT_POS, p, 125, n)) {
        const int32_t* cn = C.cell_nodes + size_t(par) * 27;
        for (int b = 0; b < 27; ++b) {
            const double w = q2_at(px, b % 3) * q2_at(py, (b / 3) % 3) * q2_at(pz, b / 9);
            if (w == 0.0) continue;
            const int32_t node = cn[b];
            if (!idx_ok(C.dbg, OCT_CELL_NODES, node, (long long)C.nn, size_t(par) * 27 + b)) continue;
            for (int c = 0; c < 3; ++c) v[c] += T(w) * coarse[c * C.nn + node];
        }
    }
    for (int c = 0; c < 3; ++c) fine[c * F.nn + n] = (add ? fine[c * F.nn + n] : T(0)) + v[c];
}

template <typename T>
__global__ void k_oct_restrict_add(OctLevelDev F, OctLevelDev C, const T* __restrict__ fine, T* __restrict__ coarse) {
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= F.nn || (F.flags[n] & 1)) return;
    const uint32_t par = F.parent[n];
    const int p = F.pos[n], px = p % 5, py = (p / 5) % 5, pz = p / 25;
    if (!idx_ok(F.dbg, OCT_PARENT, par, C.n_cells, n) || !idx_ok(F.dbg, OCT_POS, p, 125, n)) return;
    const int32_t* cn = C.cell_nodes + size_t(par) * 27;
    const T f[3] = {fine[n], fine[F.nn + n], fine[2 * F.nn + n]};
    for (int b = 0; b < 27; ++b) {
        const double w = q2_at(px, b % 3) * q2_at(py, (b / 3) % 3) * q2_at(pz, b / 9);
        if (w == 0.0) continue;
        const int32_t node = cn[b];
        if (!idx_ok(C.dbg, OCT_CELL_NODES, node, (long long)C.nn, size_t(par) * 27 + b)) continue;
        if (C.flags[node] & 1) continue;
        for (int c = 0; c < 3; ++c) atomicAdd(coarse + c * C.nn + node, T(w) * f[c]);
    }
}

template <typename T>
__global__ void k_oct_copy_to_level(size_t n, const int32_t* __restrict__ ai, const int32_t* __restrict__ li,
                                    size_t nu, size_t nn, const double* __restrict__ active, T* __restrict__ level,
                                    OctDebug dbg) {
    const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (!idx_ok(dbg, OCT_COPY_ACTIVE, ai[t], (long long)nu, t) || !idx_ok(dbg, OCT_COPY_LEVEL, li[t], (long long)nn, t))
        return;
    for (int c = 0; c < 3; ++c) level[c * nn + li[t]] = T(active[c * nu + ai[t]]);
}

template <typename T>
__global__ void k_oct_copy_from_level(size_t n, const int32_t* __restrict__ ai, const int32_t* __restrict__ li,
                                      size_t nu, size_t nn, const T* __restrict__ level, double* __restrict__ active,
                                      OctDebug dbg) {
    const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (!idx_ok(dbg, OCT_COPY_ACTIVE, ai[t], (long long)nu, t) || !idx_ok(dbg, OCT_COPY_LEVEL, li[t], (long long)nn, t))
        return;
    for (int c = 0; c < 3; ++c) active[c * nu + ai[t]] = double(level[c * nn + li[t]]);
}

// ---- active blocks with hanging-node constraints
// A reference r read at position `at` of leaf_u / leaf_p is a node (r >= 0) or constraint -r-1.
__device__ __forceinline__ double gather_u(const OctActiveDev& a, const double* src, int c, int32_t r, size_t at) {
    if (r >= 0) {
        if (!idx_ok(a.dbg, OCT_LEAF_U, r, (long long)a.nu_nodes, at)) return 0.0;
        return a.ubnd[r] ? 0.0 : src[c * a.nu_nodes + r];
    }
    const long long k = -(long long)r - 1;
    if (!idx_ok(a.dbg, OCT_LEAF_U, k, (long long)a.n_ucon, at)) return 0.0;
    const int32_t* nd = a.ucon_node + size_t(k) * kOctUCon;
    const double* wt = a.ucon_w + size_t(k) * kOctUCon;
    double v = 0.0;
#pragma unroll 1
    for (int t = 0; t < kOctUCon; ++t) {
        const int32_t node = nd[t];
        if (node < 0) break;
        if (!idx_ok(a.dbg, OCT_UCON_NODE, node, (long long)a.nu_nodes, size_t(k) * kOctUCon + t)) continue;
        if (!a.ubnd[node]) v += wt[t] * src[c * a.nu_nodes + node];
    }
    return v;
}
__device__ __forceinline__ void scatter_u(const OctActiveDev& a, double* dst, int c, int32_t r, double v, size_t at) {
    if (r >= 0) {
        if (!idx_ok(a.dbg, OCT_LEAF_U, r, (long long)a.nu_nodes, at)) return;
        if (!a.ubnd[r]) atomicAdd(dst + c * a.nu_nodes + r, v);
        return;
    }
    const long long k = -(long long)r - 1;
    if (!idx_ok(a.dbg, OCT_LEAF_U, k, (long long)a.n_ucon, at)) return;
    const int32_t* nd = a.ucon_node + size_t(k) * kOctUCon;
    const double* wt = a.ucon_w + size_t(k) * kOctUCon;
#pragma unroll 1
    for (int t = 0; t < kOctUCon; ++t) {
        const int32_t node = nd[t];
        if (node < 0) break;
        if (!idx_ok(a.dbg, OCT_UCON_NODE, node, (long long)a.nu_nodes, size_t(k) * kOctUCon + t)) continue;
        if (!a.ubnd[node]) atomicAdd(dst + c * a.nu_nodes + node, wt[t] * v);
    }
}
__device__ __forceinline__ double gather_p(const OctActiveDev& a, const double* src, int32_t r, size_t at) {
    if (r >= 0) return idx_ok(a.dbg, OCT_LEAF_P, r, (long long)a.np, at) ? src[r] : 0.0;
    const long long k = -(long long)r - 1;
    if (!idx_ok(a.dbg, OCT_LEAF_P, k, (long long)a.n_pcon, at)) return 0.0;
    const int32_t* nd = a.pcon_node + size_t(k) * kOctPCon;
    const double* wt = a.pcon_w + size_t(k) * kOctPCon;
    double v = 0.0;
#pragma unroll 1
    for (int t = 0; t < kOctPCon; ++t) {
        if (nd[t] < 0) break;
        if (!idx_ok(a.dbg, OCT_PCON_NODE, nd[t], (long long)a.np, size_t(k) * kOctPCon + t)) continue;
        v += wt[t] * src[nd[t]];
    }
    return v;
}
__device__ __forceinline__ void scatter_p(const OctActiveDev& a, double* dst, int32_t r, double v, size_t at) {
    if (r >= 0) {
        if (idx_ok(a.dbg, OCT_LEAF_P, r, (long long)a.np, at)) atomicAdd(dst + r, v);
        return;
    }
    const long long k = -(long long)r - 1;
    if (!idx_ok(a.dbg, OCT_LEAF_P, k, (long long)a.n_pcon, at)) return;
    const int32_t* nd = a.pcon_node + size_t(k) * kOctPCon;
    const double* wt = a.pcon_w + size_t(k) * kOctPCon;
#pragma unroll 1
    for (int t = 0; t < kOctPCon; ++t) {
        if (nd[t] < 0) break;
        if (!idx_ok(a.dbg, OCT_PCON_NODE, nd[t], (long long)a.np, size_t(k) * kOctPCon + t)) continue;
        atomicAdd(dst + nd[t], wt[t] * v);
    }
}

template <bool DO_A, bool DO_BT, bool DO_B>
__global__ void __launch_bounds__(128) k_oct_active(OctActiveDev a, const double* __restrict__ src_u,
                                                    const double* __restrict__ src_p, double* __restrict__ dst_u,
                                                    double* __restrict__ dst_p) {
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= a.n_leaves) return;
    const int32_t* ru = a.leaf_u + size_t(leaf) * 27;
    const int32_t* rp = a.leaf_p + size_t(leaf) * 8;
    const double h = ldexp(1.0, -int(a.level[leaf]));
    const double s = -h * h;
    double w[3][27];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 27; ++m) w[c][m] = 0.0;
    if (DO_A || DO_B) {
        double u[3][27];
#pragma unroll
        for (int m = 0; m < 27; ++m) {
            const int32_t r = ru[m];
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c][m] = gather_u(a, src_u, c, r, size_t(leaf) * 27 + m);
        }
        if (DO_B) {
            double pb[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) pb[v] = 0.0;
            q2::b_component<0>(u[0], pb);
            q2::b_component<1>(u[1], pb);
            q2::b_component<2>(u[2], pb);
#pragma unroll
            for (int v = 0; v < 8; ++v) scatter_p(a, dst_p, rp[v], s * pb[v], size_t(leaf) * 8 + v);
        }
        if (DO_A) {
            q2::cell_A(u, w);
            const double sa = a.mu[leaf] * h;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int m = 0; m < 27; ++m) w[c][m] *= sa;
        }
    }
    if (DO_BT) {
        double p8[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) p8[v] = s * gather_p(a, src_p, rp[v], size_t(leaf) * 8 + v);
        q2::bt_component<0>(p8, w[0]);
        q2::bt_component<1>(p8, w[1]);
        q2::bt_component<2>(p8, w[2]);
    }
    if (DO_A || DO_BT) {
#pragma unroll
        for (int m = 0; m < 27; ++m) {
            const int32_t r = ru[m];
#pragma unroll
            for (int c = 0; c < 3; ++c) scatter_u(a, dst_u, c, r, w[c][m], size_t(leaf) * 27 + m);
        }
    }
}

__global__ void k_oct_active_boundary(OctActiveDev a, const double* __restrict__ src_u, double* __restrict__ dst_u) {
    const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= a.nu_nodes || !a.ubnd[n]) return;
    for (int c = 0; c < 3; ++c) dst_u[c * a.nu_nodes + n] = src_u[c * a.nu_nodes + n];
}

__global__ void k_oct_mass_p(OctActiveDev a, const double* __restrict__ src, double* __restrict__ dst) {
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= a.n_leaves) return;
    const int32_t* rp = a.leaf_p + size_t(leaf) * 8;
    const double h = ldexp(1.0, -int(a.level[leaf]));
    const double sc = h * h * h / a.mu[leaf];
    double p[8];
    for (int v = 0; v < 8; ++v) p[v] = gather_p(a, src, rp[v], size_t(leaf) * 8 + v);
    for (int v = 0; v < 8; ++v) {
        double o = 0.0;
        for (int q = 0; q < 8; ++q) {
            double m = 1.0;
            for (int d = 0; d < 3; ++d) m *= (((v >> d) & 1) == ((q >> d) & 1)) ? (1.0 / 3.0) : (1.0 / 6.0);
            o += m * p[q];
        }
        scatter_p(a, dst, rp[v], sc * o, size_t(leaf) * 8 + v);
    }
}

}  // namespace

const char* oct_table_name(int table) {
    static const char* names[OCT_NTABLES] = {"cell_nodes", "parent", "pos", "leaf_u", "ucon_node",
                                             "leaf_p", "pcon_node", "copy_active", "copy_level"};
    return table >= 0 && table < OCT_NTABLES ? names[table] : "?";
}

template <typename T>
cudaError_t launch_oct_level_cells(const OctLevelDev& L, const T* mu, const T* src, T* acc, cudaStream_t s) {
    if (L.n_cells == 0) return cudaSuccess;
    LAUNCH(sizeof(T) == 4 ? PROF_VMULT_F32 : PROF_VMULT_F64, s,
           (k_oct_cells<T><<<blocks_for(L.n_cells, 128), 128, 0, s>>>(L, mu, src, acc)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oct_copy_boundary(const OctLevelDev& L, const T* src, T* dst, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, (k_oct_copy_boundary<T><<<blocks_for(L.nn, 256), 256, 0, s>>>(L, src, dst)));
    return cudaGetLastError();
}

cudaError_t launch_oct_inv_diag(const OctLevelDev& L, const double* mu, const double* ref_diag81, double* tmp,
                                double* dinv, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tmp, 0, 3 * L.nn * sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (L.n_cells) LAUNCH(PROF_SMOOTH_VEC, s, (k_oct_diag<<<blocks_for(L.n_cells, 128), 128, 0, s>>>(L, mu, ref_diag81, tmp)));
    LAUNCH(PROF_SMOOTH_VEC, s, (k_oct_dinv<<<blocks_for(L.nn, 256), 256, 0, s>>>(L, tmp, dinv)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oct_prolongate(const OctLevelDev& F, const OctLevelDev& C, const T* coarse, T* fine, bool add,
                                  cudaStream_t s) {
    LAUNCH(PROF_TRANSFER, s, (k_oct_prolongate<T><<<blocks_for(F.nn, 128), 128, 0, s>>>(F, C, coarse, fine, add)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oct_restrict_add(const OctLevelDev& F, const OctLevelDev& C, const T* fine, T* coarse,
                                    cudaStream_t s) {
    LAUNCH(PROF_TRANSFER, s, (k_oct_restrict_add<T><<<blocks_for(F.nn, 128), 128, 0, s>>>(F, C, fine, coarse)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oct_copy_to_level(size_t n_copy, const int32_t* active_idx, const int32_t* level_idx,
                                     size_t nu_nodes, size_t level_nn, const double* active, T* level,
                                     const OctDebug& dbg, cudaStream_t s) {
    if (n_copy == 0) return cudaSuccess;
    LAUNCH(PROF_CAST, s, (k_oct_copy_to_level<T><<<blocks_for(n_copy, 256), 256, 0, s>>>(
                             n_copy, active_idx, level_idx, nu_nodes, level_nn, active, level, dbg)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oct_copy_from_level(size_t n_copy, const int32_t* active_idx, const int32_t* level_idx,
                                       size_t nu_nodes, size_t level_nn, const T* level, double* active,
                                       const OctDebug& dbg, cudaStream_t s) {
    if (n_copy == 0) return cudaSuccess;
    LAUNCH(PROF_CAST, s, (k_oct_copy_from_level<T><<<blocks_for(n_copy, 256), 256, 0, s>>>(
                             n_copy, active_idx, level_idx, nu_nodes, level_nn, level, active, dbg)));
    return cudaGetLastError();
}

cudaError_t launch_oct_active(const OctActiveDev& a, const double* src_u, const double* src_p, double* dst_u,
                              double* dst_p, bool do_a, bool do_bt, bool do_b, cudaStream_t s) {
    cudaError_t e;
    if ((do_a || do_bt) && (e = cudaMemsetAsync(dst_u, 0, 3 * a.nu_nodes * sizeof(double), s)) != cudaSuccess) return e;
    if (do_b && (e = cudaMemsetAsync(dst_p, 0, a.np * sizeof(double), s)) != cudaSuccess) return e;
    const unsigned g = blocks_for(a.n_leaves, 128);
    const int cls = do_a ? PROF_STOKES_F64 : (do_bt ? PROF_BT_F64 : PROF_STOKES_F64);
    if (do_a && do_bt && do_b) LAUNCH(cls, s, (k_oct_active<true, true, true><<<g, 128, 0, s>>>(a, src_u, src_p, dst_u, dst_p)));
    else if (do_a && !do_bt && !do_b) LAUNCH(cls, s, (k_oct_active<true, false, false><<<g, 128, 0, s>>>(a, src_u, src_p, dst_u, dst_p)));
    else if (!do_a && do_bt && !do_b) LAUNCH(cls, s, (k_oct_active<false, true, false><<<g, 128, 0, s>>>(a, src_u, src_p, dst_u, dst_p)));
    else if (!do_a && !do_bt && do_b) LAUNCH(cls, s, (k_oct_active<false, false, true><<<g, 128, 0, s>>>(a, src_u, src_p, dst_u, dst_p)));
    else return cudaErrorInvalidValue;
    if (do_a) LAUNCH(cls, s, (k_oct_active_boundary<<<blocks_for(a.nu_nodes, 256), 256, 0, s>>>(a, src_u, dst_u)));
    return cudaGetLastError();
}

cudaError_t launch_oct_identity_rows(const OctActiveDev& a, const double* src_u, double* dst_u, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, (k_oct_active_boundary<<<blocks_for(a.nu_nodes, 256), 256, 0, s>>>(a, src_u, dst_u)));
    return cudaGetLastError();
}

cudaError_t launch_oct_mass_p(const OctActiveDev& a, const double* src, double* dst, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(dst, 0, a.np * sizeof(double), s);
    if (e != cudaSuccess) return e;
    LAUNCH(PROF_MASS_P, s, (k_oct_mass_p<<<blocks_for(a.n_leaves, 128), 128, 0, s>>>(a, src, dst)));
    return cudaGetLastError();
}

#define INST(T)                                                                                                     \
    template cudaError_t launch_oct_level_cells<T>(const OctLevelDev&, const T*, const T*, T*, cudaStream_t);      \
    template cudaError_t launch_oct_copy_boundary<T>(const OctLevelDev&, const T*, T*, cudaStream_t);              \
    template cudaError_t launch_oct_prolongate<T>(const OctLevelDev&, const OctLevelDev&, const T*, T*, bool,      \
                                                  cudaStream_t);                                                  \
    template cudaError_t launch_oct_restrict_add<T>(const OctLevelDev&, const OctLevelDev&, const T*, T*,          \
                                                    cudaStream_t);                                                \
    template cudaError_t launch_oct_copy_to_level<T>(size_t, const int32_t*, const int32_t*, size_t, size_t,       \
                                                     const double*, T*, const OctDebug&, cudaStream_t);           \
    template cudaError_t launch_oct_copy_from_level<T>(size_t, const int32_t*, const int32_t*, size_t, size_t,     \
                                                       const T*, double*, const OctDebug&, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace stk
