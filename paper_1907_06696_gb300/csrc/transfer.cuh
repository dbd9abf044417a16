// transfer.cuh -- per-node bodies of the Q2 level transfers (Section 2.2.1, GMG transfer):
// prolongation = evaluation of the coarse Q2 field at the fine nodes (1D weights at 0, 1/4, 1/2,
// 3/4, 1 of a coarse cell: [1,0,0], [3/8,3/4,-1/8], [0,1,0], [-1/8,3/4,3/8], [0,0,1]); restriction
// = its transpose; boundary nodes zero. Shared by the transfer kernels (vec.cu) and the batched
// V-cycle (batch.cu). CG = true reads the input through L2 only (ld.global.cg), for kernels that
// read vectors other blocks of the same launch have written.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace stk {

template <typename T, bool CG>
__device__ __forceinline__ T load_vec(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

__device__ __forceinline__ bool on_bnd(int gi, int M) { return gi == 0 || gi == M - 1; }

// Coarse nodes and weights feeding fine node index f (one axis).
__device__ __forceinline__ int pro_axis(int f, int* idx, float* wt) {
    if ((f & 1) == 0) { idx[0] = f >> 1; wt[0] = 1.0f; return 1; }
    const int m = f >> 2;
    idx[0] = 2 * m; idx[1] = 2 * m + 1; idx[2] = 2 * m + 2;
    if ((f & 3) == 1) { wt[0] = 0.375f; wt[1] = 0.75f; wt[2] = -0.125f; }
    else { wt[0] = -0.125f; wt[1] = 0.75f; wt[2] = 0.375f; }
    return 3;
}

// Fine nodes and weights of coarse node index c (one axis), nc coarse cells.
__device__ __forceinline__ int res_axis(int c, int nc, int* idx, float* wt) {
    int k = 0;
    if (c & 1) {
        const int m = c >> 1;
        idx[k] = 4 * m + 2; wt[k++] = 1.0f;
        idx[k] = 4 * m + 1; wt[k++] = 0.75f;
        idx[k] = 4 * m + 3; wt[k++] = 0.75f;
        return k;
    }
    const int m = c >> 1;
    idx[k] = 4 * m; wt[k++] = 1.0f;
    if (m < nc) { idx[k] = 4 * m + 1; wt[k++] = 0.375f; idx[k] = 4 * m + 3; wt[k++] = -0.125f; }
    if (m >= 1) { idx[k] = 4 * m - 1; wt[k++] = 0.375f; idx[k] = 4 * m - 3; wt[k++] = -0.125f; }
    return k;
}

// Fine node `node` of a level with nf cells per axis: fine (+)= P coarse.
template <typename T, bool CG>
__device__ __forceinline__ void prolongate_node(int nf, const T* coarse, T* fine, bool add, size_t node) {
    const int Mf = 2 * nf + 1, Mc = nf + 1;
    const size_t nodes_f = size_t(Mf) * Mf * Mf, nodes_c = size_t(Mc) * Mc * Mc;
    const int i = int(node % Mf), j = int((node / Mf) % Mf), k = int(node / (size_t(Mf) * Mf));
    if (on_bnd(i, Mf) || on_bnd(j, Mf) || on_bnd(k, Mf)) {
        if (!add)
            for (int c = 0; c < 3; ++c) fine[c * nodes_f + node] = T(0);
        return;
    }
    int ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    const int nx = pro_axis(i, ix, wx), ny = pro_axis(j, iy, wy), nz = pro_axis(k, iz, wz);
    T acc[3] = {T(0), T(0), T(0)};
    for (int c3 = 0; c3 < nz; ++c3)
        for (int c2 = 0; c2 < ny; ++c2) {
            const T wyz = T(wy[c2]) * T(wz[c3]);
            const size_t base = size_t(Mc) * (iy[c2] + size_t(Mc) * iz[c3]);
            for (int c1 = 0; c1 < nx; ++c1) {
                const T wgt = wyz * T(wx[c1]);
                const size_t cn = base + ix[c1];
                for (int c = 0; c < 3; ++c) acc[c] += wgt * load_vec<T, CG>(coarse + c * nodes_c + cn);
            }
        }
    for (int c = 0; c < 3; ++c) {
        if (add) fine[c * nodes_f + node] = load_vec<T, CG>(fine + c * nodes_f + node) + acc[c];
        else fine[c * nodes_f + node] = acc[c];
    }
}

// Coarse node `node` of the level below one with nf cells per axis: coarse = P^T fine.
template <typename T, bool CG>
__device__ __forceinline__ void restrict_node(int nf, const T* fine, T* coarse, size_t node) {
    const int Mf = 2 * nf + 1, Mc = nf + 1, nc = nf / 2;
    const size_t nodes_f = size_t(Mf) * Mf * Mf, nodes_c = size_t(Mc) * Mc * Mc;
    const int i = int(node % Mc), j = int((node / Mc) % Mc), k = int(node / (size_t(Mc) * Mc));
    if (on_bnd(i, Mc) || on_bnd(j, Mc) || on_bnd(k, Mc)) {
        for (int c = 0; c < 3; ++c) coarse[c * nodes_c + node] = T(0);
        return;
    }
    int ix[5], iy[5], iz[5];
    float wx[5], wy[5], wz[5];
    const int nx = res_axis(i, nc, ix, wx), ny = res_axis(j, nc, iy, wy), nz = res_axis(k, nc, iz, wz);
    T acc[3] = {T(0), T(0), T(0)};
    for (int c3 = 0; c3 < nz; ++c3)
        for (int c2 = 0; c2 < ny; ++c2) {
            const T wyz = T(wy[c2]) * T(wz[c3]);
            const size_t base = size_t(Mf) * (iy[c2] + size_t(Mf) * iz[c3]);
            for (int c1 = 0; c1 < nx; ++c1) {
                const T wgt = wyz * T(wx[c1]);
                const size_t fn = base + ix[c1];
                for (int c = 0; c < 3; ++c) acc[c] += wgt * load_vec<T, CG>(fine + c * nodes_f + fn);
            }
        }
    for (int c = 0; c < 3; ++c) coarse[c * nodes_c + node] = acc[c];
}

// ---- transfers by coarse cells (sum-factorised), the bodies of k_prolong_cells and
// k_restrict_cells (vec.cu); plain functions of the thread's (component, plane, cell), so that a
// host program can run them cell by cell. A coarse cell C has the 3 x 3 x 3 coarse nodes
// 2C + {0,1,2} and the 5 x 5 x 5 fine nodes 4C + {0..4}. Along one axis the fine values at 0, 1/4,
// 1/2, 3/4, 1 of the coarse cell are
//   p0 = a0, p1 = 3/8 a0 + 3/4 a1 - 1/8 a2, p2 = a1, p3 = -1/8 a0 + 3/4 a1 + 3/8 a2, p4 = a2,
// and restriction applies the transpose. A fine node shared by neighbouring coarse cells belongs to
// the cell in which its local index is 0..3 along each axis (4 in the last cell along that axis), so
// each is written (prolongation) or counted (restriction) once; the Q2 field is continuous, so the
// owner's values are everyone's.
template <typename T>
__host__ __device__ __forceinline__ void pro5(T a0, T a1, T a2, T (&p)[5]) {
    p[0] = a0;
    p[1] = T(0.375) * a0 + T(0.75) * a1 - T(0.125) * a2;
    p[2] = a1;
    p[3] = T(-0.125) * a0 + T(0.75) * a1 + T(0.375) * a2;
    p[4] = a2;
}
template <typename T>
__host__ __device__ __forceinline__ void res3(const T (&v)[5], T& o0, T& o1, T& o2) {
    o0 = v[0] + T(0.375) * v[1] - T(0.125) * v[3];
    o1 = T(0.75) * v[1] + v[2] + T(0.75) * v[3];
    o2 = T(-0.125) * v[1] + T(0.375) * v[3] + v[4];
}

template <typename T>
__host__ __device__ __forceinline__ void add_to(T* p, T v) {
#ifdef __CUDA_ARCH__
    atomicAdd(p, v);
#else
    *p += v;
#endif
}

// fine (+)= P coarse on fine plane z (0..4) of coarse cell `cell`, component c (fine boundary nodes:
// 0, or left unchanged with add): the x and y sweeps of the cell's 27 values and the z
// interpolation for the plane; the 25 old values of the plane are loaded before any is stored, so
// that the thread's memory round trips do not line up one behind the other.
template <typename T>
__host__ __device__ __forceinline__ void prolong_cell_plane(int nc, const T* __restrict__ coarse,
                                                            T* __restrict__ fine, bool add, int c, int z,
                                                            size_t cell) {
    const int ci = int(cell % nc), cj = int((cell / nc) % nc), ck = int(cell / (size_t(nc) * nc));
    if (z == 4 && ck != nc - 1) return;   // that plane belongs to the next cell along z
    const int Mc = 2 * nc + 1, Mf = 4 * nc + 1;
    const size_t nodes_c = size_t(Mc) * Mc * Mc, nodes_f = size_t(Mf) * Mf * Mf;
    const T* cp = coarse + size_t(c) * nodes_c + (size_t(2 * ci) + size_t(Mc) * (size_t(2 * cj) + size_t(Mc) * 2 * ck));
    T t1[5][3][3];   // [x][b][d] after the x sweep
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T* r = cp + size_t(Mc) * (b + size_t(Mc) * d);
            T p[5];
            pro5(r[0], r[1], r[2], p);
#pragma unroll
            for (int x = 0; x < 5; ++x) t1[x][b][d] = p[x];
        }
    // the z weights of this plane (row z of the 5 x 3 interpolation)
    const T wz0 = z == 0 ? T(1) : z == 1 ? T(0.375) : z == 3 ? T(-0.125) : T(0);
    const T wz1 = z == 1 || z == 3 ? T(0.75) : z == 2 ? T(1) : T(0);
    const T wz2 = z == 4 ? T(1) : z == 1 ? T(-0.125) : z == 3 ? T(0.375) : T(0);
    const bool lx = ci == nc - 1, ly = cj == nc - 1;
    const bool bz = (4 * ck + z == 0) || (4 * ck + z == Mf - 1);
    T* fp = fine + size_t(c) * nodes_f + (size_t(4 * ci) + size_t(Mf) * (size_t(4 * cj) + size_t(Mf) * (4 * ck + z)));
    T out[5][5];
#pragma unroll
    for (int x = 0; x < 5; ++x) {
        T p[5];
#pragma unroll
        for (int y = 0; y < 5; ++y) p[y] = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const T w = d == 0 ? wz0 : d == 1 ? wz1 : wz2;
            T q[5];
            pro5(t1[x][0][d], t1[x][1][d], t1[x][2][d], q);
#pragma unroll
            for (int y = 0; y < 5; ++y) p[y] += w * q[y];
        }
#pragma unroll
        for (int y = 0; y < 5; ++y) out[x][y] = p[y];
    }
    // owned nodes of the plane: x, y in 0..3 (4 in the last cell along the axis)
    auto owned = [&](int x, int y) { return (x < 4 || lx) && (y < 4 || ly); };
    auto bnd = [&](int x, int y) {
        return bz || (4 * ci + x == 0) || (4 * ci + x == Mf - 1) || (4 * cj + y == 0) || (4 * cj + y == Mf - 1);
    };
    if (add) {
        T old[5][5];
#pragma unroll
        for (int y = 0; y < 5; ++y)
#pragma unroll
            for (int x = 0; x < 5; ++x) old[x][y] = owned(x, y) && !bnd(x, y) ? fp[x + size_t(Mf) * y] : T(0);
#pragma unroll
        for (int y = 0; y < 5; ++y)
#pragma unroll
            for (int x = 0; x < 5; ++x)
                if (owned(x, y) && !bnd(x, y)) fp[x + size_t(Mf) * y] = old[x][y] + out[x][y];
    } else {
#pragma unroll
        for (int y = 0; y < 5; ++y)
#pragma unroll
            for (int x = 0; x < 5; ++x)
                if (owned(x, y)) fp[x + size_t(Mf) * y] = bnd(x, y) ? T(0) : out[x][y];
    }
}

// coarse += P^T r on the free coarse nodes of coarse cell `cell`, component c, from the fine nodes
// the cell owns (coarse zero on entry; neighbouring cells add to shared coarse nodes, atomically
// on the device).
template <typename T>
__host__ __device__ __forceinline__ void restrict_cell(int nc, const T* __restrict__ fine_r, T* __restrict__ coarse,
                                                       int c, size_t cell) {
    const int ci = int(cell % nc), cj = int((cell / nc) % nc), ck = int(cell / (size_t(nc) * nc));
    const int Mc = 2 * nc + 1, Mf = 4 * nc + 1;
    const size_t nodes_c = size_t(Mc) * Mc * Mc, nodes_f = size_t(Mf) * Mf * Mf;
    const bool lx = ci == nc - 1, ly = cj == nc - 1, lz = ck == nc - 1;
    const size_t fbase = size_t(c) * nodes_f + (size_t(4 * ci) + size_t(Mf) * (size_t(4 * cj) + size_t(Mf) * 4 * ck));
    T t2[5][5][3];   // [x][y][d] after the z sweep
#pragma unroll
    for (int y = 0; y < 5; ++y)
#pragma unroll
        for (int x = 0; x < 5; ++x) {
            T v[5];
#pragma unroll
            for (int z = 0; z < 5; ++z) {
                const bool own = (x < 4 || lx) && (y < 4 || ly) && (z < 4 || lz);
                const size_t f = fbase + x + size_t(Mf) * (y + size_t(Mf) * z);
                v[z] = own ? fine_r[f] : T(0);
            }
            res3(v, t2[x][y][0], t2[x][y][1], t2[x][y][2]);
        }
    T t1[5][3][3];   // [x][b][d]
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int x = 0; x < 5; ++x) {
            T v[5];
#pragma unroll
            for (int y = 0; y < 5; ++y) v[y] = t2[x][y][d];
            res3(v, t1[x][0][d], t1[x][1][d], t1[x][2][d]);
        }
    T* cp = coarse + size_t(c) * nodes_c + (size_t(2 * ci) + size_t(Mc) * (size_t(2 * cj) + size_t(Mc) * 2 * ck));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const bool bd = (2 * ck + d == 0) || (2 * ck + d == Mc - 1);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            const bool bb_ = bd || (2 * cj + bb == 0) || (2 * cj + bb == Mc - 1);
            T v[5];
#pragma unroll
            for (int x = 0; x < 5; ++x) v[x] = t1[x][bb][d];
            T o[3];
            res3(v, o[0], o[1], o[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (bb_ || (2 * ci + a == 0) || (2 * ci + a == Mc - 1)) continue;
                add_to(cp + a + size_t(Mc) * (bb + size_t(Mc) * d), o[a]);
            }
        }
    }
}

}  // namespace stk
