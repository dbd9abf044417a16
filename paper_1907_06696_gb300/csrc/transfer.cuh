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

}  // namespace stk
