// brick.cuh -- the velocity operator A_l (Section 2.1, definition of A) as a
// deterministic, atomic-free, brick-tiled kernel with a fused vector epilogue
// (the Jacobi-Chebyshev update of Section 2.2.1, a residual, or a plain product).
//
// Work decomposition: the n^3 cells of a level are cut into bricks of
// BX x BY x BZ cells, one CTA per brick, one thread per cell.
//   1. Each thread gathers its cell's 81 values from global memory (neighbouring
//      cells of the brick hit the same L1 lines; constrained nodes read as 0)
//      and applies q2::cell_A in registers (results times mu h).
//   2. Every node of the brick has one owner cell: the cell in which its local
//      index is 0 or 1 along each axis, or 2 where the cell is the last one of
//      the brick along that axis. Each thread exports its 19 local nodes that
//      have an index 2 (57 values) to a shared buffer laid out [57][cells]
//      (consecutive threads, consecutive words: no bank conflicts).
//   3. After one barrier, each thread sums each node it owns: its own value
//      plus the exported values of the <= 7 neighbouring cells of the brick
//      that contain the node, at compile-time offsets, in a fixed order (no
//      atomics, deterministic), and stores the sum in a shared node tile.
//   4. After a second barrier, one compact loop over the tile's node rows runs
//      the epilogue (kept out of the unrolled code so the kernel stays small
//      enough for the instruction cache).
//      - A node strictly inside the brick is complete: the epilogue runs now.
//      - A node on an internal brick plane (node index a multiple of 2B along
//        some axis, not on the domain boundary) is shared with 2, 4 or 8
//        bricks: this brick writes its partial sum to its own slot (one slot
//        per brick side) and the plane kernel later adds the slots and runs
//        the epilogue.
//      - A boundary node gets the identity row: the epilogue sees Ax = x.
// In-place update of x in the Chebyshev epilogue is safe: a node strictly
// inside a brick is staged by that brick only, and plane nodes are updated by
// the plane kernel after every brick has finished reading.
//
// The phases are plain functions of (thread, brick) so that a host program can
// run them block by block and check every index against its buffer.
#pragma once

#include "internal.cuh"
#include "q2_basis.cuh"

namespace stk {

enum Epilogue { EPI_PLAIN = 0, EPI_RESID = 1, EPI_CHEB = 2 };

// Brick shape used by the library (cells per brick along x, y, z; one thread per cell).
constexpr int kBrickX = 8, kBrickY = 4, kBrickZ = 4;

// Slot storage for the nodes on internal brick planes of one level. A node
// on the planes of the axis set P (bitmask x=1, y=2, z=4) is shared by 2^|P|
// bricks; the brick on the upper side along axis d (the node is its local
// index 0 there) sets bit rank_P(d) of its slot number.
struct PlaneLayout {
    int M;             // nodes per axis, 2n + 1
    int B[3];          // cells per brick along each axis
    int np[3];         // internal planes per axis (bricks per axis - 1)
    size_t F[8];       // entries per (slot, component) of family P
    size_t off[8];     // offset of family P
    size_t total;      // entries of all families
};

inline PlaneLayout make_plane_layout(int n, int bx, int by, int bz) {
    PlaneLayout L{};
    L.M = 2 * n + 1;
    const int B[3] = {bx, by, bz};
    for (int d = 0; d < 3; ++d) {
        L.B[d] = B[d];
        const int nb = (n + B[d] - 1) / B[d];
        L.np[d] = nb - 1;
    }
    size_t off = 0;
    for (int P = 1; P < 8; ++P) {
        size_t F = 1;
        for (int d = 0; d < 3; ++d) F *= ((P >> d) & 1) ? size_t(L.np[d]) : size_t(L.M);
        L.F[P] = F;
        L.off[P] = off;
        const int slots = 1 << __builtin_popcount(P);
        off += size_t(slots) * 3 * F;
    }
    L.total = off;
    return L;
}

__host__ __device__ __forceinline__ bool on_plane(int g, int twoB, int M) {
    return g > 0 && g < M - 1 && (g % twoB) == 0;
}

__host__ __device__ __forceinline__ size_t plane_entry(const PlaneLayout& L, int P, int slot, int c, int gi, int gj,
                                                       int gk) {
    const int g[3] = {gi, gj, gk};
    size_t e[3], E[3];
    for (int d = 0; d < 3; ++d) {
        if ((P >> d) & 1) {
            e[d] = size_t(g[d] / (2 * L.B[d]) - 1);
            E[d] = size_t(L.np[d]);
        } else {
            e[d] = size_t(g[d]);
            E[d] = size_t(L.M);
        }
    }
    return L.off[P] + (size_t(slot) * 3 + c) * L.F[P] + e[0] + E[0] * (e[1] + E[1] * e[2]);
}

template <typename T>
struct BrickArgs {
    int n, M;
    size_t nodes;
    T h;
    const T* mu;     // cell viscosity
    const T* src;    // operand x (for EPI_CHEB also updated in place)
    T* dst;          // EPI_PLAIN: A x; EPI_RESID: b - A x
    const T* b;      // right-hand side (EPI_RESID, EPI_CHEB)
    const T* dinv;   // inverse diagonal (EPI_CHEB)
    T* d;            // Chebyshev direction (EPI_CHEB)
    T c1, c2;        // d <- c1 d + c2 dinv (b - A x); x <- x + d
    T* slots;        // PlaneLayout.total entries
    PlaneLayout L;
};

// Epilogue for one DoF with the complete product ax.
template <typename T, int EPI>
__host__ __device__ __forceinline__ void epilogue(const BrickArgs<T>& a, size_t i, T ax) {
    if (EPI == EPI_PLAIN) {
        a.dst[i] = ax;
    } else if (EPI == EPI_RESID) {
        a.dst[i] = a.b[i] - ax;
    } else {
        const T r = a.dinv[i] * (a.b[i] - ax);
        const T dn = (a.c1 != T(0) ? a.c1 * a.d[i] : T(0)) + a.c2 * r;
        a.d[i] = dn;
        const_cast<T*>(a.src)[i] = a.src[i] + dn;
    }
}

// Epilogue of a constrained (boundary) DoF: identity row, A x = x.
template <typename T, int EPI>
__host__ __device__ __forceinline__ void epilogue_boundary(const BrickArgs<T>& a, size_t i) {
    if (EPI == EPI_PLAIN) a.dst[i] = a.src[i];
    else if (EPI == EPI_RESID) a.dst[i] = T(0);
    // EPI_CHEB: dinv = 0 and d = 0 there, so x and d are unchanged
}

template <int BX, int BY, int BZ>
struct BrickShape {
    static constexpr int TX = 2 * BX + 1, TY = 2 * BY + 1, TZ = 2 * BZ + 1;
    static constexpr int TILE = TX * TY * TZ;     // nodes per brick tile
    static constexpr int NC = BX * BY * BZ;       // cells (= threads) per brick
    // exported values (19 nodes x 3 components per cell) + the node tile (3 components)
    static constexpr int EXPORT = 57 * NC;
    template <typename T>
    static constexpr size_t smem_bytes() { return sizeof(T) * (size_t(EXPORT) + size_t(3) * TILE); }
};

// Plane slot index with the brick shape known at compile time.
template <int BX, int BY, int BZ>
__host__ __device__ __forceinline__ size_t plane_entry_c(const PlaneLayout& L, int P, int slot, int c, int gi, int gj,
                                                         int gk) {
    const size_t M = size_t(L.M);
    const size_t ex = (P & 1) ? size_t(gi / (2 * BX) - 1) : size_t(gi);
    const size_t ey = (P & 2) ? size_t(gj / (2 * BY) - 1) : size_t(gj);
    const size_t ez = (P & 4) ? size_t(gk / (2 * BZ) - 1) : size_t(gk);
    const size_t Ex = (P & 1) ? size_t(L.np[0]) : M;
    const size_t Ey = (P & 2) ? size_t(L.np[1]) : M;
    return L.off[P] + (size_t(slot) * 3 + c) * L.F[P] + ex + Ex * (ey + Ey * ez);
}



// Position of local node (i,j,k) among the 19 local nodes with some index equal to 2
// (lexicographic in k, j, i); only called for such nodes.
__host__ __device__ __forceinline__ constexpr int export_index(int i, int j, int k) {
    int e = 0;
    for (int kk = 0; kk < 3; ++kk)
        for (int jj = 0; jj < 3; ++jj)
            for (int ii = 0; ii < 3; ++ii) {
                if (ii == i && jj == j && kk == k) return e;
                if (ii == 2 || jj == 2 || kk == 2) ++e;
            }
    return -1;
}

// Phase 1: one cell per thread: gather from global memory and apply the operator in registers.
// Returns false for a thread whose cell lies outside the level.
template <typename T, int BX, int BY, int BZ>
__host__ __device__ __forceinline__ bool brick_compute(const BrickArgs<T>& a, int bx, int by, int bz, int tid,
                                                       T (&w)[3][27]) {
    const int cx = tid % BX, cy = (tid / BX) % BY, cz = tid / (BX * BY);
    const int ci = BX * bx + cx, cj = BY * by + cy, ck = BZ * bz + cz;
    if (ci >= a.n || cj >= a.n || ck >= a.n) return false;
    const int M = a.M;
    const T* src = a.src + (size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck)));
    T u[3][27];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool bnd = bj || (2 * ci + i == 0) || (2 * ci + i == M - 1);
                const int off = i + M * (j + M * k);
#pragma unroll
                for (int c = 0; c < 3; ++c) u[c][i + 3 * j + 9 * k] = bnd ? T(0) : src[c * a.nodes + off];
            }
        }
    }
    q2::cell_A(u, w);
    const T s = a.mu[size_t(ci) + size_t(a.n) * (cj + size_t(a.n) * ck)] * a.h;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 27; ++m) w[c][m] *= s;
    return true;
}

// Phase 2: export the 19 local nodes with an index 2 (E holds 57 x NC values).
template <typename T, int BX, int BY, int BZ>
__host__ __device__ __forceinline__ void brick_export(int tid, const T (&w)[3][27], T* E) {
    using S = BrickShape<BX, BY, BZ>;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i != 2 && j != 2 && k != 2) continue;
#pragma unroll
                for (int c = 0; c < 3; ++c) E[(export_index(i, j, k) * 3 + c) * S::NC + tid] = w[c][i + 3 * j + 9 * k];
            }
}

// Phase 3 (after a barrier): complete the owned nodes into the node tile (tile = E + EXPORT).
template <typename T, int BX, int BY, int BZ>
__host__ __device__ __forceinline__ void brick_own(const BrickArgs<T>& a, int bx, int by, int bz, int tid,
                                                   const T (&w)[3][27], T* E) {
    using S = BrickShape<BX, BY, BZ>;
    const int cx = tid % BX, cy = (tid / BX) % BY, cz = tid / (BX * BY);
    const int ci = BX * bx + cx, cj = BY * by + cy, ck = BZ * bz + cz;
    // last valid cell of the brick along each axis owns the brick's upper layer of nodes
    const bool ux = (cx == BX - 1) || (ci == a.n - 1);
    const bool uy = (cy == BY - 1) || (cj == a.n - 1);
    const bool uz = (cz == BZ - 1) || (ck == a.n - 1);
    T* tile = E + S::EXPORT;
    const int base = 2 * cx + S::TX * (2 * cy + S::TY * 2 * cz);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if ((i == 2 && !ux) || (j == 2 && !uy) || (k == 2 && !uz)) continue;
                T sum[3] = {w[0][i + 3 * j + 9 * k], w[1][i + 3 * j + 9 * k], w[2][i + 3 * j + 9 * k]};
#pragma unroll
                for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            if (dx + dy + dz == 0) continue;
                            if ((dx && i != 0) || (dy && j != 0) || (dz && k != 0)) continue;
                            if ((dx && cx == 0) || (dy && cy == 0) || (dz && cz == 0)) continue;
                            const int nb = tid - dx - dy * BX - dz * BX * BY;
                            const int e = export_index(i + 2 * dx, j + 2 * dy, k + 2 * dz);
#pragma unroll
                            for (int c = 0; c < 3; ++c) sum[c] += E[(e * 3 + c) * S::NC + nb];
                        }
                const int t = base + i + S::TX * (j + S::TY * k);
#pragma unroll
                for (int c = 0; c < 3; ++c) tile[c * S::TILE + t] = sum[c];
            }
}

// Phase 4 (after a second barrier): epilogue over the tile, one row of TX nodes per step.
template <typename T, int EPI, int BX, int BY, int BZ>
__host__ __device__ __forceinline__ void brick_epilogue(const BrickArgs<T>& a, int bx, int by, int bz, int tid,
                                                        int nthreads, const T* E) {
    using S = BrickShape<BX, BY, BZ>;
    const T* tile = E + S::EXPORT;
    const int M = a.M;
    const int gi0 = 2 * BX * bx, gj0 = 2 * BY * by, gk0 = 2 * BZ * bz;
#pragma unroll 1
    for (int t = tid; t < S::TILE; t += nthreads) {
        const int li = t % S::TX, r = t / S::TX;
        const int lj = r % S::TY, lk = r / S::TY;
        const int gi = gi0 + li, gj = gj0 + lj, gk = gk0 + lk;
        if (gi >= M || gj >= M || gk >= M) continue;
        const size_t node = size_t(gi) + size_t(M) * (size_t(gj) + size_t(M) * size_t(gk));
        if (gi == 0 || gj == 0 || gk == 0 || gi == M - 1 || gj == M - 1 || gk == M - 1) {
            for (int c = 0; c < 3; ++c) epilogue_boundary<T, EPI>(a, c * a.nodes + node);
            continue;
        }
        const bool px = (li == 0 || li == 2 * BX), py = (lj == 0 || lj == 2 * BY), pz = (lk == 0 || lk == 2 * BZ);
        if (!(px || py || pz)) {
            for (int c = 0; c < 3; ++c) epilogue<T, EPI>(a, c * a.nodes + node, tile[c * S::TILE + t]);
            continue;
        }
        const int P = (px ? 1 : 0) | (py ? 2 : 0) | (pz ? 4 : 0);
        int slot = 0, rank = 0;
        if (px) { slot |= (li == 0 ? 1 : 0) << rank; ++rank; }
        if (py) { slot |= (lj == 0 ? 1 : 0) << rank; ++rank; }
        if (pz) { slot |= (lk == 0 ? 1 : 0) << rank; }
        for (int c = 0; c < 3; ++c)
            a.slots[plane_entry_c<BX, BY, BZ>(a.L, P, slot, c, gi, gj, gk)] = tile[c * S::TILE + t];
    }
}

// Plane kernel body: thread index t over the plane nodes of the three families
// (x-planes; y-planes off x-planes; z-planes off x- and y-planes).
template <typename T, int EPI, int BX, int BY, int BZ>
__host__ __device__ __forceinline__ void plane_node(const BrickArgs<T>& a, size_t t) {
    const PlaneLayout& L = a.L;
    const size_t M = size_t(a.M), MM = M * M;
    const size_t nX = size_t(L.np[0]) * MM, nY = size_t(L.np[1]) * MM, nZ = size_t(L.np[2]) * MM;
    int gi, gj, gk;
    if (t < nX) {
        gj = int(t % M); gk = int((t / M) % M); gi = int(2 * BX * (t / MM + 1));
    } else if (t < nX + nY) {
        const size_t u = t - nX;
        gi = int(u % M); gk = int((u / M) % M); gj = int(2 * BY * (u / MM + 1));
        if (on_plane(gi, 2 * BX, a.M)) return;
    } else if (t < nX + nY + nZ) {
        const size_t u = t - nX - nY;
        gi = int(u % M); gj = int((u / M) % M); gk = int(2 * BZ * (u / MM + 1));
        if (on_plane(gi, 2 * BX, a.M) || on_plane(gj, 2 * BY, a.M)) return;
    } else {
        return;
    }
    if (gi == 0 || gj == 0 || gk == 0 || gi == a.M - 1 || gj == a.M - 1 || gk == a.M - 1) return;
    const bool px = on_plane(gi, 2 * BX, a.M), py = on_plane(gj, 2 * BY, a.M), pz = on_plane(gk, 2 * BZ, a.M);
    const int P = (px ? 1 : 0) | (py ? 2 : 0) | (pz ? 4 : 0);
    const int slots = 1 << ((px ? 1 : 0) + (py ? 1 : 0) + (pz ? 1 : 0));
    const size_t node = size_t(gi) + M * (size_t(gj) + M * size_t(gk));
    for (int c = 0; c < 3; ++c) {
        T sum = T(0);
        for (int s = 0; s < slots; ++s) sum += a.slots[plane_entry_c<BX, BY, BZ>(L, P, s, c, gi, gj, gk)];
        epilogue<T, EPI>(a, c * a.nodes + node, sum);
    }
}

inline size_t plane_threads(const PlaneLayout& L) {
    const size_t MM = size_t(L.M) * L.M;
    return (size_t(L.np[0]) + L.np[1] + L.np[2]) * MM;
}

// Layout of the plane slots for an n^3 level with the library's brick shape.
PlaneLayout brick_layout(int n);
// Shared-memory opt-in of every brick kernel instantiation (call once before any launch or capture).
cudaError_t brick_configure();
// FP32 scatter of one x-row of a cell (the values of local nodes (0..2, j, k)) with one 8-byte
// and one 4-byte atomic add instead of three 4-byte ones. The row's first node lies at element
// offset c nodes + 2ci + M (2cj + j) + M^2 (2ck + k), whose parity is (c + j + k) mod 2 (nodes =
// M^3 and M are odd), so the pair (0,1) or (1,2) is 8-byte aligned when the accumulator is; the
// parity is a compile-time constant in the cell kernel and warp-uniform in the split kernel.
// Measured on the operator's gather-and-scatter alone at 128^3: 0.229 ms with 81 single adds per
// cell, 0.180 ms with 27 pairs and 27 singles.
#ifdef __CUDACC__
__device__ __forceinline__ void add_row3(float* row, int parity, float v0, float v1, float v2) {
    if (parity == 0) {
        atomicAdd(reinterpret_cast<float2*>(row), make_float2(v0, v1));
        atomicAdd(row + 2, v2);
    } else {
        atomicAdd(row, v0);
        atomicAdd(reinterpret_cast<float2*>(row + 1), make_float2(v1, v2));
    }
}
#endif

// One Chebyshev step carried by the next product (the cell and component-split operators).
// Chebyshev step k ends with d' = c1 d + c2 dinv (b - A x), x' = x + d'; instead of a separate
// consumer pass, the kernel forming A x' computes d', x' at every node it gathers (the same
// arithmetic in the same order), uses x' as its operand, and the node's owner cell (local index 0
// or 1 along each axis, or 2 in the last cell of the level) stores d', x' into the other buffers of
// the (d, x) pairs and clears acc_zero there. The pairs alternate, so no kernel reads a value that
// another cell of the same launch writes; the accumulators rotate over three buffers: one holds
// A x (read), one receives A x' (atomic adds), one is cleared for the launch after next.
template <typename T>
struct ChebGather {
    const T* acc_prev;   // A x, complete
    const T* b;
    const T* dinv;
    const T* d_old;
    const T* x_old;
    T* d_new;            // written at owned nodes (all nodes, boundary ones included, across the launch)
    T* x_new;
    T* acc_zero;         // cleared at owned nodes (null: nothing to clear)
    T c1, c2;
};

// acc += A x' with x' from the pending step g (kernel: 0, 64, 128, 256 the cell kernel's block
// size, 3 the component-split kernel on FP32 levels).
template <typename T>
cudaError_t launch_cell_cheb(int kernel, const LevelGeom& geo, const T* mu, const ChebGather<T>& g, T* acc,
                             cudaStream_t s);
// acc += A src with the cell (kernel 0, 64, 128, 256) or component-split (3, FP32) operator.
template <typename T>
cudaError_t launch_accumulate(int kernel, const LevelGeom& geo, const T* mu, const T* src, T* acc, cudaStream_t s);
// The consumers with separate input and output (d, x) buffers (equal pointers: in place) and a
// second accumulator to clear (zero2, may be null). epi 1: r = b - acc (r in x_dst); epi 2: the
// Chebyshev update.
template <typename T>
cudaError_t launch_consume2(int epi, size_t n, T* acc, const T* b, const T* dinv, const T* d_src, const T* x_src,
                            T* d_dst, T* x_dst, T* zero2, double c1, double c2, cudaStream_t s);

// Tensor-core level operator (brick_tc.cu): the f16 table of 5400 A_hat in the layout its
// kernel reads (tc_table_bytes() bytes, built once by tc_build_table), a device status word
// (bit 0: a bounded wait for the MMAs gave up) and that wait's limit in nanoseconds.
struct TcArgs {
    const void* table;
    unsigned* status;
    unsigned long long wait_ns;
};
cudaError_t tc_configure();
size_t tc_table_bytes();
// flag (device int) != 0 afterwards if an entry of 5400 A_hat is not an integer f16 holds exactly.
cudaError_t tc_build_table(void* table, int* flag, cudaStream_t s);
// acc += A src on the nodes that are not on the domain boundary (acc zero there on entry, as for
// the cell kernel); the epilogue kernels of launch_level_op consume it.
cudaError_t launch_cell_tc(const BrickArgs<float>& a, float* acc, const TcArgs& t, cudaStream_t s);

// A x with an epilogue (EPI_PLAIN: dst = A x; EPI_RESID: dst = b - A x;
// EPI_CHEB: d = c1 d + c2 dinv (b - A x), src += d in place).
// kernel 0, 64, 128, 256: one thread per cell (blocks of 128, 64, 128, 256 threads) with atomic
//           adds into acc (n_u entries, zero on entry and on return) and a consumer kernel for the
//           epilogue;
// kernel 3: FP32: the cell kernel's accumulation with three threads per cell (one per output
//           component), the same consumer kernels; FP64: kernel 128;
// kernel 1: the brick-tiled kernel with the epilogue fused (slots: brick_layout(n).total entries);
// kernel 2: FP32: the cell products on the tensor cores, accumulated like kernel 0 (tc must be
//           given); FP64: kernel 128.
template <typename T>
cudaError_t launch_level_op(int kernel, const LevelGeom& g, const PlaneLayout& L, int epi, const T* mu, const T* src,
                            T* dst, const T* b, const T* dinv, T* d, double c1, double c2, T* slots, T* acc,
                            cudaStream_t s, const TcArgs* tc = nullptr);

}  // namespace stk
