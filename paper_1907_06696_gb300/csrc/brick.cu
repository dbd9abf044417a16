// brick.cu -- launchers of the brick-tiled velocity operator (brick.cuh).
#include "brick.cuh"
#include "prof.cuh"

#include <cstdint>

#define LAUNCH(cls, s, ...)              \
    do {                                \
        prof_begin((cls), (s));         \
        __VA_ARGS__;                    \
        prof_end((cls), (s));           \
        prof_count(1);                  \
    } while (0)

namespace stk {

namespace {

template <typename T, int EPI, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ, sizeof(T) == 4 ? 3 : 1) k_brick(BrickArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    {
        T w[3][27];
        const bool valid = brick_compute<T, BX, BY, BZ>(a, bx, by, bz, threadIdx.x, w);
        if (valid) brick_export<T, BX, BY, BZ>(threadIdx.x, w, sm);
        __syncthreads();
        if (valid) brick_own<T, BX, BY, BZ>(a, bx, by, bz, threadIdx.x, w, sm);
    }
    __syncthreads();
    brick_epilogue<T, EPI, BX, BY, BZ>(a, bx, by, bz, threadIdx.x, blockDim.x, sm);
}

// ---- cell-parallel variant: one thread per cell, atomic adds into a zeroed accumulator;
// the consumer kernels below run the epilogue and clear the accumulator again.
// Threads per block BS: 64, 128 or 256 (the register budget per thread is the same, 170 for FP32).
// Scatter of a cell's scaled output w into acc (boundary nodes untouched: rows on the boundary
// are skipped, boundary nodes inside a row get 0 added, so acc stays 0 there).
template <typename T, bool PAIRS>
__device__ __forceinline__ void scatter_cell(T* out, size_t nodes, int M, int ci, int cj, int ck, const T (&w)[3][27]) {
    if constexpr (PAIRS && sizeof(T) == 4) {
        const bool b0 = ci == 0, b2 = 2 * ci + 2 == M - 1;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (bk || (2 * cj + j == 0) || (2 * cj + j == M - 1)) continue;
                const int off = M * (j + M * k);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    add_row3(out + c * nodes + off, (c + j + k) & 1, b0 ? 0.0f : w[c][3 * j + 9 * k],
                             w[c][1 + 3 * j + 9 * k], b2 ? 0.0f : w[c][2 + 3 * j + 9 * k]);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (bj || (2 * ci + i == 0) || (2 * ci + i == M - 1)) continue;
                    const int off = i + M * (j + M * k);
#pragma unroll
                    for (int c = 0; c < 3; ++c) atomicAdd(out + c * nodes + off, w[c][i + 3 * j + 9 * k]);
                }
            }
        }
    }
}

template <typename T, int BS, bool PAIRS>
__global__ void __launch_bounds__(BS, sizeof(T) == 4 ? 384 / BS : 1) k_cell_atomic(BrickArgs<T> a, T* acc) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= size_t(a.n) * a.n * a.n) return;
    const int ci = int(cell % a.n), cj = int((cell / a.n) % a.n), ck = int(cell / (size_t(a.n) * a.n));
    T w[3][27];
    // brick_compute with a 1x1x1 brick at (ci, cj, ck)
    if (!brick_compute<T, 1, 1, 1>(a, ci, cj, ck, 0, w)) return;
    const int M = a.M;
    T* out = acc + (size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck)));
    scatter_cell<T, PAIRS>(out, a.nodes, M, ci, cj, ck, w);
}

// ---- component-split variant: three threads per cell, warp c of each group of three computes
// output component c. A cell's output row c is
//   w_c = 2 D_c^T W (d_c U_c) + sum_{d != c} D_d^T W (d_d U_c + d_c U_d),
// so the thread of component c interpolates only its own component U_c, forms its three
// derivatives d_e U_c, and takes the cross terms d_c U_d from the other two threads through
// shared memory. The arithmetic per cell is that of the one-thread kernel (the same sweeps), the
// serial work per thread a third of it: the small levels, where a level operator is one wave of
// a few warps and its time is one thread's latency, get faster; the product is the same up to
// the order of the sums.
constexpr int kSplitCells = 32;   // cells per block; block = 3 warps

// The cell product of the component-split kernels: u holds the nodal values of this thread's
// component on entry and the cell's output row c (without mu h) on return; all threads of the
// block take part (the exchange has a barrier).
__device__ __forceinline__ void split_apply(float (&u)[27], float (&D)[3][3][27][kSplitCells], int c, int lc) {
    q2::interp<0>(u);
    q2::interp<1>(u);
    q2::interp<2>(u);
    float g[27];
    q2::deriv<0, false>(u, g);
#pragma unroll
    for (int q = 0; q < 27; ++q) D[c][0][q][lc] = g[q];
    q2::deriv<1, false>(u, g);
#pragma unroll
    for (int q = 0; q < 27; ++q) D[c][1][q][lc] = g[q];
    q2::deriv<2, false>(u, g);
#pragma unroll
    for (int q = 0; q < 27; ++q) D[c][2][q][lc] = g[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 27; ++q) u[q] = 0.0f;
    // d = 0, 1, 2 at compile time; the diagonal term (d == c) carries the factor 2
#pragma unroll
    for (int q = 0; q < 27; ++q) g[q] = c == 0 ? D[0][0][q][lc] : D[c][0][q][lc] + D[0][c][q][lc];
    if (c == 0) q2::derivT_w<0, 2>(g, u); else q2::derivT_w<0, 1>(g, u);
#pragma unroll
    for (int q = 0; q < 27; ++q) g[q] = c == 1 ? D[1][1][q][lc] : D[c][1][q][lc] + D[1][c][q][lc];
    if (c == 1) q2::derivT_w<1, 2>(g, u); else q2::derivT_w<1, 1>(g, u);
#pragma unroll
    for (int q = 0; q < 27; ++q) g[q] = c == 2 ? D[2][2][q][lc] : D[c][2][q][lc] + D[2][c][q][lc];
    if (c == 2) q2::derivT_w<2, 2>(g, u); else q2::derivT_w<2, 1>(g, u);
    q2::interpT<0>(u);
    q2::interpT<1>(u);
    q2::interpT<2>(u);
}

// Scatter of component c of a cell's output row (times sc) into acc at out = acc + c nodes +
// the cell's first node; with PAIRS the rows go as pairs (parity (c + j + k) mod 2, uniform over
// the warp of component c).
template <bool PAIRS>
__device__ __forceinline__ void split_scatter(float* out, int c, int M, int ci, int cj, int ck, float sc,
                                              const float (&u)[27]) {
    const bool b0 = ci == 0, b2 = 2 * ci + 2 == M - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (bk || (2 * cj + j == 0) || (2 * cj + j == M - 1)) continue;
            float* row = out + M * (j + M * k);
            if (PAIRS) {
                add_row3(row, (c + j + k) & 1, b0 ? 0.0f : u[3 * j + 9 * k] * sc, u[1 + 3 * j + 9 * k] * sc,
                         b2 ? 0.0f : u[2 + 3 * j + 9 * k] * sc);
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if ((i == 0 && b0) || (i == 2 && b2)) continue;
                    atomicAdd(row + i, u[i + 3 * j + 9 * k] * sc);
                }
            }
        }
    }
}

template <bool PAIRS>
__global__ void __launch_bounds__(3 * kSplitCells) k_cell_split(BrickArgs<float> a, float* acc) {
    __shared__ float D[3][3][27][kSplitCells];   // D[c][e][q][cell] = d_e U_c at Gauss point q
    const int c = threadIdx.x / kSplitCells;     // warp-uniform
    const int lc = threadIdx.x % kSplitCells;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const size_t cell = size_t(blockIdx.x) * kSplitCells + lc;
    const bool valid = cell < cells;
    const int ci = valid ? int(cell % a.n) : 0;
    const int cj = valid ? int((cell / a.n) % a.n) : 0;
    const int ck = valid ? int(cell / (size_t(a.n) * a.n)) : 0;
    const int M = a.M;
    const size_t base = size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck));
    const float* src = a.src + size_t(c) * a.nodes + base;
    float u[27];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool bnd = !valid || bj || (2 * ci + i == 0) || (2 * ci + i == M - 1);
                u[i + 3 * j + 9 * k] = bnd ? 0.0f : src[i + M * (j + M * k)];
            }
        }
    }
    split_apply(u, D, c, lc);
    if (!valid) return;
    split_scatter<PAIRS>(acc + size_t(c) * a.nodes + base, c, M, ci, cj, ck, a.mu[cell] * a.h, u);
}

// ---- the two operators with the pending Chebyshev step applied at the gather (ChebGather)
// The step's buffers are passed as separate restrict-qualified parameters: the owners' stores
// cannot alias the gathered loads, so the loads of all 27 nodes may be issued before any store
// (through the struct the compiler has to keep each node's loads behind the previous node's
// stores, one memory latency per node).
template <typename T>
__device__ __forceinline__ T cheb_node(const T* __restrict__ acc_prev, const T* __restrict__ b,
                                       const T* __restrict__ dinv, const T* __restrict__ d_old,
                                       const T* __restrict__ x_old, T* __restrict__ d_new, T* __restrict__ x_new,
                                       T* __restrict__ acc_zero, T c1, T c2, size_t i, bool own) {
    const T dn = (c1 != T(0) ? c1 * d_old[i] : T(0)) + c2 * (dinv[i] * (b[i] - acc_prev[i]));
    const T xn = x_old[i] + dn;
    if (own) {
        d_new[i] = dn;
        x_new[i] = xn;
        if (acc_zero) acc_zero[i] = T(0);
    }
    return xn;
}

template <typename T, int BS>
__global__ void __launch_bounds__(BS, sizeof(T) == 4 ? 384 / BS : 1)
    k_cell_cheb(BrickArgs<T> a, const T* __restrict__ acc_prev, const T* __restrict__ b, const T* __restrict__ dinv,
                const T* __restrict__ d_old, const T* __restrict__ x_old, T* __restrict__ d_new,
                T* __restrict__ x_new, T* __restrict__ acc_zero, T c1, T c2, T* __restrict__ acc) {
    const size_t cell = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= size_t(a.n) * a.n * a.n) return;
    const int ci = int(cell % a.n), cj = int((cell / a.n) % a.n), ck = int(cell / (size_t(a.n) * a.n));
    const int M = a.M;
    const size_t base = size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck));
    T u[3][27], w[3][27];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
        const bool ok = k < 2 || ck == a.n - 1;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
            const bool oj = ok && (j < 2 || cj == a.n - 1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool bnd = bj || (2 * ci + i == 0) || (2 * ci + i == M - 1);
                const bool own = oj && (i < 2 || ci == a.n - 1);
                const size_t off = base + size_t(i + M * (j + M * k));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T xn = cheb_node(acc_prev, b, dinv, d_old, x_old, d_new, x_new, acc_zero, c1, c2,
                                           size_t(c) * a.nodes + off, own);
                    u[c][i + 3 * j + 9 * k] = bnd ? T(0) : xn;
                }
            }
        }
    }
    q2::cell_A(u, w);
    const T sc = a.mu[cell] * a.h;
    T* out = acc + base;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (bj || (2 * ci + i == 0) || (2 * ci + i == M - 1)) continue;
                const int off = i + M * (j + M * k);
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(out + c * a.nodes + off, w[c][i + 3 * j + 9 * k] * sc);
            }
        }
    }
}

template <bool PAIRS>
__global__ void __launch_bounds__(3 * kSplitCells)
    k_cell_split_cheb(BrickArgs<float> a, const float* __restrict__ acc_prev, const float* __restrict__ b,
                      const float* __restrict__ dinv, const float* __restrict__ d_old, const float* __restrict__ x_old,
                      float* __restrict__ d_new, float* __restrict__ x_new, float* __restrict__ acc_zero, float c1,
                      float c2, float* __restrict__ acc) {
    __shared__ float D[3][3][27][kSplitCells];
    const int c = threadIdx.x / kSplitCells;
    const int lc = threadIdx.x % kSplitCells;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const size_t cell = size_t(blockIdx.x) * kSplitCells + lc;
    const bool valid = cell < cells;
    const int ci = valid ? int(cell % a.n) : 0;
    const int cj = valid ? int((cell / a.n) % a.n) : 0;
    const int ck = valid ? int(cell / (size_t(a.n) * a.n)) : 0;
    const int M = a.M;
    const size_t base = size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck));
    const size_t cbase = size_t(c) * a.nodes + base;
    float u[27];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
        const bool ok = k < 2 || ck == a.n - 1;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
            const bool oj = ok && (j < 2 || cj == a.n - 1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool bnd = bj || (2 * ci + i == 0) || (2 * ci + i == M - 1);
                const bool own = oj && (i < 2 || ci == a.n - 1);
                float xn = 0.0f;
                if (valid)
                    xn = cheb_node(acc_prev, b, dinv, d_old, x_old, d_new, x_new, acc_zero, c1, c2,
                                   cbase + size_t(i + M * (j + M * k)), own);
                u[i + 3 * j + 9 * k] = (!valid || bnd) ? 0.0f : xn;
            }
        }
    }
    split_apply(u, D, c, lc);
    if (!valid) return;
    split_scatter<PAIRS>(acc + cbase, c, M, ci, cj, ck, a.mu[cell] * a.h, u);
}

// Consume the accumulated product and clear it. Constrained entries need no special
// case: acc, b, dinv and d are 0 there. 128-bit accesses on the aligned bulk, scalar tail.
// Each thread loads two 128-bit items of every operand before it stores anything, and clears
// acc after its data-dependent stores: clearing acc first (right behind its load) measured
// 2.8 TB/s for the Chebyshev consumer and 1.4 TB/s for the residual one at 128^3, against
// 6.9 and 6.7 TB/s in this order.
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double2; };

__device__ __forceinline__ float4 vzero(float4) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 vzero(double2) { return make_double2(0.0, 0.0); }

constexpr int kConsumeItems = 2;   // 128-bit items per thread and iteration

inline unsigned consume_blocks(size_t n, size_t per) {
    const size_t nb = (n / per + 256 * kConsumeItems - 1) / (256 * kConsumeItems);
    return unsigned(nb < 1 ? 1 : (nb < 4864 ? nb : 4864));
}

// d_dst = c1 d_src + c2 dinv (b - acc); x_dst = x_src + d_dst; acc = 0 (and zero2 = 0 when given).
// The (d, x) outputs may be the inputs (in place): each entry is read before it is written.
template <typename T>
__global__ void __launch_bounds__(256) k_consume_cheb(size_t n, T* __restrict__ acc, const T* __restrict__ b,
                                                     const T* __restrict__ dinv, const T* d_src, const T* x_src,
                                                     T* d, T* x, T* __restrict__ zero2, T c1, T c2, bool vec) {
    using V = typename Vec4<T>::type;
    constexpr int W = sizeof(V) / sizeof(T);
    constexpr int U = kConsumeItems;
    const size_t nv = vec ? n / W : 0;
    const size_t stride = size_t(gridDim.x) * blockDim.x * U;
    for (size_t v0 = size_t(blockIdx.x) * blockDim.x * U + threadIdx.x; v0 < nv; v0 += stride) {
        V A[U], B[U], Di[U], Dd[U], X[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t v = v0 + size_t(u) * blockDim.x;
            if (v < nv) {
                A[u] = reinterpret_cast<const V*>(acc)[v];
                B[u] = reinterpret_cast<const V*>(b)[v];
                Di[u] = reinterpret_cast<const V*>(dinv)[v];
                Dd[u] = reinterpret_cast<const V*>(d_src)[v];
                X[u] = reinterpret_cast<const V*>(x_src)[v];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t v = v0 + size_t(u) * blockDim.x;
            if (v >= nv) continue;
            const T* a_ = reinterpret_cast<const T*>(&A[u]);
            const T* b_ = reinterpret_cast<const T*>(&B[u]);
            const T* di_ = reinterpret_cast<const T*>(&Di[u]);
            T* d_ = reinterpret_cast<T*>(&Dd[u]);
            T* x_ = reinterpret_cast<T*>(&X[u]);
#pragma unroll
            for (int q = 0; q < W; ++q) {
                const T dn = (c1 != T(0) ? c1 * d_[q] : T(0)) + c2 * (di_[q] * (b_[q] - a_[q]));
                d_[q] = dn;
                x_[q] += dn;
            }
            reinterpret_cast<V*>(d)[v] = Dd[u];
            reinterpret_cast<V*>(x)[v] = X[u];
            reinterpret_cast<V*>(acc)[v] = vzero(A[u]);
            if (zero2) reinterpret_cast<V*>(zero2)[v] = vzero(A[u]);
        }
    }
    const size_t tail_stride = size_t(gridDim.x) * blockDim.x;
    for (size_t i = nv * W + size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += tail_stride) {
        const T dn = (c1 != T(0) ? c1 * d_src[i] : T(0)) + c2 * (dinv[i] * (b[i] - acc[i]));
        const T xn = x_src[i] + dn;
        d[i] = dn;
        x[i] = xn;
        acc[i] = T(0);
        if (zero2) zero2[i] = T(0);
    }
}

// r = b - acc; acc = 0 (and zero2 = 0 when given)
template <typename T>
__global__ void __launch_bounds__(256) k_consume_resid(size_t n, T* __restrict__ acc, const T* __restrict__ b,
                                                      T* __restrict__ r, T* __restrict__ zero2, bool vec) {
    using V = typename Vec4<T>::type;
    constexpr int W = sizeof(V) / sizeof(T);
    constexpr int U = kConsumeItems;
    const size_t nv = vec ? n / W : 0;
    const size_t stride = size_t(gridDim.x) * blockDim.x * U;
    for (size_t v0 = size_t(blockIdx.x) * blockDim.x * U + threadIdx.x; v0 < nv; v0 += stride) {
        V A[U], B[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t v = v0 + size_t(u) * blockDim.x;
            if (v < nv) {
                A[u] = reinterpret_cast<const V*>(acc)[v];
                B[u] = reinterpret_cast<const V*>(b)[v];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t v = v0 + size_t(u) * blockDim.x;
            if (v >= nv) continue;
            V R;
            const T* a_ = reinterpret_cast<const T*>(&A[u]);
            const T* b_ = reinterpret_cast<const T*>(&B[u]);
            T* r_ = reinterpret_cast<T*>(&R);
#pragma unroll
            for (int q = 0; q < W; ++q) r_[q] = b_[q] - a_[q];
            reinterpret_cast<V*>(r)[v] = R;
            reinterpret_cast<V*>(acc)[v] = vzero(A[u]);
            if (zero2) reinterpret_cast<V*>(zero2)[v] = vzero(A[u]);
        }
    }
    const size_t tail_stride = size_t(gridDim.x) * blockDim.x;
    for (size_t i = nv * W + size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += tail_stride) {
        r[i] = b[i] - acc[i];
        acc[i] = T(0);
        if (zero2) zero2[i] = T(0);
    }
}

template <typename T, int EPI>
__global__ void k_planes(BrickArgs<T> a, size_t total) {
    const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < total) plane_node<T, EPI, kBrickX, kBrickY, kBrickZ>(a, t);
}

template <typename T, int EPI>
cudaError_t configure_epi() {
    using S = BrickShape<kBrickX, kBrickY, kBrickZ>;
    return cudaFuncSetAttribute(k_brick<T, EPI, kBrickX, kBrickY, kBrickZ>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::template smem_bytes<T>()));
}

template <typename T, int EPI>
cudaError_t launch_epi(const BrickArgs<T>& a, cudaStream_t s) {
    using S = BrickShape<kBrickX, kBrickY, kBrickZ>;
    constexpr size_t smem = S::template smem_bytes<T>();
    const dim3 grid(unsigned((a.n + kBrickX - 1) / kBrickX), unsigned((a.n + kBrickY - 1) / kBrickY),
                    unsigned((a.n + kBrickZ - 1) / kBrickZ));
    const int cls = sizeof(T) == 4 ? PROF_VMULT_F32 : PROF_VMULT_F64;
    LAUNCH(cls, s, (k_brick<T, EPI, kBrickX, kBrickY, kBrickZ><<<grid, S::NC, smem, s>>>(a)));
    const size_t total = plane_threads(a.L);
    if (total > 0) LAUNCH(PROF_SMOOTH_VEC, s, (k_planes<T, EPI><<<unsigned((total + 255) / 256), 256, 0, s>>>(a, total)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cell(const BrickArgs<T>& a, T* acc, int bs, cudaStream_t s) {
    const size_t cells = size_t(a.n) * a.n * a.n;
    const int cls = sizeof(T) == 4 ? PROF_VMULT_F32 : PROF_VMULT_F64;
    // pair atomics need an 8-byte aligned accumulator (callers may pass offset views)
    const bool pairs = (reinterpret_cast<uintptr_t>(acc) & 7u) == 0;
    if (bs == 64) {
        if (pairs) LAUNCH(cls, s, (k_cell_atomic<T, 64, true><<<unsigned((cells + 63) / 64), 64, 0, s>>>(a, acc)));
        else LAUNCH(cls, s, (k_cell_atomic<T, 64, false><<<unsigned((cells + 63) / 64), 64, 0, s>>>(a, acc)));
    } else if (bs == 256) {
        if (pairs) LAUNCH(cls, s, (k_cell_atomic<T, 256, true><<<unsigned((cells + 255) / 256), 256, 0, s>>>(a, acc)));
        else LAUNCH(cls, s, (k_cell_atomic<T, 256, false><<<unsigned((cells + 255) / 256), 256, 0, s>>>(a, acc)));
    } else {
        if (pairs) LAUNCH(cls, s, (k_cell_atomic<T, 128, true><<<unsigned((cells + 127) / 128), 128, 0, s>>>(a, acc)));
        else LAUNCH(cls, s, (k_cell_atomic<T, 128, false><<<unsigned((cells + 127) / 128), 128, 0, s>>>(a, acc)));
    }
    return cudaGetLastError();
}

// Accumulate A src into acc: the cell kernel with bs threads per block, or for FP32 levels the
// component-split kernel (bs = kSplitKernel) or (tc given) the tensor-core kernel.
constexpr int kSplitKernel = 3;

template <typename T>
cudaError_t accumulate(const BrickArgs<T>& a, T* acc, int bs, const TcArgs* tc, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (tc) return launch_cell_tc(a, acc, *tc, s);
        if (bs == kSplitKernel) {
            const size_t cells = size_t(a.n) * a.n * a.n;
            const unsigned blocks = unsigned((cells + kSplitCells - 1) / kSplitCells);
            if ((reinterpret_cast<uintptr_t>(acc) & 7u) == 0)
                LAUNCH(PROF_VMULT_F32, s, (k_cell_split<true><<<blocks, 3 * kSplitCells, 0, s>>>(a, acc)));
            else
                LAUNCH(PROF_VMULT_F32, s, (k_cell_split<false><<<blocks, 3 * kSplitCells, 0, s>>>(a, acc)));
            return cudaGetLastError();
        }
    }
    return launch_cell<T>(a, acc, bs == kSplitKernel ? 128 : bs, s);
}

template <typename T>
cudaError_t launch_cell_epi(const BrickArgs<T>& a, int epi, T* acc, size_t n_u, int bs, cudaStream_t s,
                            const TcArgs* tc = nullptr) {
    if (epi == EPI_PLAIN) {
        // dst = A src: accumulate straight into the zeroed dst, identity rows afterwards
        cudaError_t e = cudaMemsetAsync(a.dst, 0, n_u * sizeof(T), s);
        if (e != cudaSuccess) return e;
        e = accumulate<T>(a, a.dst, bs, tc, s);
        if (e != cudaSuccess) return e;
        LevelGeom g = make_geom(a.n);
        return launch_copy_boundary<T>(g, a.src, a.dst, s);
    }
    cudaError_t e = accumulate<T>(a, acc, bs, tc, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = consume_blocks(n_u, sizeof(T) == 4 ? 4 : 2);
    // 128-bit accesses only when every operand is 16-byte aligned (callers may pass offset views)
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (epi == EPI_RESID) {
        const bool vec = al(acc) && al(a.b) && al(a.dst);
        LAUNCH(PROF_SMOOTH_VEC, s, (k_consume_resid<T><<<blocks, 256, 0, s>>>(n_u, acc, a.b, a.dst, nullptr, vec)));
    } else {
        const bool vec = al(acc) && al(a.b) && al(a.dinv) && al(a.d) && al(a.src);
        LAUNCH(PROF_SMOOTH_VEC, s, (k_consume_cheb<T><<<blocks, 256, 0, s>>>(n_u, acc, a.b, a.dinv, a.d, a.src, a.d,
                                                                            const_cast<T*>(a.src), nullptr, a.c1,
                                                                            a.c2, vec)));
    }
    return cudaGetLastError();
}

}  // namespace

PlaneLayout brick_layout(int n) { return make_plane_layout(n, kBrickX, kBrickY, kBrickZ); }

template <typename T>
cudaError_t launch_consume(int epi, size_t n, T* acc, const T* b, const T* dinv, T* d, T* x_or_r, double c1,
                           double c2, cudaStream_t s) {
    const unsigned blocks = consume_blocks(n, sizeof(T) == 4 ? 4 : 2);
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (epi == EPI_RESID) {
        const bool vec = al(acc) && al(b) && al(x_or_r);
        LAUNCH(PROF_SMOOTH_VEC, s, (k_consume_resid<T><<<blocks, 256, 0, s>>>(n, acc, b, x_or_r, nullptr, vec)));
    } else {
        const bool vec = al(acc) && al(b) && al(dinv) && al(d) && al(x_or_r);
        LAUNCH(PROF_SMOOTH_VEC, s, (k_consume_cheb<T><<<blocks, 256, 0, s>>>(n, acc, b, dinv, d, x_or_r, d, x_or_r,
                                                                            nullptr, T(c1), T(c2), vec)));
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cell_cheb(int kernel, const LevelGeom& geo, const T* mu, const ChebGather<T>& g, T* acc,
                             cudaStream_t s) {
    BrickArgs<T> a{};
    a.n = geo.n;
    a.M = geo.M;
    a.nodes = geo.nodes;
    a.h = T(geo.h);
    a.mu = mu;
    const size_t cells = size_t(a.n) * a.n * a.n;
    const int cls = sizeof(T) == 4 ? PROF_VMULT_F32 : PROF_VMULT_F64;
    if constexpr (sizeof(T) == 4) {
        if (kernel == kSplitKernel) {
            const unsigned blocks = unsigned((cells + kSplitCells - 1) / kSplitCells);
            if ((reinterpret_cast<uintptr_t>(acc) & 7u) == 0)
                LAUNCH(cls, s, (k_cell_split_cheb<true><<<blocks, 3 * kSplitCells, 0, s>>>(
                                   a, g.acc_prev, g.b, g.dinv, g.d_old, g.x_old, g.d_new, g.x_new, g.acc_zero, g.c1,
                                   g.c2, acc)));
            else
                LAUNCH(cls, s, (k_cell_split_cheb<false><<<blocks, 3 * kSplitCells, 0, s>>>(
                                   a, g.acc_prev, g.b, g.dinv, g.d_old, g.x_old, g.d_new, g.x_new, g.acc_zero, g.c1,
                                   g.c2, acc)));
            return cudaGetLastError();
        }
    }
#define STK_CHEB_ARGS a, g.acc_prev, g.b, g.dinv, g.d_old, g.x_old, g.d_new, g.x_new, g.acc_zero, g.c1, g.c2, acc
    if (kernel == 64)
        LAUNCH(cls, s, (k_cell_cheb<T, 64><<<unsigned((cells + 63) / 64), 64, 0, s>>>(STK_CHEB_ARGS)));
    else if (kernel == 256)
        LAUNCH(cls, s, (k_cell_cheb<T, 256><<<unsigned((cells + 255) / 256), 256, 0, s>>>(STK_CHEB_ARGS)));
    else
        LAUNCH(cls, s, (k_cell_cheb<T, 128><<<unsigned((cells + 127) / 128), 128, 0, s>>>(STK_CHEB_ARGS)));
#undef STK_CHEB_ARGS
    return cudaGetLastError();
}
template cudaError_t launch_cell_cheb<float>(int, const LevelGeom&, const float*, const ChebGather<float>&, float*,
                                             cudaStream_t);
template cudaError_t launch_cell_cheb<double>(int, const LevelGeom&, const double*, const ChebGather<double>&, double*,
                                              cudaStream_t);

template <typename T>
cudaError_t launch_accumulate(int kernel, const LevelGeom& geo, const T* mu, const T* src, T* acc, cudaStream_t s) {
    BrickArgs<T> a{};
    a.n = geo.n;
    a.M = geo.M;
    a.nodes = geo.nodes;
    a.h = T(geo.h);
    a.mu = mu;
    a.src = src;
    return accumulate<T>(a, acc, kernel == 0 ? 128 : kernel, nullptr, s);
}
template cudaError_t launch_accumulate<float>(int, const LevelGeom&, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_accumulate<double>(int, const LevelGeom&, const double*, const double*, double*,
                                               cudaStream_t);

template <typename T>
cudaError_t launch_consume2(int epi, size_t n, T* acc, const T* b, const T* dinv, const T* d_src, const T* x_src,
                            T* d_dst, T* x_dst, T* zero2, double c1, double c2, cudaStream_t s) {
    const unsigned blocks = consume_blocks(n, sizeof(T) == 4 ? 4 : 2);
    auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (epi == EPI_RESID) {
        const bool vec = al(acc) && al(b) && al(x_dst) && al(zero2);
        LAUNCH(PROF_SMOOTH_VEC, s, (k_consume_resid<T><<<blocks, 256, 0, s>>>(n, acc, b, x_dst, zero2, vec)));
    } else {
        const bool vec = al(acc) && al(b) && al(dinv) && al(d_src) && al(x_src) && al(d_dst) && al(x_dst) && al(zero2);
        LAUNCH(PROF_SMOOTH_VEC, s, (k_consume_cheb<T><<<blocks, 256, 0, s>>>(n, acc, b, dinv, d_src, x_src, d_dst, x_dst,
                                                                            zero2, T(c1), T(c2), vec)));
    }
    return cudaGetLastError();
}
template cudaError_t launch_consume2<float>(int, size_t, float*, const float*, const float*, const float*, const float*,
                                            float*, float*, float*, double, double, cudaStream_t);
template cudaError_t launch_consume2<double>(int, size_t, double*, const double*, const double*, const double*,
                                             const double*, double*, double*, double*, double, double, cudaStream_t);
template cudaError_t launch_consume<float>(int, size_t, float*, const float*, const float*, float*, float*, double,
                                           double, cudaStream_t);
template cudaError_t launch_consume<double>(int, size_t, double*, const double*, const double*, double*, double*,
                                            double, double, cudaStream_t);

cudaError_t brick_configure() {
    cudaError_t e;
    if ((e = configure_epi<float, EPI_PLAIN>()) != cudaSuccess) return e;
    if ((e = configure_epi<float, EPI_RESID>()) != cudaSuccess) return e;
    if ((e = configure_epi<float, EPI_CHEB>()) != cudaSuccess) return e;
    if ((e = configure_epi<double, EPI_PLAIN>()) != cudaSuccess) return e;
    if ((e = configure_epi<double, EPI_RESID>()) != cudaSuccess) return e;
    return configure_epi<double, EPI_CHEB>();
}

template <typename T>
cudaError_t launch_level_op(int kernel, const LevelGeom& g, const PlaneLayout& L, int epi, const T* mu, const T* src,
                            T* dst, const T* b, const T* dinv, T* d, double c1, double c2, T* slots, T* acc,
                            cudaStream_t s, const TcArgs* tc) {
    BrickArgs<T> a;
    a.n = g.n;
    a.M = g.M;
    a.nodes = g.nodes;
    a.h = T(g.h);
    a.mu = mu;
    a.src = src;
    a.dst = dst;
    a.b = b;
    a.dinv = dinv;
    a.d = d;
    a.c1 = T(c1);
    a.c2 = T(c2);
    a.slots = slots;
    a.L = L;
    if (kernel == 2) {
        if constexpr (sizeof(T) == 4) {
            if (!tc || !tc->table || !tc->status) return cudaErrorInvalidValue;
            return launch_cell_epi<T>(a, epi, acc, g.n_u, 128, s, tc);
        } else {
            kernel = 128;   // no FP64 tensor-core path
        }
    }
    if (kernel == 0 || kernel == kSplitKernel || kernel == 64 || kernel == 128 || kernel == 256)
        return launch_cell_epi<T>(a, epi, acc, g.n_u, kernel == 0 ? 128 : kernel, s);
    switch (epi) {
        case EPI_PLAIN: return launch_epi<T, EPI_PLAIN>(a, s);
        case EPI_RESID: return launch_epi<T, EPI_RESID>(a, s);
        case EPI_CHEB: return launch_epi<T, EPI_CHEB>(a, s);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_level_op<float>(int, const LevelGeom&, const PlaneLayout&, int, const float*,
                                            const float*, float*, const float*, const float*, float*, double, double,
                                            float*, float*, cudaStream_t, const TcArgs*);
template cudaError_t launch_level_op<double>(int, const LevelGeom&, const PlaneLayout&, int, const double*,
                                             const double*, double*, const double*, const double*, double*, double,
                                             double, double*, double*, cudaStream_t, const TcArgs*);

}  // namespace stk
