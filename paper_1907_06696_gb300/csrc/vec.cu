// vec.cu -- level transfers, Chebyshev updates, coarse solve and the FP64
// vector kernels of the Krylov solver.
//
// Transfers (Section 2.2.1; level data of Section 2.3): prolongation is the
// Q2 embedding of a coarse field into the fine space. Along one axis, fine
// node i_f of a fine level with 2 nc cells takes the coarse value at i_f/2
// when i_f is even; when odd it sits at 1/4 or 3/4 of coarse cell m = i_f/4
// and takes l_0, l_1, l_2 of the coarse cell at that point:
// (3/8, 3/4, -1/8) at 1/4 and (-1/8, 3/4, 3/8) at 3/4. The 3D weights are the
// products over the axes. Restriction is the exact transpose. Both run per
// coarse cell as three 1D sweeps (k_prolong_cells, k_restrict_cells); the
// per-node forms of transfer.cuh serve the batched V-cycle and the deterministic
// restriction of the brick-operator V-cycle.
#include "internal.cuh"
#include "prof.cuh"
#include "transfer.cuh"

#define LAUNCH(cls, s, ...)              \
    do {                                \
        prof_begin((cls), (s));         \
        __VA_ARGS__;                    \
        prof_end((cls), (s));           \
        prof_count(1);                  \
    } while (0)

namespace stk {

namespace {

inline unsigned blocks_for(size_t n, int t) { return unsigned((n + t - 1) / t); }


// Restriction as a gather per coarse node (no atomics, the same sums in the same order on every
// run): the form of the deterministic brick-operator V-cycle.
template <typename T>
__global__ void k_restrict_nodes(int nf, const T* __restrict__ fine, T* __restrict__ coarse) {
    const size_t node = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int Mc = nf + 1;
    if (node >= size_t(Mc) * Mc * Mc) return;
    restrict_node<T, false>(nf, fine, coarse, node);
}

// ---- transfers by coarse cells (transfer.cuh: prolong_cell_plane, restrict_cell)
template <typename T>
__global__ void __launch_bounds__(128) k_prolong_cells(int nc, const T* __restrict__ coarse, T* __restrict__ fine,
                                                       bool add) {
    const size_t ncell = size_t(nc) * nc * nc;
    const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= 15 * ncell) return;
    prolong_cell_plane<T>(nc, coarse, fine, add, int(t / (5 * ncell)), int((t / ncell) % 5), t % ncell);
}

template <typename T>
__global__ void __launch_bounds__(128) k_restrict_cells(int nc, const T* __restrict__ fine_r, T* __restrict__ coarse) {
    const size_t ncell = size_t(nc) * nc * nc;
    const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= 3 * ncell) return;
    restrict_cell<T>(nc, fine_r, coarse, int(t / ncell), t % ncell);
}

template <typename T>
__global__ void k_cheb_update(size_t n, const T* __restrict__ b, const T* __restrict__ Ax,
                              const T* __restrict__ dinv, T* __restrict__ d, T* __restrict__ x, T c1, T c2,
                              bool x_valid) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const T r = dinv[i] * (Ax ? b[i] - Ax[i] : b[i]);
        const T dn = (c1 != T(0) ? c1 * d[i] : T(0)) + c2 * r;
        d[i] = dn;
        x[i] = (x_valid ? x[i] : T(0)) + dn;
    }
}

template <typename T>
__global__ void k_residual(size_t n, const T* __restrict__ b, const T* __restrict__ Ax, T* __restrict__ r) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        r[i] = b[i] - Ax[i];
}

__global__ void k_cast_d2f(size_t n, const double* __restrict__ in, float* __restrict__ out) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        out[i] = float(in[i]);
}
__global__ void k_cast_f2d(size_t n, const float* __restrict__ in, double* __restrict__ out) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        out[i] = double(in[i]);
}

template <typename T>
__global__ void k_coarse_solve(int nf, const int* __restrict__ idx, const double* __restrict__ Ainv,
                               const T* __restrict__ b, T* __restrict__ x) {
    // one warp per row of the inverse: coalesced row reads, lane sums reduced in a fixed order
    const int r = int((size_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5), lane = int(threadIdx.x & 31);
    if (r >= nf) return;   // whole warps leave together
    const double* row = Ainv + size_t(r) * nf;
    double s = 0.0;
    for (int j = lane; j < nf; j += 32) s += row[j] * double(b[idx[j]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[idx[r]] = T(s);
}

__global__ void k_axpby(size_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}
__global__ void k_axpby_f(size_t n, float a, const float* __restrict__ x, float b, float* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = a * x[i] + (b == 0.0f ? 0.0f : b * y[i]);
}
__global__ void k_mul(size_t n, const double* __restrict__ a, const double* __restrict__ x, double* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = a[i] * x[i];
}
__global__ void k_sqrt(size_t n, const double* __restrict__ a, double* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = sqrt(a[i]);
}
__global__ void k_recip(size_t n, const double* __restrict__ a, double* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = 1.0 / a[i];
}
__global__ void k_add_scalar(size_t n, double v, double* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] += v;
}
__global__ void k_fill(size_t n, double v, double* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = v;
}

// splitmix64 (Steele, Lea, Flood 2014): output i of seed s is mix(s + (i+1) * golden);
// uniform double = top 53 bits * 2^-53; the vector entry is (u - 1/2) * mask.
__global__ void k_splitmix(size_t n, unsigned long long seed, const double* __restrict__ mask,
                           double* __restrict__ y) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        const double u = double(z >> 11) * (1.0 / 9007199254740992.0);
        y[i] = (u - 0.5) * (mask ? mask[i] : 1.0);
    }
}

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 608;   // 4 per SM on 152 SMs

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_part[kDotThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_part[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kDotThreads / 32; ++i) s += warp_part[i];
    __syncthreads();
    return s;
}

constexpr int kDotBatch = 8;

// grid (kDotBlocks, ceil((k + self) / kDotBatch)): partials[i * kDotBlocks + bx] = the block's slice
// of V_i . w for the kDotBatch vectors of its batch (vector k is w itself when self = 1), so w is
// read once per batch and every V_i once.
__global__ void __launch_bounds__(kDotThreads) k_multidot_partial(size_t n, int k, int self,
                                                                 const double* __restrict__ V, size_t ld,
                                                                 const double* __restrict__ w,
                                                                 double* __restrict__ partials) {
    const int i0 = blockIdx.y * kDotBatch;
    const int kt = k + self;
    double acc[kDotBatch];
#pragma unroll
    for (int b = 0; b < kDotBatch; ++b) acc[b] = 0.0;
    for (size_t e = size_t(blockIdx.x) * kDotThreads + threadIdx.x; e < n; e += size_t(kDotBlocks) * kDotThreads) {
        const double we = w[e];
#pragma unroll
        for (int b = 0; b < kDotBatch; ++b) {
            const int i = i0 + b;
            if (i < kt) acc[b] += (i < k ? V[size_t(i) * ld + e] : we) * we;
        }
    }
#pragma unroll
    for (int b = 0; b < kDotBatch; ++b) {
        const double s = block_sum(acc[b]);
        if (threadIdx.x == 0 && i0 + b < kt) partials[size_t(i0 + b) * kDotBlocks + blockIdx.x] = s;
    }
}

__global__ void k_multidot_final(int k, const double* __restrict__ partials, double* __restrict__ out) {
    const int i = blockIdx.x;
    if (i >= k) return;
    double acc = 0.0;
    for (int b = threadIdx.x; b < kDotBlocks; b += kDotThreads) acc += partials[size_t(i) * kDotBlocks + b];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) out[i] = s;
}

__global__ void k_multiaxpy(size_t n, int k, const double* __restrict__ V, size_t ld, const double* __restrict__ h,
                            double* __restrict__ w, double sign) {
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += h[i] * V[size_t(i) * ld + e];
        w[e] += sign * s;
    }
}

// ---- fused vector passes of the memory-light solvers (IDR(s), MINRES): several updates of the
// same entries, and the norm of an updated vector, in one sweep. Grid kDotBlocks x kDotThreads so
// that the per-block partial sums land where k_multidot_final reads them.

// y1 += a1 x1, y2 += a2 x2 (x2 null: y2 untouched); partials non-null: row 0 = slices of y1 . y1
__global__ void __launch_bounds__(kDotThreads) k_axpy2(size_t n, double a1, const double* __restrict__ x1,
                                                       double* __restrict__ y1, double a2,
                                                       const double* __restrict__ x2, double* __restrict__ y2,
                                                       double* __restrict__ partials) {
    double acc = 0.0;
    for (size_t e = size_t(blockIdx.x) * kDotThreads + threadIdx.x; e < n; e += size_t(kDotBlocks) * kDotThreads) {
        const double v = y1[e] + a1 * x1[e];
        y1[e] = v;
        acc += v * v;
        if (x2) y2[e] += a2 * x2[e];
    }
    if (partials) {
        const double sum = block_sum(acc);
        if (threadIdx.x == 0) partials[blockIdx.x] = sum;
    }
}

// rows 0, 1 = slices of x . y1 and x . y2
__global__ void __launch_bounds__(kDotThreads) k_dot2_partial(size_t n, const double* __restrict__ x,
                                                              const double* __restrict__ y1,
                                                              const double* __restrict__ y2,
                                                              double* __restrict__ partials) {
    double a = 0.0, b = 0.0;
    for (size_t e = size_t(blockIdx.x) * kDotThreads + threadIdx.x; e < n; e += size_t(kDotBlocks) * kDotThreads) {
        const double xe = x[e];
        a += xe * y1[e];
        b += xe * y2[e];
    }
    const double sa = block_sum(a), sb = block_sum(b);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = sa;
        partials[kDotBlocks + blockIdx.x] = sb;
    }
}

// w = a src + sign sum_i h_i V_i; w may be src or one of the rows V_i (each entry is read before
// it is written, by the same thread), so no restrict on them
__global__ void k_lincomb(size_t n, int k, const double* V, size_t ld, const double* __restrict__ h, double a,
                          const double* src, double* w, double sign) {
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += h[i] * V[size_t(i) * ld + e];
        w[e] = a * src[e] + sign * s;
    }
}

// MINRES: the next Lanczos vector and the two recurrences of the search directions,
//   vo = q + bv vo + cv v,  kwo = q + bk kwo + ck kw,  wo = z + bw wo + cw w,
// each as the two axpby steps of the unfused form in the same order
__global__ void k_minres_dirs(size_t n, const double* __restrict__ q, const double* __restrict__ z,
                              double* __restrict__ vo, const double* __restrict__ v, double bv, double cv,
                              double* __restrict__ kwo, const double* __restrict__ kw, double bk, double ck,
                              double* __restrict__ wo, const double* __restrict__ w, double bw, double cw) {
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
        const double qe = q[e];
        vo[e] = cv * v[e] + (qe + bv * vo[e]);
        kwo[e] = ck * kw[e] + (qe + bk * kwo[e]);
        wo[e] = cw * w[e] + (z[e] + bw * wo[e]);
    }
}

// MINRES: scale the new directions by f, x += e w, r -= e K w; row 0 of partials = slices of r . r
__global__ void __launch_bounds__(kDotThreads) k_minres_update(size_t n, double f, double* __restrict__ w,
                                                               double* __restrict__ kw, double e_,
                                                               double* __restrict__ x, double* __restrict__ r,
                                                               double* __restrict__ partials) {
    double acc = 0.0;
    for (size_t e = size_t(blockIdx.x) * kDotThreads + threadIdx.x; e < n; e += size_t(kDotBlocks) * kDotThreads) {
        const double we = f * w[e], kwe = f * kw[e];
        w[e] = we;
        kw[e] = kwe;
        x[e] += e_ * we;
        const double re = r[e] - e_ * kwe;
        r[e] = re;
        acc += re * re;
    }
    const double sum = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = sum;
}

inline unsigned grid_stride_blocks(size_t n) {
    const size_t b = (n + 255) / 256;
    return unsigned(b < 4864 ? (b == 0 ? 1 : b) : 4864);
}

}  // namespace

int multidot_blocks() { return kDotBlocks; }

template <typename T>
cudaError_t launch_prolongate(const LevelGeom& fine, const T* coarse, T* finev, bool add, cudaStream_t s) {
    const int nc = fine.n / 2;
    const size_t threads = 15 * size_t(nc) * nc * nc;
    LAUNCH(PROF_TRANSFER, s, k_prolong_cells<T><<<blocks_for(threads, 128), 128, 0, s>>>(nc, coarse, finev, add));
    return cudaGetLastError();
}
template cudaError_t launch_prolongate<float>(const LevelGeom&, const float*, float*, bool, cudaStream_t);
template cudaError_t launch_prolongate<double>(const LevelGeom&, const double*, double*, bool, cudaStream_t);

template <typename T>
cudaError_t launch_restrict(const LevelGeom& fine, const T* finev, T* coarse, cudaStream_t s, bool deterministic) {
    if (deterministic) {
        const size_t Mc = size_t(fine.n) + 1;
        LAUNCH(PROF_TRANSFER, s, k_restrict_nodes<T><<<blocks_for(Mc * Mc * Mc, 256), 256, 0, s>>>(fine.n, finev, coarse));
        return cudaGetLastError();
    }
    const int nc = fine.n / 2;
    const size_t Mc = size_t(2 * nc) + 1;
    cudaError_t e = cudaMemsetAsync(coarse, 0, 3 * Mc * Mc * Mc * sizeof(T), s);
    if (e != cudaSuccess) return e;
    const size_t threads = 3 * size_t(nc) * nc * nc;
    LAUNCH(PROF_TRANSFER, s, k_restrict_cells<T><<<blocks_for(threads, 128), 128, 0, s>>>(nc, finev, coarse));
    return cudaGetLastError();
}
template cudaError_t launch_restrict<float>(const LevelGeom&, const float*, float*, cudaStream_t, bool);
template cudaError_t launch_restrict<double>(const LevelGeom&, const double*, double*, cudaStream_t, bool);

template <typename T>
cudaError_t launch_cheb_update(size_t n, const T* b, const T* Ax, const T* dinv, T* d, T* x, double c1, double c2,
                               bool x_valid, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_cheb_update<T><<<grid_stride_blocks(n), 256, 0, s>>>(n, b, Ax, dinv, d, x, T(c1), T(c2), x_valid));
    return cudaGetLastError();
}
template cudaError_t launch_cheb_update<float>(size_t, const float*, const float*, const float*, float*, float*,
                                               double, double, bool, cudaStream_t);
template cudaError_t launch_cheb_update<double>(size_t, const double*, const double*, const double*, double*,
                                                double*, double, double, bool, cudaStream_t);

template <typename T>
cudaError_t launch_residual(size_t n, const T* b, const T* Ax, T* r, cudaStream_t s) {
    LAUNCH(PROF_SMOOTH_VEC, s, k_residual<T><<<grid_stride_blocks(n), 256, 0, s>>>(n, b, Ax, r));
    return cudaGetLastError();
}
template cudaError_t launch_residual<float>(size_t, const float*, const float*, float*, cudaStream_t);
template cudaError_t launch_residual<double>(size_t, const double*, const double*, double*, cudaStream_t);

cudaError_t launch_cast_d2f(size_t n, const double* in, float* out, cudaStream_t s) {
    LAUNCH(PROF_CAST, s, k_cast_d2f<<<grid_stride_blocks(n), 256, 0, s>>>(n, in, out));
    return cudaGetLastError();
}
cudaError_t launch_cast_f2d(size_t n, const float* in, double* out, cudaStream_t s) {
    LAUNCH(PROF_CAST, s, k_cast_f2d<<<grid_stride_blocks(n), 256, 0, s>>>(n, in, out));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(int nf, const int* free_idx, const double* Ainv, const T* b, T* x, cudaStream_t s) {
    if (nf <= 0) return cudaSuccess;
    LAUNCH(PROF_COARSE, s, k_coarse_solve<T><<<blocks_for(size_t(nf) * 32, 128), 128, 0, s>>>(nf, free_idx, Ainv, b, x));
    return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<float>(int, const int*, const double*, const float*, float*, cudaStream_t);
template cudaError_t launch_coarse_solve<double>(int, const int*, const double*, const double*, double*,
                                                 cudaStream_t);

cudaError_t launch_axpby(size_t n, double a, const double* x, double b, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_axpby<<<grid_stride_blocks(n), 256, 0, s>>>(n, a, x, b, y));
    return cudaGetLastError();
}
cudaError_t launch_axpby_f(size_t n, float a, const float* x, float b, float* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_axpby_f<<<grid_stride_blocks(n), 256, 0, s>>>(n, a, x, b, y));
    return cudaGetLastError();
}
cudaError_t launch_mul(size_t n, const double* a, const double* x, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_mul<<<grid_stride_blocks(n), 256, 0, s>>>(n, a, x, y));
    return cudaGetLastError();
}
cudaError_t launch_sqrt_vec(size_t n, const double* a, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_sqrt<<<grid_stride_blocks(n), 256, 0, s>>>(n, a, y));
    return cudaGetLastError();
}
cudaError_t launch_recip(size_t n, const double* a, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_recip<<<grid_stride_blocks(n), 256, 0, s>>>(n, a, y));
    return cudaGetLastError();
}
cudaError_t launch_add_scalar(size_t n, double v, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_add_scalar<<<grid_stride_blocks(n), 256, 0, s>>>(n, v, y));
    return cudaGetLastError();
}
cudaError_t launch_fill(size_t n, double v, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_fill<<<grid_stride_blocks(n), 256, 0, s>>>(n, v, y));
    return cudaGetLastError();
}
cudaError_t launch_splitmix_vector(size_t n, uint64_t seed, const double* mask, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_splitmix<<<grid_stride_blocks(n), 256, 0, s>>>(n, (unsigned long long)seed, mask, y));
    return cudaGetLastError();
}

cudaError_t launch_multidot(size_t n, int k, const double* V, size_t ld, const double* w, double* partials,
                            double* out, cudaStream_t s, bool self) {
    const int kt = k + (self ? 1 : 0);
    if (kt <= 0) return cudaSuccess;
    dim3 grid(kDotBlocks, unsigned((kt + kDotBatch - 1) / kDotBatch));
    LAUNCH(PROF_KRYLOV, s, k_multidot_partial<<<grid, kDotThreads, 0, s>>>(n, k, self ? 1 : 0, V, ld, w, partials));
    LAUNCH(PROF_KRYLOV, s, k_multidot_final<<<unsigned(kt), kDotThreads, 0, s>>>(kt, partials, out));
    return cudaGetLastError();
}

cudaError_t launch_axpy2(size_t n, double a1, const double* x1, double* y1, double a2, const double* x2, double* y2,
                         double* partials, double* out, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_axpy2<<<kDotBlocks, kDotThreads, 0, s>>>(n, a1, x1, y1, a2, x2, y2, out ? partials : nullptr));
    if (out) LAUNCH(PROF_KRYLOV, s, k_multidot_final<<<1, kDotThreads, 0, s>>>(1, partials, out));
    return cudaGetLastError();
}

cudaError_t launch_dot2(size_t n, const double* x, const double* y1, const double* y2, double* partials, double* out,
                        cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_dot2_partial<<<kDotBlocks, kDotThreads, 0, s>>>(n, x, y1, y2, partials));
    LAUNCH(PROF_KRYLOV, s, k_multidot_final<<<2, kDotThreads, 0, s>>>(2, partials, out));
    return cudaGetLastError();
}

cudaError_t launch_lincomb(size_t n, int k, const double* V, size_t ld, const double* h, double a, const double* src,
                           double* w, double sign, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_lincomb<<<grid_stride_blocks(n), 256, 0, s>>>(n, k, V, ld, h, a, src, w, sign));
    return cudaGetLastError();
}

cudaError_t launch_minres_dirs(size_t n, const double* q, const double* z, double* vo, const double* v, double bv,
                               double cv, double* kwo, const double* kw, double bk, double ck, double* wo,
                               const double* w, double bw, double cw, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_minres_dirs<<<grid_stride_blocks(n), 256, 0, s>>>(n, q, z, vo, v, bv, cv, kwo, kw, bk, ck,
                                                                             wo, w, bw, cw));
    return cudaGetLastError();
}

cudaError_t launch_minres_update(size_t n, double f, double* w, double* kw, double e, double* x, double* r,
                                 double* partials, double* out, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, k_minres_update<<<kDotBlocks, kDotThreads, 0, s>>>(n, f, w, kw, e, x, r, partials));
    LAUNCH(PROF_KRYLOV, s, k_multidot_final<<<1, kDotThreads, 0, s>>>(1, partials, out));
    return cudaGetLastError();
}

cudaError_t launch_multiaxpy(size_t n, int k, const double* V, size_t ld, const double* h, double* w, double sign,
                             cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    LAUNCH(PROF_KRYLOV, s, k_multiaxpy<<<grid_stride_blocks(n), 256, 0, s>>>(n, k, V, ld, h, w, sign));
    return cudaGetLastError();
}

}  // namespace stk
