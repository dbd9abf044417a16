// krylov.cu -- the Gram-Schmidt passes of the FGMRES Arnoldi step
// (Section 2.2.2) in double-float arithmetic on FP64 vectors.
//
// Classical Gram-Schmidt applied twice to w against V_0..V_{k-1}:
//   pass A   h1 = V^T w
//   pass B   w1 = w - V h1,  h2 = V^T w1,  |w1|^2,
//            hn = sqrt(max(|w1|^2 - |h2|^2, 0))   (h2 is small after pass A)
//   pass C   V_k = (w1 - V h2) / hn
// so that H(:, k-1) = h1 + h2 and H(k, k-1) = hn: every basis vector is read
// three times per iteration instead of four (pass B forms w1 and its dot
// products in one sweep).
//
// Why double-float: each basis entry read costs one multiply-add, and on this
// GPU the FP64 pipe (about 1/72 of the FP32 rate) retires fewer multiply-adds
// per second than HBM delivers doubles, so native FP64 Gram-Schmidt runs at
// the FP64 pipe's speed, not at memory speed. Here the basis V is stored as
// double-float pairs (hi, lo floats in the 8 bytes of a double; ~47
// significant bits), w stays FP64 and is split once per entry (split_double,
// integer instructions), products are exact (FMA two_prod) and sums are
// compensated (mac), so every dot product carries about 44 significant bits,
// far below anything the solver's 1e-8 tolerance can see; the preconditioner
// receives V_j converted back to FP64 (df_to_double). The native FP64 passes
// (vec.cu) remain available and are the arithmetic of the FP64 option.
//
// Layout: a pair of adjacent vector entries is handled by 1, 2 or 4 adjacent
// threads, each owning a share of the basis rows. A thread copies its rows'
// 16-byte entry pairs into its own column of shared memory with asynchronous
// copies that bypass L1 (all in flight without holding registers; the next
// sweep's copies are issued before the current sweep is computed) and works
// from there; the projection sums are combined across the entry's threads by
// shuffles. The per-thread dot sums are reduced per warp and CTA in
// double-float and written as doubles to `partials`, which one CTA adds in a
// fixed order, so the results do not depend on scheduling. Basis rows have an
// even stride so that every entry pair is 16-byte aligned.
#include "df64.cuh"
#include "internal.cuh"
#include "prof.cuh"

#define LAUNCH(cls, s, ...)              \
    do {                                \
        prof_begin((cls), (s));         \
        __VA_ARGS__;                    \
        prof_end((cls), (s));           \
        prof_count(1);                  \
    } while (0)

namespace stk {

namespace {

using q2::df64;

constexpr int kGsThreads = 128;
constexpr int kGsMaxK = 64;                 // largest basis of the double-float passes
constexpr int kGsMaxBlocks = 2432;          // 16 per SM on 152 SMs; the partials buffer is sized for this

enum GsMode { GS_DOT = 0, GS_PROJECT_DOT = 1, GS_PROJECT_SCALE = 2, GS_LAG = 3 };

// An entry pair is handled by TPE = KB / RB threads (adjacent lanes), each owning RB <= STK_GS_RB
// basis rows: with 16, one thread up to KB = 8, two up to 32, four at 64. Measured on whole 64^3
// and 96^3 solves: 32 rows per thread is slower, and so are 8 (Krylov kernels +10% / +13%) and 4
// (+69% / +84%): fewer rows per thread add shuffles and partial sums faster than the higher
// occupancy hides latency.
#ifndef STK_GS_RB
#define STK_GS_RB 16
#endif
__host__ __device__ constexpr int gs_rb(int /*mode*/, int kb) {
    return kb <= 8 ? kb : kb / 2 > STK_GS_RB ? STK_GS_RB : kb / 2;
}
template <int MODE, int KB>
struct GsShape {
    static constexpr int RB = gs_rb(MODE, KB);
    static constexpr int TPE = KB / RB;
    static constexpr int PPB = kGsThreads / TPE;   // entry pairs per CTA and sweep
};

// per thread: two buffers of RB rows x 16 bytes (an entry pair), then coefficients (two sets
// for GS_LAG) and sums
inline size_t gs_smem(int mode, int kb) {
    return (4 * size_t(gs_rb(mode, kb)) * kGsThreads + size_t(kb) * (mode == GS_LAG ? 2 : 1) + 4 * (size_t(kb) + 1)) *
           sizeof(double);
}

// 16-byte asynchronous copy global -> shared, not cached in L1.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned sa = unsigned(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ df64 shfl_down_df(const df64& v, int o) {
    return df64(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ df64 shfl_xor_df(const df64& v, int o) {
    return df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// V holds double-float entries (hi, lo floats in 8 bytes) in rows of stride ld (even, > n when
// n is odd, and 16-byte aligned rows); w, h and scale are FP64.
// MODE GS_DOT:           partials <- V^T w                           (rows 0..k-1)
// MODE GS_PROJECT_DOT:   w <- w - V h; partials <- V^T w, w . w      (rows 0..k)
// MODE GS_PROJECT_SCALE: y <- (w - V h) * scale[0], y double-float   (no partials)
// MODE GS_LAG (delayed re-orthogonalisation; j = k - 1, row j holds u_j, the once-projected
//   vector of the previous step, and scale = its record c = V_{<j}^T u_j, |u_j|^2, alpha,
//   1 / alpha with alpha = |u_j - V_{<j} c|, or null for j = 0 where row 0 is final):
//   v_j = (u_j - V_{<j} c) / alpha is written over row j; w1 = w - V_{<=j} h with v_j in row j,
//   written as double-float to row j + 1 (y = V); partials <- V_{<=j}^T w1 (row j: v_j), w1 . w1.
// KB >= k is the compile-time bound on the basis size (8, 16, 32 or 64). A thread handles the
// entry pair (2p, 2p + 1): one 16-byte copy per row.
template <int MODE, int KB>
__global__ void __launch_bounds__(kGsThreads) k_gs_df(size_t n, int k, const double* __restrict__ V, size_t ld,
                                                      const double* __restrict__ h, double* __restrict__ w,
                                                      const double* __restrict__ scale, double* y,
                                                      double* __restrict__ partials) {
    using S = GsShape<MODE, KB>;
    constexpr int RB = S::RB, TPE = S::TPE, PPB = S::PPB;
    extern __shared__ double smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int g = tid % TPE;              // row group: rows r0 .. r0 + rb - 1
    const int slot = tid / TPE;           // entry pair within the CTA's sweep
    const int rb = (k + TPE - 1) / TPE;   // rows per group (<= RB), balanced over the groups
    const int r0 = g * rb;
    float4* col = reinterpret_cast<float4*>(smem) + tid;                       // [2][RB][kGsThreads], own column
    constexpr int NH = MODE == GS_LAG ? 2 : 1;
    df64* hs = reinterpret_cast<df64*>(smem + 4 * RB * kGsThreads);            // split coefficients
    df64* hb = hs + KB;                                                        // GS_LAG: those of v_j
    df64* red = reinterpret_cast<df64*>(smem + 4 * RB * kGsThreads + NH * KB); // [4][KB + 1] warp sums
    if constexpr (MODE == GS_LAG) {
        // w1 = w - sum_{i<j} h_i v_i - h_j v_j with v_j = (u_j - sum_{i<j} c_i v_i) / alpha, as one
        // combination of the stored rows (a) and v_j itself (b)
        const int j = k - 1;
        const double ia = scale ? scale[j + 2] : 1.0;
        for (int i = tid; i < k; i += kGsThreads) {
            const double ci = (scale && i < j) ? scale[i] : 0.0;
            hs[i] = q2::split_double(i < j ? h[i] - h[j] * ci * ia : h[j] * ia);
            hb[i] = q2::split_double(i < j ? -ci * ia : ia);
        }
    } else if constexpr (MODE != GS_DOT) {
        for (int i = tid; i < k; i += kGsThreads) hs[i] = q2::split_double(h[i]);
    }
    __syncthreads();
    const df64 sc = MODE == GS_PROJECT_SCALE ? q2::split_double(scale[0]) : df64();
    constexpr int NA = MODE == GS_PROJECT_SCALE ? 1 : RB;
    df64 acc[NA];
#pragma unroll
    for (int r = 0; r < NA; ++r) acc[r] = df64();
    df64 self, vdot;
    // Every lane of a warp runs the same number of sweeps (pairs past the end are masked), so
    // that the full-warp shuffles below are always convergent. The copies of sweep s + 1 are
    // issued before sweep s is computed (two buffers per thread).
    const size_t np = (n + 1) / 2;
    const size_t warp_first = size_t(blockIdx.x) * PPB + size_t(wid) * (32 / TPE);
    const size_t stride = size_t(gridDim.x) * PPB;
    const size_t p0 = size_t(blockIdx.x) * PPB + slot;
    auto issue = [&](size_t base, int buf) {
        const size_t p = p0 + base;
        if (p < np) {
            // the row pointer is advanced row by row (not precomputed per row) to keep registers low
            const double* src = V + 2 * p + size_t(r0) * ld;
            float4* dst = col + buf * (RB * kGsThreads);
            const int nr = min(rb, k - r0);
#pragma unroll 4
            for (int r = 0; r < nr; ++r) {
                cp_async16(dst + r * kGsThreads, src);
                src += ld;
            }
        }
        cp_async_commit();
    };
    auto load_w = [&](size_t p, double& a, double& b) {
        a = 0.0;
        b = 0.0;
        if (p < np) {
            a = w[2 * p];
            if (2 * p + 1 < n) b = w[2 * p + 1];
        }
    };
    size_t base = 0;
    issue(base, 0);
    double wn0, wn1;
    load_w(p0, wn0, wn1);
    for (int it = 0; warp_first + base < np; ++it) {
        const size_t p = p0 + base;
        const bool in = p < np;
        const bool in1 = 2 * p + 1 < n;
        issue(base + stride, (it + 1) & 1);
        df64 w0 = q2::split_double(wn0), w1 = q2::split_double(wn1);
        load_w(p + stride, wn0, wn1);
        cp_async_wait_prev();
        const float4* cv = col + (it & 1) * (RB * kGsThreads);
        if constexpr (MODE == GS_DOT) {
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r < rb && in && r0 + r < k) {
                    const float4 v = cv[r * kGsThreads];
                    q2::mac(acc[r], df64(v.x, v.y), w0);
                    q2::mac(acc[r], df64(v.z, v.w), w1);
                }
        } else if constexpr (MODE == GS_LAG) {
            df64 s0, s1, t0, t1;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r < rb && in && r0 + r < k) {
                    const float4 v = cv[r * kGsThreads];
                    q2::mac(s0, hs[r0 + r], df64(v.x, v.y));
                    q2::mac(s1, hs[r0 + r], df64(v.z, v.w));
                    q2::mac(t0, hb[r0 + r], df64(v.x, v.y));
                    q2::mac(t1, hb[r0 + r], df64(v.z, v.w));
                }
            q2::renorm(s0);
            q2::renorm(s1);
            q2::renorm(t0);
            q2::renorm(t1);
#pragma unroll
            for (int o = 1; o < TPE; o <<= 1) {
                s0 += shfl_xor_df(s0, o);
                s1 += shfl_xor_df(s1, o);
                t0 += shfl_xor_df(t0, o);
                t1 += shfl_xor_df(t1, o);
            }
            w0 = w0 - s0;
            w1 = w1 - s1;
            if (in && g == 0) {
                float4* vj = reinterpret_cast<float4*>(y + size_t(k - 1) * ld);
                float4* uk = reinterpret_cast<float4*>(y + size_t(k) * ld);
                if (in1) {
                    vj[p] = make_float4(t0.hi, t0.lo, t1.hi, t1.lo);
                    uk[p] = make_float4(w0.hi, w0.lo, w1.hi, w1.lo);
                } else {
                    reinterpret_cast<df64*>(vj)[2 * p] = t0;
                    reinterpret_cast<df64*>(uk)[2 * p] = w0;
                }
                q2::mac(self, w0, w0);
                q2::mac(self, w1, w1);
                q2::mac(vdot, t0, w0);
                q2::mac(vdot, t1, w1);
            }
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r < rb && in && r0 + r < k - 1) {
                    const float4 v = cv[r * kGsThreads];
                    q2::mac(acc[r], df64(v.x, v.y), w0);
                    q2::mac(acc[r], df64(v.z, v.w), w1);
                }
        } else {
            df64 s0, s1;
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r < rb && in && r0 + r < k) {
                    const float4 v = cv[r * kGsThreads];
                    q2::mac(s0, hs[r0 + r], df64(v.x, v.y));
                    q2::mac(s1, hs[r0 + r], df64(v.z, v.w));
                }
            q2::renorm(s0);
            q2::renorm(s1);
#pragma unroll
            for (int o = 1; o < TPE; o <<= 1) {
                s0 += shfl_xor_df(s0, o);
                s1 += shfl_xor_df(s1, o);
            }
            w0 = w0 - s0;
            w1 = w1 - s1;
            if constexpr (MODE == GS_PROJECT_SCALE) {
                if (in && g == 0) {
                    const df64 y0 = w0 * sc, y1 = w1 * sc;
                    if (in1) reinterpret_cast<float4*>(y)[p] = make_float4(y0.hi, y0.lo, y1.hi, y1.lo);
                    else reinterpret_cast<df64*>(y)[2 * p] = y0;
                }
            } else {
                if (in && g == 0) {
                    w[2 * p] = w0.to_double();
                    if (in1) w[2 * p + 1] = w1.to_double();
                    q2::mac(self, w0, w0);
                    q2::mac(self, w1, w1);
                }
#pragma unroll
                for (int r = 0; r < RB; ++r)
                    if (r < rb && in && r0 + r < k) {
                        const float4 v = cv[r * kGsThreads];
                        q2::mac(acc[r], df64(v.x, v.y), w0);
                        q2::mac(acc[r], df64(v.z, v.w), w1);
                    }
            }
        }
        if ((it & 1) == 1) {
#pragma unroll
            for (int r = 0; r < NA; ++r) q2::renorm(acc[r]);
            q2::renorm(self);
            if constexpr (MODE == GS_LAG) q2::renorm(vdot);
        }
        base += stride;
    }
    cp_async_wait_all();
    if constexpr (MODE != GS_PROJECT_SCALE) {
#pragma unroll
        for (int r = 0; r < RB; ++r) q2::renorm(acc[r]);
        q2::renorm(self);
        q2::renorm(vdot);
        // sums over the warp's entries (lanes with the same g), then over the CTA's 4 warps
#pragma unroll
        for (int r = 0; r < RB; ++r)
            for (int o = 16; o >= TPE; o >>= 1) acc[r] += shfl_down_df(acc[r], o);
        for (int o = 16; o >= TPE; o >>= 1) self += shfl_down_df(self, o);
        if constexpr (MODE == GS_LAG)
            for (int o = 16; o >= TPE; o >>= 1) vdot += shfl_down_df(vdot, o);
        // GS_LAG: row j's sum is vdot (v_j is not in shared memory)
        const int kd = MODE == GS_LAG ? k - 1 : k;
        if (lane < TPE) {
#pragma unroll
            for (int r = 0; r < RB; ++r)
                if (r < rb && r0 + r < kd) red[wid * (KB + 1) + r0 + r] = acc[r];
            if (g == 0) red[wid * (KB + 1) + k] = self;
            if (MODE == GS_LAG && g == 0) red[wid * (KB + 1) + k - 1] = vdot;
        }
        __syncthreads();
        const int rows = MODE == GS_PROJECT_DOT || MODE == GS_LAG ? k + 1 : k;
        for (int row = tid; row < rows; row += kGsThreads) {
            df64 v = red[row];
#pragma unroll
            for (int q = 1; q < kGsThreads / 32; ++q) v += red[q * (KB + 1) + row];
            partials[size_t(row) * gridDim.x + blockIdx.x] = v.to_double();
        }
    }
}

// out[row] = sum over the nb CTA partials of `row`, for rows < rows; with hn: out[rows] = hn and
// out[rows + 1] = 1 / hn, hn = sqrt(max(out[rows-1] - sum_{i < rows-1} out[i]^2, 0)).
// With lag (the record of GS_LAG's previous step, j = rows - 1): out[j] = u_j . w becomes
// v_j . w = (out[j] - sum_{i<j} c_i out[i]) / alpha.
__global__ void __launch_bounds__(1024) k_gs_final(int rows, int nb, const double* __restrict__ partials,
                                                   double* __restrict__ out, int with_hn,
                                                   const double* __restrict__ lag) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int row = wid; row < rows; row += 32) {
        double v = 0.0;
        for (int b = lane; b < nb; b += 32) v += partials[size_t(row) * nb + b];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[row] = v;
    }
    if (lag) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int j = rows - 1;
            double t = out[j];
            for (int i = 0; i < j; ++i) t = fma(-lag[i], out[i], t);
            out[j] = t * lag[j + 2];
        }
    }
    if (!with_hn) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sq = 0.0;
        for (int i = 0; i + 1 < rows; ++i) sq = fma(out[i], out[i], sq);
        const double hn = sqrt(fmax(out[rows - 1] - sq, 0.0));
        out[rows] = hn;
        out[rows + 1] = 1.0 / hn;
    }
}

// Blocks per launch: as many CTAs as fit on the GPU at once (at most kGsMaxBlocks), per KB.
int gs_blocks[4][4];
int gs_device = -1;

inline int kb_index(int k) { return k <= 8 ? 0 : k <= 16 ? 1 : k <= 32 ? 2 : 3; }

template <int MODE, int KB>
cudaError_t configure_one(int sms) {
    cudaError_t e = cudaFuncSetAttribute(k_gs_df<MODE, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(gs_smem(MODE, KB)));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_df<MODE, KB>, kGsThreads, gs_smem(MODE, KB));
    if (e != cudaSuccess) return e;
    const int nb = per_sm * sms;
    gs_blocks[MODE][kb_index(KB)] = nb < 1 ? 1 : (nb > kGsMaxBlocks ? kGsMaxBlocks : nb);
    return cudaSuccess;
}

template <int MODE>
cudaError_t configure_mode(int sms) {
    cudaError_t e;
    if ((e = configure_one<MODE, 8>(sms)) != cudaSuccess) return e;
    if ((e = configure_one<MODE, 16>(sms)) != cudaSuccess) return e;
    if ((e = configure_one<MODE, 32>(sms)) != cudaSuccess) return e;
    return configure_one<MODE, 64>(sms);
}

// Launches k_gs_df<MODE, KB> for the smallest KB >= k; returns its grid size.
template <int MODE>
int launch_df(size_t n, int k, const double* V, size_t ld, const double* h, double* w, const double* scale,
              double* y, double* partials, cudaStream_t s) {
    const int ki = kb_index(k);
    const int nb = gs_blocks[MODE][ki];
    switch (ki) {
        case 0:
            LAUNCH(PROF_KRYLOV, s, (k_gs_df<MODE, 8><<<nb, kGsThreads, gs_smem(MODE, 8), s>>>(n, k, V, ld, h, w, scale, y, partials)));
            break;
        case 1:
            LAUNCH(PROF_KRYLOV, s, (k_gs_df<MODE, 16><<<nb, kGsThreads, gs_smem(MODE, 16), s>>>(n, k, V, ld, h, w, scale, y, partials)));
            break;
        case 2:
            LAUNCH(PROF_KRYLOV, s, (k_gs_df<MODE, 32><<<nb, kGsThreads, gs_smem(MODE, 32), s>>>(n, k, V, ld, h, w, scale, y, partials)));
            break;
        default:
            LAUNCH(PROF_KRYLOV, s, (k_gs_df<MODE, 64><<<nb, kGsThreads, gs_smem(MODE, 64), s>>>(n, k, V, ld, h, w, scale, y, partials)));
            break;
    }
    return nb;
}

// Native FP64: out[k+1] = hn, out[k+2] = 1 / hn from out[0..k-1] = h2 and out[k] = |w1|^2.
__global__ void k_gs_hn(int k, double* __restrict__ out) {
    double sq = 0.0;
    for (int i = 0; i < k; ++i) sq = fma(out[i], out[i], sq);
    const double hn = sqrt(fmax(out[k] - sq, 0.0));
    out[k + 1] = hn;
    out[k + 2] = 1.0 / hn;
}

// Native FP64: y = (w - V h) * scale[0], one entry per thread.
__global__ void k_gs_project_scale_fp64(size_t n, int k, const double* __restrict__ V, size_t ld,
                                        const double* __restrict__ h, const double* __restrict__ w,
                                        const double* __restrict__ scale, double* __restrict__ y) {
    const double sc = scale[0];
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < k; ++i) s = fma(h[i], V[size_t(i) * ld + e], s);
        y[e] = (w[e] - s) * sc;
    }
}

// y = w * scale as double-float pairs; x = double-float pairs as FP64.
__global__ void k_df_store_scaled(size_t n, const double* __restrict__ w, double scale, df64* __restrict__ y) {
    const df64 sc = q2::split_double(scale);
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x)
        y[e] = q2::split_double(w[e]) * sc;
}
__global__ void k_df_to_double(size_t n, const df64* __restrict__ v, double scale, double* __restrict__ x) {
    for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += size_t(gridDim.x) * blockDim.x)
        x[e] = v[e].to_double() * scale;
}

inline unsigned stride_blocks(size_t n) {
    const size_t b = (n + 255) / 256;
    return unsigned(b < 4864 ? (b == 0 ? 1 : b) : 4864);
}

}  // namespace

int gs_partials_blocks() { return kGsMaxBlocks; }
int gs_max_k() { return kGsMaxK; }

cudaError_t launch_df_store_scaled(size_t n, const double* w, double scale, double* y, cudaStream_t s) {
    LAUNCH(PROF_KRYLOV, s, (k_df_store_scaled<<<stride_blocks(n), 256, 0, s>>>(n, w, scale, reinterpret_cast<df64*>(y))));
    return cudaGetLastError();
}
cudaError_t launch_df_to_double(size_t n, const double* v, double* x, cudaStream_t s, double scale) {
    LAUNCH(PROF_KRYLOV, s, (k_df_to_double<<<stride_blocks(n), 256, 0, s>>>(n, reinterpret_cast<const df64*>(v), scale, x)));
    return cudaGetLastError();
}

cudaError_t gs_configure() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev == gs_device) return cudaSuccess;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = configure_mode<GS_DOT>(sms)) != cudaSuccess) return e;
    if ((e = configure_mode<GS_PROJECT_DOT>(sms)) != cudaSuccess) return e;
    if ((e = configure_mode<GS_PROJECT_SCALE>(sms)) != cudaSuccess) return e;
    if ((e = configure_mode<GS_LAG>(sms)) != cudaSuccess) return e;
    gs_device = dev;
    return cudaSuccess;
}

cudaError_t launch_gs_dot(size_t n, int k, const double* V, size_t ld, const double* w, double* partials,
                          double* out, bool df, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    if (df && k > kGsMaxK) return cudaErrorInvalidValue;
    if (!df) return launch_multidot(n, k, V, ld, w, partials, out, s, false);
    const int nb = launch_df<GS_DOT>(n, k, V, ld, nullptr, const_cast<double*>(w), nullptr, nullptr, partials, s);
    LAUNCH(PROF_KRYLOV, s, (k_gs_final<<<1, 1024, 0, s>>>(k, nb, partials, out, 0, nullptr)));
    return cudaGetLastError();
}

cudaError_t launch_gs_project_dot(size_t n, int k, const double* V, size_t ld, const double* h, double* w,
                                  double* partials, double* out, bool df, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    if (df && k > kGsMaxK) return cudaErrorInvalidValue;
    if (!df) {
        cudaError_t e = launch_multiaxpy(n, k, V, ld, h, w, -1.0, s);
        if (e != cudaSuccess) return e;
        if ((e = launch_multidot(n, k, V, ld, w, partials, out, s, true)) != cudaSuccess) return e;
        LAUNCH(PROF_KRYLOV, s, (k_gs_hn<<<1, 1, 0, s>>>(k, out)));
        return cudaGetLastError();
    }
    const int nb = launch_df<GS_PROJECT_DOT>(n, k, V, ld, h, w, nullptr, nullptr, partials, s);
    LAUNCH(PROF_KRYLOV, s, (k_gs_final<<<1, 1024, 0, s>>>(k + 1, nb, partials, out, 1, nullptr)));
    return cudaGetLastError();
}

cudaError_t launch_gs_project_scale(size_t n, int k, const double* V, size_t ld, const double* h, const double* w,
                                    const double* scale, double* y, bool df, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    if (df && k > kGsMaxK) return cudaErrorInvalidValue;
    if (!df) {
        const size_t b = (n + 255) / 256;
        const unsigned grid = unsigned(b < 4864 ? (b == 0 ? 1 : b) : 4864);
        LAUNCH(PROF_KRYLOV, s, (k_gs_project_scale_fp64<<<grid, 256, 0, s>>>(n, k, V, ld, h, w, scale, y)));
        return cudaGetLastError();
    }
    launch_df<GS_PROJECT_SCALE>(n, k, V, ld, h, const_cast<double*>(w), scale, y, nullptr, s);
    return cudaGetLastError();
}

}  // namespace stk

namespace stk {

cudaError_t launch_gs_dot_lag(size_t n, int k, const double* V, size_t ld, const double* w, double* partials,
                              double* out, const double* lag, cudaStream_t s) {
    if (k <= 0 || k > kGsMaxK) return cudaErrorInvalidValue;
    const int nb = launch_df<GS_DOT>(n, k, V, ld, nullptr, const_cast<double*>(w), nullptr, nullptr, partials, s);
    LAUNCH(PROF_KRYLOV, s, (k_gs_final<<<1, 1024, 0, s>>>(k, nb, partials, out, 0, lag)));
    return cudaGetLastError();
}

cudaError_t launch_gs_lag_project(size_t n, int k, double* V, size_t ld, const double* h, const double* lag,
                                  const double* w, double* partials, double* out, cudaStream_t s) {
    if (k <= 0 || k > kGsMaxK) return cudaErrorInvalidValue;
    const int nb = launch_df<GS_LAG>(n, k, V, ld, h, const_cast<double*>(w), lag, V, partials, s);
    LAUNCH(PROF_KRYLOV, s, (k_gs_final<<<1, 1024, 0, s>>>(k + 1, nb, partials, out, 1, nullptr)));
    return cudaGetLastError();
}

}  // namespace stk
