// outer_tc.cu -- the outer Stokes operator [A B^T; B 0] (Section 2.1) to FP64 accuracy on the
// tensor cores, by exact products of an integer element table with fixed-point digit slices of the
// FP64 inputs (arithmetic in sliced.cuh).
//
// Per cell, x = [u (81, constrained nodes read as 0); (25 h / mu_c) p (8)] and one 89 x 89 integer
// table K = [[5400 A_ref, -216 R^T], [-216 R, 0]] (exact in f16) give
//   y_u = (mu_c h / 5400) (K x)_u,   y_p = (h^2 / 216) (K x)_p.
// x is written in fixed point against its largest magnitude 2^Ex and split into 7 balanced
// base-256 digit slices; slice j of the 128 cells of a tile (8 x 4 x 4 cells) is the A operand
// (tensor memory, f16) of 6 tcgen05.mma (M 128, N 96, K 16; 89 padded to 96) against the table in
// shared memory, accumulated in FP32 in tensor memory; every partial sum is an integer below 2^24,
// so each slice product is exact. The slices are recombined in double-float as they come, scaled,
// written as FP64 with integer instructions, and added into the outputs with FP64 atomics.
// The pressure rows take u's digits against Ex; where (25 h / mu_c) p exceeds the velocity values
// by more than 2^8 (Ex - Eu > 8) they lose too many bits, and that cell's B u is formed instead
// with the sum-factorised double-float moments.
//
// Work decomposition: persistent, one CTA of 256 threads per SM (it holds all 512 TMEM columns:
// 7 x 48 digit-slice columns and a 96-column accumulator); two threads per cell, thread (half h,
// cell m) in a warp whose TMEM lane quarter holds row m, owning the inputs and output columns
// [48 h, 48 h + 48). Per tile:
//   1. gather, exchange the halves' largest magnitudes through shared memory, write the 7 digit
//      slices into tensor memory (tcgen05.st);
//   2. for each slice: one thread issues its 6 MMAs and commits them to an mbarrier; all wait
//      (bounded by %globaltimer: on timeout the kernel records STOKES_TIMEOUT in the status word,
//      waits for its MMAs and leaves), read their 48 accumulator columns (tcgen05.ld) into the
//      recombination, and meet at a barrier before the next slice overwrites the accumulator;
//   3. write the outputs (free velocity rows and the pressure rows) with FP64 atomics.
// The caller clears the outputs first and copies the constrained rows afterwards (identity).
#include "internal.cuh"
#include "prof.cuh"
#include "sliced.cuh"
#include "tcgen05.cuh"

#include <cuda_fp16.h>
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

using q2::df64;
namespace sl = sliced;

constexpr int kTX = 8, kTY = 4, kTZ = 4;           // cells of a tile
constexpr int kCells = kTX * kTY * kTZ;            // 128: one MMA row per cell
constexpr int kThreads = 2 * kCells;
constexpr int kK = 96, kN = 96;                    // 89 inputs / outputs padded to multiples of 16
constexpr int kHalf = 48;                          // inputs and output columns per thread
constexpr int kTableBytes = kN * kK * 2;
constexpr int kAcols = kK / 2;                     // TMEM columns of one digit slice (f16 pairs)
constexpr int kDcol = sl::kDigits * kAcols;        // 336: the accumulator
constexpr int kTmemCols = 512;
// dynamic shared memory: the table and the halves' exponents; asked for above half of the SM's
// shared memory so that one CTA (which holds all 512 TMEM columns) runs per SM
constexpr size_t kSmemUsed = size_t(kTableBytes) + 4 * kCells * sizeof(int);
constexpr size_t kSmemAsk = 120 * 1024;
static_assert(kSmemUsed <= kSmemAsk, "shared memory");
static_assert(kDcol + kN <= kTmemCols, "tensor memory");

// Byte offset of element (row n, column k) of the 96 x 96 f16 table in the no-swizzle K-major
// canonical layout (core matrices of 8 rows x 8 halves; adjacent along K 1536 bytes apart, along N
// 128 bytes), the layout the tensor-core level operator's table uses.
__host__ __device__ constexpr int table_offset(int n, int k) {
    return ((k >> 3) * (kN / 8) + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
}
constexpr uint32_t kLbo = (kN / 8) * 128, kSbo = 128;

// K column by column from the library's own reference-cell operators (sliced::table_column),
// checked to be integers f16 holds exactly; flag != 0 afterwards if any entry is not.
__global__ void k_outer_table_build(__half* table, int* flag) {
    const int k = int(threadIdx.x);
    if (k >= kK) return;
    double col[sl::kNu], colp[sl::kNp];
    bool ok = true;
    if (k < sl::kNx) ok = sl::table_column(k, col, colp);
    unsigned char* tb = reinterpret_cast<unsigned char*>(table);
    for (int n = 0; n < kN; ++n) {
        double v = 0.0;
        if (k < sl::kNx && n < sl::kNu) v = col[n];
        else if (k < sl::kNu && n < sl::kNx) v = colp[n - sl::kNu];
        const __half hv = __double2half(v);
        if (double(__half2float(hv)) != v) ok = false;
        *reinterpret_cast<__half*>(tb + table_offset(n, k)) = hv;
    }
    if (!ok) atomicOr(flag, 1);
}

struct OuterTcArgs {
    int n, M;
    size_t nodes;
    double h;
    const double* mu;
    const double* src_u;
    const double* src_p;
    double* dst_u;
    double* dst_p;
    const __half* table;
    unsigned* status;
    unsigned long long wait_ns;
    int nbx, nby, ntiles;
};

// Input k of the cell (ci, cj, ck): velocity DoF k < 81 (component k / 27, local node k % 27;
// constrained nodes read as 0), pressure vertex k - 81 scaled by ps = 25 h / mu_c, 0 beyond 89.
// `off` receives the DoF's offset in its output vector (velocity: component block included), or
// -1 for a constrained node or a padding entry.
__device__ __forceinline__ double cell_input(const OuterTcArgs& a, int ci, int cj, int ck, int k, double ps,
                                             long long& off) {
    off = -1;
    if (k < sl::kNu) {
        const int c = k / 27, loc = k % 27;
        const int i = 2 * ci + loc % 3, j = 2 * cj + (loc / 3) % 3, kz = 2 * ck + loc / 9;
        if (i == 0 || j == 0 || kz == 0 || i == a.M - 1 || j == a.M - 1 || kz == a.M - 1) return 0.0;
        off = (long long)(size_t(c) * a.nodes + size_t(i) + size_t(a.M) * (size_t(j) + size_t(a.M) * size_t(kz)));
        return a.src_u[off];
    }
    if (k < sl::kNx) {
        const int v = k - sl::kNu, P = a.n + 1;
        off = (long long)(size_t(ci + (v & 1)) + size_t(P) * (size_t(cj + ((v >> 1) & 1)) + size_t(P) * size_t(ck + (v >> 2))));
        return ps * a.src_p[off];
    }
    return 0.0;
}

// Offset of output row n (< 89) of the cell in its vector (velocity: component block included), or
// -1 for a constrained velocity node.
__device__ __forceinline__ long long row_offset(const OuterTcArgs& a, int ci, int cj, int ck, int n) {
    if (n < sl::kNu) {
        const int c = n / 27, loc = n % 27;
        const int i = 2 * ci + loc % 3, j = 2 * cj + (loc / 3) % 3, kz = 2 * ck + loc / 9;
        if (i == 0 || j == 0 || kz == 0 || i == a.M - 1 || j == a.M - 1 || kz == a.M - 1) return -1;
        return (long long)(size_t(c) * a.nodes + size_t(i) + size_t(a.M) * (size_t(j) + size_t(a.M) * size_t(kz)));
    }
    const int v = n - sl::kNu, P = a.n + 1;
    return (long long)(size_t(ci + (v & 1)) + size_t(P) * (size_t(cj + ((v >> 1) & 1)) + size_t(P) * size_t(ck + (v >> 2))));
}

// The cell's B u with the double-float moments (sliced::bu_moments), added into dst_p.
__device__ __noinline__ void cell_Bu_fallback(const OuterTcArgs& a, int ci, int cj, int ck) {
    df64 u[sl::kNu], bu[sl::kNp];
    for (int k = 0; k < sl::kNu; ++k) {
        long long off;
        u[k] = q2::split_double(cell_input(a, ci, cj, ck, k, 0.0, off));
    }
    sl::bu_moments(u, bu);
    for (int v = 0; v < sl::kNp; ++v)
        atomicAdd(a.dst_p + row_offset(a, ci, cj, ck, sl::kNu + v), -a.h * a.h * bu[v].to_double());
}

__device__ __forceinline__ uint32_t pack_digits(int d0, int d1) {
    const __half2 hh = __floats2half2_rn(float(d0), float(d1));
    return *reinterpret_cast<const uint32_t*>(&hh);
}

// Next digit of X (lowest first): X = d + 256 X'.
__device__ __forceinline__ int next_digit(long long& X) {
    const int d = int((signed char)(X & 0xFF));
    X = (X - d) >> 8;   // exact: X - d is a multiple of 256 (arithmetic shift)
    return d;
}

__global__ void __launch_bounds__(kThreads, 1) k_outer_tc(OuterTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base_s;
    const int half = int(threadIdx.x >> 7), m = int(threadIdx.x & 127), warp = int(threadIdx.x >> 5);
    {   // the table: 16-byte copies
        const uint4* src = reinterpret_cast<const uint4*>(a.table);
        uint4* dst = reinterpret_cast<uint4*>(smem);
        for (int i = int(threadIdx.x); i < kTableBytes / 16; i += int(blockDim.x)) dst[i] = src[i];
    }
    int* sx = reinterpret_cast<int*>(smem + kTableBytes);   // [half][cell] largest binade of x
    int* su = sx + 2 * kCells;                               // [half][cell] largest binade of u
    tc::fence_async_smem();
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base_s, kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_s;
    const uint32_t tmem_lane = tmem + (uint32_t(32 * (warp & 3)) << 16);   // this warp's TMEM lane quarter
    const uint32_t table_s = tc::smem_addr(smem);
    constexpr uint32_t idesc = tc::idesc_f16_f32(kCells, kN);
    uint32_t phase = 0;
    const int cx = m % kTX, cy = (m / kTX) % kTY, cz = m / (kTX * kTY);
    const int k0 = kHalf * half;
    const double hA = a.h / sl::kScaleA;
    const df64 sB = q2::split_double(a.h * a.h / sl::kScaleB);

#pragma unroll 1
    for (int t = int(blockIdx.x); t < a.ntiles; t += int(gridDim.x)) {
        const int bx = t % a.nbx, by = (t / a.nbx) % a.nby, bz = t / (a.nbx * a.nby);
        const int ci = kTX * bx + cx, cj = kTY * by + cy, ck = kTZ * bz + cz;
        const bool valid = ci < a.n && cj < a.n && ck < a.n;
        const double mu_c = valid ? a.mu[size_t(ci) + size_t(a.n) * (size_t(cj) + size_t(a.n) * size_t(ck))] : 1.0;
        const double ps = half == 1 ? 25.0 * a.h / mu_c : 0.0;
        // ---- 1. gather this half's inputs, exchange the largest binades, digits into TMEM
        long long X[kHalf];
        int ex = sl::kNoExp, eu = sl::kNoExp;
#pragma unroll
        for (int q = 0; q < kHalf; ++q) {
            long long off;
            const double v = valid ? cell_input(a, ci, cj, ck, k0 + q, ps, off) : 0.0;
            X[q] = (long long)q2::dbl_bits(v);   // the bits, until the exponent is known
            const int b = sl::binade(v);
            ex = b > ex ? b : ex;
            if (k0 + q < sl::kNu) eu = b > eu ? b : eu;
        }
        sx[kCells * half + m] = ex;
        su[kCells * half + m] = eu;
        __syncthreads();
        const int Ex = max(sx[m], sx[kCells + m]), Eu = max(su[m], su[kCells + m]);
#pragma unroll
        for (int q = 0; q < kHalf; ++q)
            X[q] = Ex == sl::kNoExp ? 0 : sl::to_fixed(sl::dbl_from_bits((unsigned long long)X[q]), Ex);
#pragma unroll
        for (int j = 0; j < sl::kDigits; ++j)
#pragma unroll
            for (int chunk = 0; chunk < 3; ++chunk) {   // 8 columns = 16 inputs
                uint32_t r[8];
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const int q = 16 * chunk + 2 * w;
                    const int d0 = next_digit(X[q]);
                    const int d1 = next_digit(X[q + 1]);
                    r[w] = pack_digits(d0, d1);
                }
                tc::tmem_st8(tmem_lane + uint32_t(kAcols * j + kAcols / 2 * half + 8 * chunk), r);
            }
        tc::tmem_st_wait();
        tc::fence_before_sync();
        __syncthreads();
        // ---- 2. slice by slice: one thread issues D = A_j K^T, all read and recombine
        df64 acc[kHalf];
        bool ok = true;
#pragma unroll 1
        for (int j = 0; j < sl::kDigits; ++j) {
            if (threadIdx.x == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int ks = 0; ks < kK / 16; ++ks) {
                    const uint64_t bdesc = tc::smem_desc(table_s + uint32_t(ks) * 2u * kLbo, kLbo, kSbo);
                    tc::mma_f16_ts(tmem + kDcol, tmem + uint32_t(kAcols * j + 8 * ks), bdesc, idesc, ks != 0);
                }
                tc::mma_commit(&mbar);
            }
            bool waited = true;
            if (threadIdx.x < 32) waited = tc::mbar_wait_bounded(&mbar, phase, a.wait_ns);
            ok = __syncthreads_and(waited) != 0;
            if (!ok) break;
            phase ^= 1u;
            tc::fence_after_sync();
            uint32_t r[3][16];
#pragma unroll
            for (int chunk = 0; chunk < 3; ++chunk)
                tc::tmem_ld16(tmem_lane + uint32_t(kDcol + kHalf * half + 16 * chunk), r[chunk]);
            tc::tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < kHalf; ++q) sl::slice_step(acc[q], __uint_as_float(r[q / 16][q % 16]), j == 0);
            tc::fence_before_sync();
            __syncthreads();   // the accumulator is read before the next slice's MMAs overwrite it
        }
        if (!ok) {
            if (threadIdx.x == 0) {
                atomicOr(a.status, 1u);
                tc::mbar_wait_bounded(&mbar, phase, 2000000000ull);   // let the MMAs finish
            }
            break;
        }
        // ---- 3. outputs: V s 2^(Ex - 54), V = acc 2^48
        if (valid && Ex != sl::kNoExp) {
            const df64 sA = q2::split_double(mu_c * hA);
            const int shift = Ex - sl::kFrac + sl::kCombineShift;
            const bool moments = Eu != sl::kNoExp && Ex - Eu > sl::kMaxGap;
#pragma unroll
            for (int q = 0; q < kHalf; ++q) {
                const int n = k0 + q;
                if (n < sl::kNu) {
                    const long long off = row_offset(a, ci, cj, ck, n);
                    if (off >= 0) atomicAdd(a.dst_u + off, sl::compose(acc[q] * sA, shift));
                } else if (n < sl::kNx && !moments) {
                    atomicAdd(a.dst_p + row_offset(a, ci, cj, ck, n), sl::compose(acc[q] * sB, shift));
                }
            }
            if (moments && half == 1) cell_Bu_fallback(a, ci, cj, ck);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base_s, kTmemCols);
    }
}

int sm_count_tc() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

}  // namespace

size_t outer_tc_table_bytes() { return size_t(kTableBytes); }

cudaError_t outer_tc_setup(void* table, int* flag, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_outer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemAsk));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), s)) != cudaSuccess) return e;
    k_outer_table_build<<<1, kK, 0, s>>>(static_cast<__half*>(table), flag);
    return cudaGetLastError();
}

cudaError_t launch_outer_tc(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                            double* dst_u, double* dst_p, const void* table, unsigned* status,
                            unsigned long long wait_ns, cudaStream_t s) {
    const int nbx = (g.n + kTX - 1) / kTX, nby = (g.n + kTY - 1) / kTY, nbz = (g.n + kTZ - 1) / kTZ;
    const int ntiles = nbx * nby * nbz;
    const int grid = ntiles < sm_count_tc() ? ntiles : sm_count_tc();
    OuterTcArgs a{g.n, g.M, g.nodes, g.h, mu, src_u, src_p, dst_u, dst_p, static_cast<const __half*>(table),
                  status, wait_ns, nbx, nby, ntiles};
    LAUNCH(PROF_STOKES_F64, s, (k_outer_tc<<<grid, kThreads, kSmemAsk, s>>>(a)));
    return cudaGetLastError();
}

}  // namespace stk
