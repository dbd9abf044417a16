// brick_tc.cu -- the FP32 velocity level operator A_l (Section 2.1, definition of A) with the
// cell products on the tensor cores (tcgen05, kind::f16), accumulated into the operator
// accumulator that the epilogue kernels of brick.cu consume (the plain product, the residual, or
// the Jacobi-Chebyshev step of Section 2.2.1).
//
// On a cube cell of side h with the cell-constant (averaged) viscosity mu_c of Section 2.3, the
// element operator is A_cell = mu_c h A_hat, with one fixed 81 x 81 reference matrix A_hat
// (mu = h = 1), so the product over a brick of 128 cells is one dense [128 x 81] x [81 x 81]^T
// matrix product: row m = the 81 gathered values of cell m, column n = output DoF n (component
// c, local node a at index 27 c + a). 5400 A_hat is an integer matrix whose entries have at most
// 6 significant bits and magnitude <= 2^15, so it is exact in f16. The gathered FP32 values of a
// cell are scaled by a power of two that brings their largest magnitude into [2^14, 2^15) and split
// into two f16 terms, hi = v with its significand cut to 11 bits and lo = f16(v - hi), which carry
// 22 significant bits: the product is two MMAs with f32 accumulation, D = U_hi A^T + U_lo A^T, and
// row m is multiplied by mu_c h / (5400 s_m) afterwards. Per 128-cell brick: 12 tcgen05.mma of
// M = 128, N = 96, K = 16 (81 padded to 96), A operand in tensor memory, B (the f16 table) in
// shared memory.
//
// Work decomposition: a persistent kernel, one CTA of two groups of 8 warps per SM; group g of CTA
// i takes the bricks (8 x 4 x 4 cells) 2 i + g, 2 i + g + 2 G, ... Two threads per cell: thread
// (half h, cell m) sits in a warp whose TMEM lane quarter holds row m, and handles the columns
// [48 h, 48 h + 48) of both the A row and the D row. Per brick a group
//   1. gathers its cells' values (constrained nodes read as 0), exchanges the two halves' largest
//      magnitudes through shared memory, scales, splits and stores the f16 terms into its TMEM A
//      columns (tcgen05.st);
//   2. after a group barrier one thread issues the 12 MMAs into the group's TMEM accumulator and
//      commits them to the group's mbarrier;
//   3. waits for the commit (bounded by %globaltimer; on timeout the kernel records it in the
//      status word, waits for its MMAs and leaves), loads its half of the D row (tcgen05.ld),
//      scales it and adds it into the brick's node tile in shared memory (shared atomics);
//   4. after a group barrier writes the tile out and clears it: a node strictly inside the brick
//      belongs to this brick alone and is stored; a node on a brick face is shared with the
//      neighbouring bricks and is added to the accumulator with a global atomic; nodes on the
//      domain boundary are left (identity rows, handled by the epilogue kernels).
// The two groups of a CTA overlap each other's phases.
#include "brick.cuh"
#include "prof.cuh"
#include "tcgen05.cuh"

#include <cuda_fp16.h>
#include <cstdint>

namespace stk {

namespace {

constexpr int kRows = 96;                 // 81 DoFs padded to a multiple of 16
constexpr int kTableBytes = kRows * kRows * 2;
constexpr int kTmemCols = 512;            // two groups x (A: 96 columns, D: 96 columns) at 0 / 256
constexpr int kGroupCols = 256;
constexpr int kAcol = 0, kDcol = 128;
constexpr double kTableScale = 5400.0;    // 5400 A_hat is an integer matrix
static_assert(kBrickX * kBrickY * kBrickZ == 128, "one MMA row per cell of the brick");
constexpr int kTX = 2 * kBrickX + 1, kTY = 2 * kBrickY + 1, kTZ = 2 * kBrickZ + 1;   // brick node tile
// padded tile layout: the 32 cells of a warp (8 along x, 4 along y) land on rows 2 x 24 words
// apart, so their shared atomics conflict at most 2-way
constexpr int kRowP = 24, kPlaneP = kRowP * kTY, kTileP = kPlaneP * kTZ;
constexpr size_t kTileBytes = (size_t(3) * kTileP * 4 + 127) / 128 * 128;
// dynamic shared memory: the f16 table, per group the node tile, the groups' largest-magnitude
// exchange and the node list; asked for above half of the SM's shared memory, so that one CTA
// (which holds all 512 TMEM columns) runs per SM
constexpr int kOutEntries = 3 * kTX * kTY * kTZ;   // tile nodes x components per brick
constexpr size_t kOutBytes = size_t(kOutEntries) * 8;
constexpr size_t kGroupBytes = kTileBytes;   // per group: the node tile
constexpr size_t kSmemUsed = size_t(kTableBytes) + 2 * kGroupBytes + 2 * 256 * 4 + kOutBytes;
constexpr size_t kSmemAsk = kSmemUsed > 120 * 1024 ? kSmemUsed : 120 * 1024;

// Byte offset of element (row n, column k) of the 96 x 96 table in the no-swizzle K-major
// canonical layout: core matrices of 8 rows x 8 halves (128 bytes), the one of row group n/8 and
// column group k/8 at ((k/8) * 12 + n/8) * 128; so core matrices adjacent along K are 1536 bytes
// apart and along N 128 bytes.
__host__ __device__ constexpr int table_offset(int n, int k) {
    return ((k >> 3) * (kRows / 8) + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
}
constexpr uint32_t kLbo = (kRows / 8) * 128, kSbo = 128;

// Reference matrix A_hat column by column with the library's own sum-factorised cell operator
// (mu = h = 1), in FP64, scaled by 5400, checked to be an integer that f16 holds exactly, stored
// in the canonical layout. flag != 0 afterwards if any entry is not.
__global__ void k_table_build(__half* table, int* flag) {
    const int j = threadIdx.x;   // input DoF 27 c + a
    if (j >= kRows) return;
    double u[3][27], w[3][27];
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 27; ++a) u[c][a] = (c * 27 + a == j) ? 1.0 : 0.0;
    if (j < 81) q2::cell_A(u, w);
    unsigned char* tb = reinterpret_cast<unsigned char*>(table);
    for (int n = 0; n < kRows; ++n) {
        double v = 0.0;
        if (j < 81 && n < 81) v = w[n / 27][n % 27] * kTableScale;
        const double r = rint(v);
        const __half hv = __double2half(r);
        if (fabs(v - r) > 1e-6 * (1.0 + fabs(v)) || double(__half2float(hv)) != r) atomicOr(flag, 1);
        *reinterpret_cast<__half*>(tb + table_offset(n, j)) = hv;
    }
}

// bar.red over one group: true iff v is true on every thread of the group.
__device__ __forceinline__ bool group_all(int id, int count, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"(uint32_t(v)), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// Node list entry e = (component c, tile node li, lj, lk), x fastest: .x = li + M (lj + M lk), the
// node's offset from the brick's node (0,0,0) in the level; .y = its tile index | 1 << 13 if it lies
// on a face of the brick | li << 14 | lj << 19 | lk << 23 | c << 27.
struct BrickNodes {
    int gi0, gj0, gk0;
    bool edge;          // the brick reaches the domain boundary: test each node
};

__device__ __forceinline__ BrickNodes brick_nodes(int b, int nbx, int nby, int M) {
    BrickNodes bn;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    bn.gi0 = 2 * kBrickX * bx;
    bn.gj0 = 2 * kBrickY * by;
    bn.gk0 = 2 * kBrickZ * bz;
    bn.edge = bn.gi0 == 0 || bn.gj0 == 0 || bn.gk0 == 0 || bn.gi0 + kTX - 1 >= M - 1 || bn.gj0 + kTY - 1 >= M - 1 ||
              bn.gk0 + kTZ - 1 >= M - 1;
    return bn;
}

// True if the node of list word y lies inside the level and off its boundary (a free node).
__device__ __forceinline__ bool free_node(const BrickNodes& bn, uint32_t y, int M) {
    const int gi = bn.gi0 + int((y >> 14) & 31u), gj = bn.gj0 + int((y >> 19) & 15u), gk = bn.gk0 + int((y >> 23) & 15u);
    return gi > 0 && gj > 0 && gk > 0 && gi < M - 1 && gj < M - 1 && gk < M - 1;
}

// Where the cell sits against the domain boundary: its local nodes with index 0 / 2 along an axis
// are constrained when the cell is the first / last one along that axis; an invalid cell (outside
// the level) reads nothing.
struct CellFlags {
    bool valid, xlo, xhi, ylo, yhi, zlo, zhi;
};

// Gathered values k in [K0, K1) (k = 27 c + i + 3 j + 9 k_z) of the cell whose node (0,0,0) is at
// `cell` (constrained nodes and invalid cells: 0) into u[k - K0]; row offsets roff[j + 3 k_z] =
// M j + M^2 k_z (32-bit, fixed per launch), the three nodes of a row at immediate offsets.
// Returns the largest magnitude.
template <int K0, int K1>
__device__ __forceinline__ float gather_part(const float* __restrict__ cell, size_t nodes, const int (&roff)[9],
                                             const CellFlags& f, float (&u)[K1 - K0]) {
    float mx = 0.0f;
#pragma unroll
    for (int kk = K0; kk < K1; ++kk) {
        const int c = kk / 27, loc = kk % 27, i = loc % 3, j = (loc / 3) % 3, k = loc / 9;
        const bool skip = !f.valid || (k == 0 && f.zlo) || (k == 2 && f.zhi) || (j == 0 && f.ylo) ||
                          (j == 2 && f.yhi) || (i == 0 && f.xlo) || (i == 2 && f.xhi);
        const float* row = cell + size_t(c) * nodes + roff[j + 3 * k];
        const float v = skip ? 0.0f : __ldg(row + i);
        u[kk - K0] = v;
        mx = fmaxf(mx, fabsf(v));
    }
    return mx;
}

// hi = v with the significand cut to 11 bits (exact in f16 for the scaled range), lo = v - hi
// (exact in FP32, rounded once to f16); packed two per 32-bit TMEM column, lower k low.
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
    const float h0 = __uint_as_float(__float_as_uint(v0) & 0xFFFFE000u);
    const float h1 = __uint_as_float(__float_as_uint(v1) & 0xFFFFE000u);
    const __half2 hh = __floats2half2_rn(h0, h1);
    const __half2 ll = __floats2half2_rn(v0 - h0, v1 - h1);
    hi = *reinterpret_cast<const uint32_t*>(&hh);
    lo = *reinterpret_cast<const uint32_t*>(&ll);
}

// Scaled and split values k in [K0, K0 + 48) (u holds k in [K0, K1), zero beyond) into the TMEM
// A columns: hi terms at K0 / 2 + [0, 24), lo terms at 48 + K0 / 2 + [0, 24).
template <int K0, int K1>
__device__ __forceinline__ void store_part(uint32_t tmem_lane, const float (&u)[K1 - K0], float s) {
#pragma unroll
    for (int chunk = 0; chunk < 3; ++chunk) {   // 8 columns = 16 values
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k0 = K0 + 16 * chunk + 2 * q;
            const float v0 = k0 < K1 ? u[k0 - K0] * s : 0.0f;
            const float v1 = k0 + 1 < K1 ? u[k0 + 1 - K0] * s : 0.0f;
            split_pair(v0, v1, hi[q], lo[q]);
        }
        tc::tmem_st8(tmem_lane + uint32_t(kAcol + K0 / 2 + 8 * chunk), hi);
        tc::tmem_st8(tmem_lane + uint32_t(kAcol + 48 + K0 / 2 + 8 * chunk), lo);
    }
}

// D columns [N0, N0 + 48) of this thread's row, times f, added into the node tile (base = the
// cell's local node (0,0,0) in the tile) when add is set. Every thread of the warp must call it:
// tcgen05.ld is warp-collective (.sync.aligned), so only the adds depend on the thread's cell.
template <int N0>
__device__ __forceinline__ void scatter_part(uint32_t tmem_lane, float f, int base, float* tile, bool add) {
    uint32_t r[3][16];
#pragma unroll
    for (int chunk = 0; chunk < 3; ++chunk) tc::tmem_ld16(tmem_lane + uint32_t(kDcol + N0 + 16 * chunk), r[chunk]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int chunk = 0; chunk < 3; ++chunk)
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int n = N0 + 16 * chunk + q;
            if (n < 81 && add) {
                const int c = n / 27, loc = n % 27, i = loc % 3, j = (loc / 3) % 3, k = loc / 9;
                atomicAdd(tile + c * kTileP + base + i + kRowP * j + kPlaneP * k, __uint_as_float(r[chunk][q]) * f);
            }
        }
}

// DIRECT variant of phases 3-4: this thread's half of the D row, times f, added straight into the
// accumulator row by row (row r = component r / 9, local (j, k) = ((r % 9) % 3, (r % 9) / 3), the
// three nodes n = 3r .. 3r + 2) with one 8-byte and one 4-byte atomic (add_row3's parity rule);
// rows on the domain boundary are skipped, boundary nodes inside a row get 0. Warp-collective
// like scatter_part.
template <int N0>
__device__ __forceinline__ void scatter_direct(uint32_t tmem_lane, float f, float* cell_out, size_t nodes,
                                               const int (&roff)[9], const CellFlags& fl) {
    uint32_t r[3][16];
#pragma unroll
    for (int chunk = 0; chunk < 3; ++chunk) tc::tmem_ld16(tmem_lane + uint32_t(kDcol + N0 + 16 * chunk), r[chunk]);
    tc::tmem_ld_wait();
    constexpr int R0 = N0 / 3, R1 = (N0 + 48 < 81 ? N0 + 48 : 81) / 3;
#pragma unroll
    for (int rr = R0; rr < R1; ++rr) {
        const int c = rr / 9, j = (rr % 9) % 3, k = (rr % 9) / 3;
        if (!fl.valid || (j == 0 && fl.ylo) || (j == 2 && fl.yhi) || (k == 0 && fl.zlo) || (k == 2 && fl.zhi)) continue;
        const int q = 3 * rr - N0;
        const float v0 = fl.xlo ? 0.0f : __uint_as_float(r[q / 16][q % 16]) * f;
        const float v1 = __uint_as_float(r[(q + 1) / 16][(q + 1) % 16]) * f;
        const float v2 = fl.xhi ? 0.0f : __uint_as_float(r[(q + 2) / 16][(q + 2) % 16]) * f;
        add_row3(cell_out + size_t(c) * nodes + roff[j + 3 * k], (c + j + k) & 1, v0, v1, v2);
    }
}

template <bool DIRECT>
__global__ void __launch_bounds__(512, 1)
    k_cell_tc(BrickArgs<float> a, float* __restrict__ acc, const __half* __restrict__ table, unsigned* status,
              unsigned long long wait_ns, int nbx, int nby, int nbricks) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base_s;
    const int g = int(threadIdx.x >> 8), half = int((threadIdx.x >> 7) & 1), tid = int(threadIdx.x & 127);
    const int warp = int(threadIdx.x >> 5), gt = int(threadIdx.x & 255);
    // the table: 16-byte copies
    {
        const uint4* src = reinterpret_cast<const uint4*>(table);
        uint4* dst = reinterpret_cast<uint4*>(smem);
        for (int i = int(threadIdx.x); i < kTableBytes / 16; i += int(blockDim.x)) dst[i] = src[i];
    }
    float* tile = reinterpret_cast<float*>(smem + kTableBytes + size_t(g) * kGroupBytes);
    float* smax = reinterpret_cast<float*>(smem + kTableBytes + 2 * kGroupBytes) + 256 * g;   // [half][cell]
    uint2* outl = reinterpret_cast<uint2*>(smem + kTableBytes + 2 * kGroupBytes + 2 * 256 * 4);
    const int M = a.M;
    for (int e = int(threadIdx.x); e < kOutEntries; e += int(blockDim.x)) {
        const int c = e / (kTX * kTY * kTZ), t = e % (kTX * kTY * kTZ);
        const int li = t % kTX, lj = (t / kTX) % kTY, lk = t / (kTX * kTY);
        const bool face = li == 0 || li == kTX - 1 || lj == 0 || lj == kTY - 1 || lk == 0 || lk == kTZ - 1;
        outl[e] = make_uint2(uint32_t(li + M * (lj + M * lk)),
                             uint32_t(c * kTileP + li + kRowP * lj + kPlaneP * lk) | (face ? 1u << 13 : 0u) |
                                 uint32_t(li) << 14 | uint32_t(lj) << 19 | uint32_t(lk) << 23 | uint32_t(c) << 27);
    }
    for (int i = gt; i < 3 * kTileP; i += 256) tile[i] = 0.0f;
    tc::fence_async_smem();
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base_s, kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base_s + uint32_t(g * kGroupCols);
    const uint32_t tmem_lane = tmem + (uint32_t(32 * (warp & 3)) << 16);   // this warp's TMEM lane quarter
    const uint32_t table_s = tc::smem_addr(smem);
    constexpr uint32_t idesc = tc::idesc_f16_f32(128, kRows);
    const int bar_id = 1 + g;
    uint32_t phase = 0;
    const int cx = tid % kBrickX, cy = (tid / kBrickX) % kBrickY, cz = tid / (kBrickX * kBrickY);
    const int tbase = 2 * cx + kRowP * 2 * cy + kPlaneP * 2 * cz;   // the cell's node (0,0,0) in the tile
    int roff[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) roff[r] = M * (r % 3) + M * M * (r / 3);

#pragma unroll 1
    for (int b = int(blockIdx.x) * 2 + g; b < nbricks; b += 2 * int(gridDim.x)) {
        const BrickNodes bn = brick_nodes(b, nbx, nby, M);
        const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
        const int ci = kBrickX * bx + cx, cj = kBrickY * by + cy, ck = kBrickZ * bz + cz;
        const bool valid = ci < a.n && cj < a.n && ck < a.n;
        const CellFlags fl{valid, ci == 0, ci == a.n - 1, cj == 0, cj == a.n - 1, ck == 0, ck == a.n - 1};
        const float* cell =
            a.src + (valid ? size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck)) : size_t(0));
        // ---- 1. gather this half's values, exchange the largest magnitude, split, store into TMEM
        float u0[48], u1[33];
        float mx = half == 0 ? gather_part<0, 48>(cell, a.nodes, roff, fl, u0)
                             : gather_part<48, 81>(cell, a.nodes, roff, fl, u1);
        smax[128 * half + tid] = mx;
        tc::group_sync(bar_id, 256);
        mx = fmaxf(smax[tid], smax[128 + tid]);
        // s = 2^(141 - e) for mx in [2^(e - 127), 2^(e - 126)): largest scaled magnitude in [2^14, 2^15)
        int ex = int((__float_as_uint(mx) >> 23) & 0xFFu);
        ex = ex < 15 ? 15 : (ex > 254 ? 254 : ex);
        const float s = __uint_as_float(uint32_t(268 - ex) << 23);
        const float inv_s = __uint_as_float(uint32_t(ex - 14) << 23);
        if (half == 0) store_part<0, 48>(tmem_lane, u0, s);
        else store_part<48, 81>(tmem_lane, u1, s);
        tc::tmem_st_wait();
        tc::fence_before_sync();
        tc::group_sync(bar_id, 256);
        // ---- 2. one thread issues D = U_hi A^T + U_lo A^T
        if (gt == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int part = 0; part < 2; ++part)
#pragma unroll
                for (int kstep = 0; kstep < kRows / 16; ++kstep) {
                    const uint64_t bdesc = tc::smem_desc(table_s + uint32_t(kstep) * 2u * kLbo, kLbo, kSbo);
                    tc::mma_f16_ts(tmem + kDcol, tmem + uint32_t(kAcol + 48 * part + 8 * kstep), bdesc, idesc,
                                   (part | kstep) != 0);
                }
            tc::mma_commit(&mbar[g]);
        }
        // ---- 3. one warp waits (bounded) for the MMAs; all add their half of the D row to the tile
        bool waited = true;
        if (gt < 32) waited = tc::mbar_wait_bounded(&mbar[g], phase, wait_ns);
        const bool ok = group_all(bar_id, 256, waited);
        if (!ok) {
            if (gt == 0) {
                atomicOr(status, 1u);
                tc::mbar_wait_bounded(&mbar[g], phase, 2000000000ull);   // let the MMAs finish
            }
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        if constexpr (DIRECT) {
            const float f = valid ? a.mu[size_t(ci) + size_t(a.n) * (cj + size_t(a.n) * ck)] * a.h * inv_s *
                                        float(1.0 / kTableScale)
                                  : 0.0f;
            float* cell_out = acc + (valid ? size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck))
                                           : size_t(0));
            if (half == 0) scatter_direct<0>(tmem_lane, f, cell_out, a.nodes, roff, fl);
            else scatter_direct<48>(tmem_lane, f, cell_out, a.nodes, roff, fl);
            tc::fence_before_sync();
            continue;   // the next brick's first group barrier orders these TMEM loads before its MMAs
        }
        {
            const float f = valid ? a.mu[size_t(ci) + size_t(a.n) * (cj + size_t(a.n) * ck)] * a.h * inv_s *
                                        float(1.0 / kTableScale)
                                  : 0.0f;
            if (half == 0) scatter_part<0>(tmem_lane, f, tbase, tile, valid);
            else scatter_part<48>(tmem_lane, f, tbase, tile, valid);
        }
        tc::fence_before_sync();
        tc::group_sync(bar_id, 256);
        // ---- 4. write the tile out and clear it
        float* const out0 = acc + (size_t(bn.gi0) + size_t(M) * (size_t(bn.gj0) + size_t(M) * size_t(bn.gk0)));
#pragma unroll 4
        for (int e = gt; e < kOutEntries; e += 256) {
            const uint2 w = outl[e];
            float* p = tile + (w.y & 0x1FFFu);
            const float v = *p;
            *p = 0.0f;
            if (bn.edge && !free_node(bn, w.y, M)) continue;
            float* out = out0 + size_t(w.y >> 27) * a.nodes + w.x;
            if (w.y & (1u << 13)) atomicAdd(out, v);
            else *out = v;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base_s, kTmemCols);
    }
}

int sm_count() {
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

cudaError_t tc_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_cell_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemAsk));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_cell_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemAsk));
}

size_t tc_table_bytes() { return size_t(kTableBytes); }

cudaError_t tc_build_table(void* table, int* flag, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_table_build<<<1, kRows, 0, s>>>(static_cast<__half*>(table), flag);
    return cudaGetLastError();
}

cudaError_t launch_cell_tc(const BrickArgs<float>& a, float* acc, const TcArgs& t, cudaStream_t s) {
    const int nbx = (a.n + kBrickX - 1) / kBrickX, nby = (a.n + kBrickY - 1) / kBrickY,
              nbz = (a.n + kBrickZ - 1) / kBrickZ;
    const int nbricks = nbx * nby * nbz;
    int grid = (nbricks + 1) / 2;
    if (grid > sm_count()) grid = sm_count();
    prof_begin(PROF_VMULT_F32, s);
    // direct pair atomics need an 8-byte aligned accumulator; otherwise the node-tile scatter
    if ((reinterpret_cast<uintptr_t>(acc) & 7u) == 0)
        k_cell_tc<true><<<grid, 512, kSmemAsk, s>>>(a, acc, static_cast<const __half*>(t.table), t.status, t.wait_ns,
                                                    nbx, nby, nbricks);
    else
        k_cell_tc<false><<<grid, 512, kSmemAsk, s>>>(a, acc, static_cast<const __half*>(t.table), t.status, t.wait_ns,
                                                     nbx, nby, nbricks);
    prof_end(PROF_VMULT_F32, s);
    prof_count(1);
    return cudaGetLastError();
}

}  // namespace stk
