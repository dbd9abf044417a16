// sliced.cuh -- the outer Stokes operator [A B^T; B 0] of one cube cell (Section 2.1) as exact
// products of small integer tables with fixed-point digit slices of the FP64 inputs: the
// arithmetic of a tensor-core form of the outer operator, as plain functions that a host program
// can run cell by cell.
//
// On a cube cell of side h with cell viscosity mu_c the element blocks are A = mu_c h A_ref,
// B = -h^2 R and B^T = -h^2 R^T (A_ref the mu = h = 1 velocity operator, R the moments
// int d_c(phi_m) psi_v on the reference cell). 5400 A_ref and 216 R are integer matrices (exact
// integration of the Q2 and Q1 polynomials; at most 6 significant bits and magnitude <= 2^15), so
//   y_u = (mu_c h / 5400) K_X x,   x = [u; (25 h / mu_c) p],   K_X = [5400 A_ref | -216 R^T],
//   y_p = (h^2 / 216) K_U u,                                  K_U = -216 R.
// The 89 inputs x of a cell are written in fixed point against their largest magnitude 2^E
// (|v| < 2^E): X = round(v 2^(54 - E)), |X| <= 2^54, then as 7 balanced base-256 digits,
// X = sum_j d_j 256^j with d_j in [-128, 127]. One digit slice times a row of K = [K_X; K_U 0] is an
// integer below 78,464 * 2^7 < 2^24 in magnitude at every partial sum (78,464 is the largest row
// absolute sum), so a product of f16 digits with the f16-exact table accumulated in FP32 is exact
// in any order: D_j = K d_j exactly. The slices are recombined, V = sum_j 256^j D_j (up to 2^72),
// in double-float, multiplied by the cell's scale, and written as the FP64 value V s 2^(E - 54)
// with integer instructions only (GB300 runs FP64 instructions at 1/72 of the FP32 rate). The
// pressure rows see u against x's exponent; a cell where (25 h / mu_c) p exceeds u by more than
// 2^8 forms its B u with double-float moments instead. Error against exact arithmetic: 2^-55 of
// the largest input per input, ~2^-46 of the recombined value per output.
// Splitting the inputs into fixed-point slices whose products a low-precision matrix unit forms
// exactly is the error-free transformation of K. Ozaki, T. Ogita, S. Oishi and S. M. Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012); here the element table is itself an integer matrix, so
// only the inputs are split, and the slices are balanced base-256 digits of one 54-bit integer per
// input.
#pragma once

#include "df64.cuh"
#include "q2_basis.cuh"

namespace stk {
namespace sliced {

constexpr int kNu = 81;            // velocity DoFs of a cell (27 c + a)
constexpr int kNp = 8;             // pressure DoFs of a cell
constexpr int kNx = kNu + kNp;     // inputs of the y_u product
constexpr int kDigits = 7;         // balanced base-256 digits of a 54-bit fixed-point value
constexpr int kFrac = 54;          // X = round(v 2^(kFrac - E))
constexpr double kScaleA = 5400.0; // 5400 A_ref is an integer matrix
constexpr double kScaleB = 216.0;  // 216 R is an integer matrix

// ---- the integer tables, built from the library's own reference-cell operators
// Column k of K_X (k < 81: velocity DoF k; k >= 81: pressure vertex k - 81) into col[0..80];
// column k of K_U (k < 81) into colp[0..7]. Values are the integers in double; entries that are
// not integers to 1e-6 are reported through the return value (false).
__host__ __device__ inline bool table_column(int k, double (&col)[kNu], double (&colp)[kNp]) {
    for (int n = 0; n < kNu; ++n) col[n] = 0.0;
    for (int v = 0; v < kNp; ++v) colp[v] = 0.0;
    if (k < kNu) {
        double u[3][27], w[3][27];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 27; ++a) u[c][a] = (27 * c + a == k) ? 1.0 : 0.0;
        double ulin[81];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 27; ++a) ulin[27 * c + a] = u[c][a];
        q2::cell_A(u, w);   // overwrites u
        for (int n = 0; n < kNu; ++n) col[n] = kScaleA * w[n / 27][n % 27];
        double r[kNp] = {0, 0, 0, 0, 0, 0, 0, 0};
        q2::b_component<0>(ulin, r);
        q2::b_component<1>(ulin + 27, r);
        q2::b_component<2>(ulin + 54, r);
        for (int v = 0; v < kNp; ++v) colp[v] = -kScaleB * r[v];
    } else {
        double p[kNp] = {0, 0, 0, 0, 0, 0, 0, 0};
        p[k - kNu] = 1.0;
        double out[kNu];
        for (int n = 0; n < kNu; ++n) out[n] = 0.0;
        q2::bt_component<0>(p, out);
        q2::bt_component<1>(p, out + 27);
        q2::bt_component<2>(p, out + 54);
        for (int n = 0; n < kNu; ++n) col[n] = -kScaleB * out[n];
    }
    bool ok = true;
    auto snap = [&ok](double& v) {
        const double r = double((long long)(v < 0 ? v - 0.5 : v + 0.5));
        if (v - r > 1e-6 || r - v > 1e-6) ok = false;
        v = r;
    };
    for (int n = 0; n < kNu; ++n) snap(col[n]);
    for (int v = 0; v < kNp; ++v) snap(colp[v]);
    return ok;
}

// ---- fixed point and digits
// Exponent of the binade of v (v = m 2^E with 1/2 <= |m| < 1, so |v| < 2^E); zero and FP64
// subnormals give kNoExp (they read as 0 in fixed point).
constexpr int kNoExp = -4096;
__host__ __device__ __forceinline__ int binade(double v) {
    const unsigned long long b = q2::dbl_bits(v);
    const int e = int((b >> 52) & 0x7FFu);
    return e == 0 ? kNoExp : e - 1022;
}

// X = round(v 2^(kFrac - E)) (ties away from zero) for |v| < 2^E, by integer instructions on the
// bits of v: |X| <= 2^54.
__host__ __device__ __forceinline__ long long to_fixed(double v, int E) {
    const unsigned long long b = q2::dbl_bits(v);
    const int e = int((b >> 52) & 0x7FFu);
    if (e == 0) return 0;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // |v| = m 2^(e - 1075)
    const int r = 1075 - kFrac + E - e;   // right shift of m; >= -1 when |v| < 2^E
    unsigned long long X;
    if (r <= 0) X = m << (-r);
    else if (r >= 64) X = 0;
    else X = (m + (1ull << (r - 1))) >> r;
    return (b >> 63) ? -(long long)X : (long long)X;
}

// X = sum_j d[j] 256^j, d[j] in [-128, 127] (balanced digits, lowest first) for |X| <= 2^55.
__host__ __device__ __forceinline__ void digits(long long X, int (&d)[kDigits]) {
#pragma unroll
    for (int j = 0; j < kDigits; ++j) {
        const int dj = int((signed char)(X & 0xFF));
        d[j] = dj;
        X = (X - dj) / 256;   // exact: X - dj is a multiple of 256
    }
}

// The digits of X all at once: Y = X + 0x80808080808080 (>= 0, < 2^56 for |X| <= 2^54) has the
// biased digits d_j + 128 as its bytes. For two values, the f16 bits of 1536 + d_j, packed (first
// value in the low half): 1408 + byte lies in [1024, 2048), where f16 has unit spacing, so its bits
// are 0x6400 + (1408 + byte - 1024) = 0x6580 + byte. One f16 subtraction of 1536 per pair gives the
// digits exactly.
constexpr long long kDigitBias = 0x80808080808080LL;
__host__ __device__ __forceinline__ unsigned long long biased_digits(long long X) {
    return (unsigned long long)(X + kDigitBias);
}
__host__ __device__ __forceinline__ unsigned digit_pair_f16(unsigned long long Y0, unsigned long long Y1, int j) {
    const unsigned b0 = unsigned(Y0 >> (8 * j)) & 0xFFu, b1 = unsigned(Y1 >> (8 * j)) & 0xFFu;
    return (b0 | (b1 << 16)) + 0x65806580u;
}

// ---- recombination of the slice products and the FP64 result
// The slice products arrive lowest digit first. acc <- acc 2^-8 + D (exact scaling, then a two_sum
// of D into the high part), starting from acc = D[0]; after the 7 slices acc = V 2^-48 with
// V = sum_j 256^j D[j]. D integer-valued, |D| < 2^24.
__host__ __device__ __forceinline__ void slice_step(q2::df64& acc, float D, bool first) {
    if (first) {
        acc = q2::df64(D, 0.0f);
        return;
    }
    const float hi = q2::mul_f(acc.hi, 0.00390625f), lo = q2::mul_f(acc.lo, 0.00390625f);
    const float s = q2::add_f(hi, D);
    const float bb = q2::sub_f(s, hi);
    const float e = q2::add_f(q2::sub_f(hi, q2::sub_f(s, bb)), q2::sub_f(D, bb));
    acc = q2::fast_two_sum(s, q2::add_f(lo, e));
}
constexpr int kCombineShift = 48;   // combine() returns V 2^-48
__host__ __device__ __forceinline__ q2::df64 combine(const float (&D)[kDigits]) {
    q2::df64 acc;
#pragma unroll
    for (int j = 0; j < kDigits; ++j) slice_step(acc, D[j], j == 0);
    return acc;
}

// The pressure rows take u's digits against the exponent of the whole input x; when x's largest
// magnitude exceeds u's by more than 2^kMaxGap, the cell's B u is formed from u directly with the
// sum-factorised double-float moments (R u, without the factor -h^2).
constexpr int kMaxGap = 8;
__host__ __device__ __forceinline__ void bu_moments(const q2::df64 (&u)[kNu], q2::df64 (&out)[kNp]) {
    for (int v = 0; v < kNp; ++v) out[v] = q2::df64();
    q2::b_component<0>(u, out);
    q2::b_component<1>(u + 27, out);
    q2::b_component<2>(u + 54, out);
}

__host__ __device__ __forceinline__ int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}
__host__ __device__ __forceinline__ unsigned flt_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    unsigned u;
    __builtin_memcpy(&u, &f, sizeof u);
    return u;
#endif
}
__host__ __device__ __forceinline__ double dbl_from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    __builtin_memcpy(&d, &b, sizeof d);
    return d;
#endif
}

// The FP64 value (double(v.hi) + double(v.lo)) 2^shift rounded to nearest even, as FP64 arithmetic
// would give it, with integer instructions: v.hi's 24-bit significand and v.lo aligned below it in
// a 64-bit integer with 8 guard bits and a sticky bit, one add, one rounding. Needs a normalised
// pair (|v.lo| <= ulp(v.hi) / 2, as fast_two_sum leaves it); zero, subnormal floats and results
// outside the normal FP64 range take the FP64 instructions instead.
__host__ __device__ __forceinline__ double compose(q2::df64 v, int shift) {
    const unsigned bh = flt_bits(v.hi), bl = flt_bits(v.lo);
    const int eh = int((bh >> 23) & 0xFFu), el = int((bl >> 23) & 0xFFu);
    constexpr int G = 8;
    if (eh != 0 && eh != 255 && el != 255 && (el != 0 || (bl & 0x7FFFFFFFu) == 0)) {
        const unsigned long long H = (unsigned long long)((bh & 0x7FFFFFu) | 0x800000u) << (29 + G);
        unsigned long long L = 0;
        if (el != 0) {
            const unsigned long long ml = (bl & 0x7FFFFFu) | 0x800000u;
            const int s = el - eh + 29 + G;   // lo's significand position in H's units
            if (s >= 0) L = ml << s;   // s <= G + 5: |lo| <= ulp(hi) / 2
            else if (s > -64) L = (ml >> (-s)) | ((ml & ((1ull << (-s)) - 1)) != 0 ? 1ull : 0ull);
            else L = 1;   // sticky only
        }
        const bool same = ((bh ^ bl) >> 31) == 0 || L == 0;
        const unsigned long long S = same ? H + L : H - L;   // > 0: |lo| < |hi|
        const int nb = 64 - clz64(S);                         // 60..62 bits
        const int r = nb - 53;                                // >= 7
        unsigned long long q = S >> r;
        const unsigned long long rem = S & ((1ull << r) - 1), half = 1ull << (r - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
        int ebias = eh - 127 - 52 - G + r + 52 + 1023 + shift;   // biased exponent of q's leading bit
        if (q == (1ull << 53)) {
            q >>= 1;
            ++ebias;
        }
        if (ebias >= 1 && ebias <= 2046)
            return dbl_from_bits((unsigned long long)(bh >> 31) << 63 | (unsigned long long)ebias << 52 |
                                 (q & 0xFFFFFFFFFFFFFull));
    }
    // rare: zero, subnormal or non-finite parts, or a result outside the normal range
    double r = double(v.hi) + double(v.lo);
    if (r == 0.0) return r;
    while (shift > 0) { const int s = shift > 1000 ? 1000 : shift; r *= dbl_from_bits((unsigned long long)(1023 + s) << 52); shift -= s; }
    while (shift < 0) { const int s = -shift > 1000 ? 1000 : -shift; r *= dbl_from_bits((unsigned long long)(1023 - s) << 52); shift += s; }
    return r;
}

}  // namespace sliced
}  // namespace stk
