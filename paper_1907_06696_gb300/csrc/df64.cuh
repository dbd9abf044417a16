// df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two floats (|lo| <= ulp(hi)/2), about 48 significant bits.
//
// Used for the FP64-accuracy outer Stokes operator: GB300 executes FP32 FMAs
// at 72x its FP64 rate, and a double-float multiply-add costs ~18 FP32
// instructions, so the operator runs several times faster than in native
// FP64 while its rounding error (~2^-44 relative per operation) stays far
// below the 1e-12 parity bound against the FP64 oracle.
//
// Error-free transformations (published methods):
//   two_sum (Knuth, TAOCP vol. 2, 4.2.2): s = a + b exactly as s + e;
//   fast_two_sum (Dekker 1971): the same when |a| >= |b|;
//   two_prod with FMA: p = a * b exactly as p + fma(a, b, -p).
// add() is the "sloppy" double-float sum (one two_sum on the high parts,
// the low parts added in float), mul() the FMA-based double-float product
// (T. J. Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18 (1971); Y. Hida, X. S. Li, D. H. Bailey,
// "Algorithms for quad-double precision floating point arithmetic", 2001).
#pragma once

#include <cuda_runtime.h>

namespace q2 {

struct df64 {
    float hi, lo;
    __host__ __device__ constexpr df64() : hi(0.0f), lo(0.0f) {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // rounds a double to the nearest double-float (exact for the constants used here to ~2^-48)
    __host__ __device__ constexpr df64(double v) : hi(float(v)), lo(float(v - double(float(v)))) {}
    __host__ __device__ constexpr df64(int v) : hi(float(v)), lo(0.0f) {}
    __host__ __device__ double to_double() const { return double(hi) + double(lo); }
};

// Rounded float operations that the compiler must not contract into FMAs
// (a contracted product would break the error-free transformations).
// Host builds of this header must use -ffp-contract=off.
__host__ __device__ __forceinline__ float fma_f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return __builtin_fmaf(a, b, c);
#endif
}
__host__ __device__ __forceinline__ float add_f(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ float sub_f(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ __forceinline__ float mul_f(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

__host__ __device__ __forceinline__ df64 fast_two_sum(float a, float b) {
    const float s = add_f(a, b);
    return df64(s, sub_f(b, sub_f(s, a)));
}

__host__ __device__ __forceinline__ df64 operator+(const df64& x, const df64& y) {
    const float s = add_f(x.hi, y.hi);
    const float bb = sub_f(s, x.hi);
    float e = add_f(sub_f(x.hi, sub_f(s, bb)), sub_f(y.hi, bb));
    e = add_f(e, add_f(x.lo, y.lo));
    return fast_two_sum(s, e);
}

__host__ __device__ __forceinline__ df64 operator-(const df64& x) { return df64(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ df64 operator-(const df64& x, const df64& y) { return x + (-y); }

__host__ __device__ __forceinline__ df64 operator*(const df64& x, const df64& y) {
    const float p = mul_f(x.hi, y.hi);
    float e = fma_f(x.hi, y.hi, -p);
    e = fma_f(x.hi, y.lo, e);
    e = fma_f(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ df64& operator+=(df64& x, const df64& y) { return x = x + y; }
__host__ __device__ __forceinline__ df64& operator*=(df64& x, const df64& y) { return x = x * y; }

// c0 x0 + c1 x1 + c2 x2 (+ acc) with one final renormalisation: the exact products'
// high parts are summed with two_sum, every rounding error and low part is collected
// in one float and added at the end (the accurate dot-product scheme of Ogita, Rump
// and Oishi, SIAM J. Sci. Comput. 26 (2005), applied to double-float operands).
__host__ __device__ __forceinline__ void two_sum_acc(float& s, float b, float& err) {
    const float t = add_f(s, b);
    const float bb = sub_f(t, s);
    err = add_f(err, add_f(sub_f(s, sub_f(t, bb)), sub_f(b, bb)));
    s = t;
}
__host__ __device__ __forceinline__ float prod_err(const df64& c, const df64& x, float p) {
    float e = fma_f(c.hi, x.hi, -p);
    e = fma_f(c.hi, x.lo, e);
    return fma_f(c.lo, x.hi, e);
}
__host__ __device__ __forceinline__ df64 dot3(const df64& c0, const df64& x0, const df64& c1, const df64& x1,
                                             const df64& c2, const df64& x2) {
    const float p0 = mul_f(c0.hi, x0.hi), p1 = mul_f(c1.hi, x1.hi), p2 = mul_f(c2.hi, x2.hi);
    float err = add_f(add_f(prod_err(c0, x0, p0), prod_err(c1, x1, p1)), prod_err(c2, x2, p2));
    float s = p0;
    two_sum_acc(s, p1, err);
    two_sum_acc(s, p2, err);
    return fast_two_sum(s, err);
}
__host__ __device__ __forceinline__ df64 dot3_acc(const df64& acc, const df64& c0, const df64& x0, const df64& c1,
                                                 const df64& x1, const df64& c2, const df64& x2) {
    const float p0 = mul_f(c0.hi, x0.hi), p1 = mul_f(c1.hi, x1.hi), p2 = mul_f(c2.hi, x2.hi);
    float err = add_f(add_f(add_f(prod_err(c0, x0, p0), prod_err(c1, x1, p1)), prod_err(c2, x2, p2)), acc.lo);
    float s = acc.hi;
    two_sum_acc(s, p0, err);
    two_sum_acc(s, p1, err);
    two_sum_acc(s, p2, err);
    return fast_two_sum(s, err);
}

// Exact split of a double into a double-float (rounding of the low part only).
__host__ __device__ __forceinline__ df64 from_double(double v) {
    const float h = float(v);
    return df64(h, float(v - double(h)));
}

// Split of a double into a double-float with integer and FP32 instructions only (no FP64
// instruction, whose throughput is the bottleneck of FP64 vector kernels on this GPU).
// For 2^-97 <= |v| < 2^128: hi = v's sign, exponent and the leading 24 significand bits
// (truncated); lo = the next 23 bits rounded to nearest, as (1 + R 2^-23) - 1 scaled by a power
// of two (both steps exact). |v - (hi + lo)| <= 2^-47 |v|. Zero and FP64 subnormals give 0;
// other magnitudes take the conversion path (from_double).
__host__ __device__ __forceinline__ unsigned long long dbl_bits(double v) {
#ifdef __CUDA_ARCH__
    return static_cast<unsigned long long>(__double_as_longlong(v));
#else
    unsigned long long b;
    __builtin_memcpy(&b, &v, sizeof b);
    return b;
#endif
}
__host__ __device__ __forceinline__ float flt_from_bits(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    __builtin_memcpy(&f, &u, sizeof f);
    return f;
#endif
}
__host__ __device__ __forceinline__ df64 split_double(double v) {
    const unsigned long long b = dbl_bits(v);
    const unsigned H = unsigned(b >> 32), L = unsigned(b);
    const unsigned e = (H >> 20) & 0x7FFu;
    const unsigned sign = H & 0x80000000u;
    if (e - 926u <= 224u) {
        const float hi = flt_from_bits(sign | ((e - 896u) << 23) | ((H & 0xFFFFFu) << 3) | (L >> 29));
        const unsigned R = ((L & 0x1FFFFFFFu) + 32u) >> 6;   // <= 2^23
        const float t = sub_f(flt_from_bits(0x3F800000u + R), 1.0f);
        const float lo = mul_f(t, flt_from_bits((e - 919u) << 23));
        return df64(hi, sign ? -lo : lo);
    }
    if (e == 0u) return df64(0.0f, 0.0f);
    return from_double(v);
}

// acc += a * b: the exact product (two_prod by FMA plus the cross terms) is added to acc.hi
// by two_sum, and the rounding errors are collected in acc.lo without renormalising; call
// renorm() every few terms so that |acc.lo| stays near ulp(acc.hi) (Ogita-Rump-Oishi Dot2
// with periodic renormalisation).
__host__ __device__ __forceinline__ void mac(df64& acc, const df64& a, const df64& b) {
    const float p = mul_f(a.hi, b.hi);
    const float ep = prod_err(a, b, p);
    const float s = add_f(acc.hi, p);
    const float bb = sub_f(s, acc.hi);
    const float e = add_f(sub_f(acc.hi, sub_f(s, bb)), sub_f(p, bb));
    acc = df64(s, add_f(acc.lo, add_f(ep, e)));
}
__host__ __device__ __forceinline__ void renorm(df64& acc) { acc = fast_two_sum(acc.hi, acc.lo); }

}  // namespace q2
