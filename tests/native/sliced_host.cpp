// Host run of the digit-sliced outer Stokes operator (csrc/sliced.cuh): the integer tables, the
// fixed-point digits of each cell's inputs, the slice products (exact integer dot products, which
// is what a tensor-core MMA with f16 digits and FP32 accumulation computes for these magnitudes),
// the recombination and the FP64 result, cell by cell, added into the outputs; boundary rows get
// the identity, as in the outer operator's launch. Also the single steps (fixed point, digits,
// compose) for the arithmetic tests. Test support only: tests/test_sliced_host.py builds this file
// with the host compiler and compares the results with exact arithmetic and with the oracle.
#include <cstddef>

#include "sliced.cuh"

using namespace stk::sliced;

extern "C" int sliced_tables_host(double* KX, double* KU) {   // KX: 81 x 89, KU: 8 x 81, row-major
    bool ok = true;
    for (int k = 0; k < kNx; ++k) {
        double col[kNu], colp[kNp];
        ok = table_column(k, col, colp) && ok;
        for (int n = 0; n < kNu; ++n) KX[n * kNx + k] = col[n];
        if (k < kNu)
            for (int v = 0; v < kNp; ++v) KU[v * kNu + k] = colp[v];
    }
    return ok ? 0 : 1;
}

extern "C" long long to_fixed_host(double v, int E) { return to_fixed(v, E); }
extern "C" int binade_host(double v) { return binade(v); }
extern "C" void digits_host(long long X, int* d) {
    int t[kDigits];
    digits(X, t);
    for (int j = 0; j < kDigits; ++j) d[j] = t[j];
}
extern "C" void digit_pairs_host(long long X0, long long X1, unsigned* bits) {   // bits[kDigits]
    const unsigned long long Y0 = biased_digits(X0), Y1 = biased_digits(X1);
    for (int j = 0; j < kDigits; ++j) bits[j] = digit_pair_f16(Y0, Y1, j);
}
extern "C" void combine_host(const float* D, float* hilo) {
    float t[kDigits];
    for (int j = 0; j < kDigits; ++j) t[j] = D[j];
    const q2::df64 v = combine(t);
    hilo[0] = v.hi;
    hilo[1] = v.lo;
}
extern "C" void compose_host(int count, const float* hi, const float* lo, const int* shift, double* out) {
    for (int i = 0; i < count; ++i) out[i] = compose(q2::df64(hi[i], lo[i]), shift[i]);
}

// D[j][n] = sum_k K[n][k] d[j][k] as exact integers (|partial sums| < 2^24 by the table bound).
template <int N, int K, int KD>
static void slice_products(const double* T, const int (&d)[KD][kDigits], float (&D)[N][kDigits]) {
    for (int n = 0; n < N; ++n)
        for (int j = 0; j < kDigits; ++j) {
            long long s = 0;
            for (int k = 0; k < K; ++k) s += (long long)T[n * K + k] * d[k][j];
            D[n][j] = float(s);
        }
}

extern "C" int sliced_apply_host(int n, const double* mu, const double* src_u, const double* src_p, double* dst_u,
                                 double* dst_p) {
    static double KX[kNu * kNx], KU[kNp * kNu];
    if (sliced_tables_host(KX, KU) != 0) return 1;
    const int M = 2 * n + 1, P = n + 1;
    const size_t nodes = size_t(M) * M * M, np = size_t(P) * P * P;
    const double h = 1.0 / n;
    for (size_t i = 0; i < 3 * nodes; ++i) dst_u[i] = 0.0;
    for (size_t i = 0; i < np; ++i) dst_p[i] = 0.0;
    for (int ck = 0; ck < n; ++ck)
        for (int cj = 0; cj < n; ++cj)
            for (int ci = 0; ci < n; ++ci) {
                const double m = mu[size_t(ci) + size_t(n) * (cj + size_t(n) * ck)];
                size_t dof[kNu], vtx[kNp];
                double x[kNx];
                for (int c = 0; c < 3; ++c)
                    for (int a = 0; a < 27; ++a) {
                        const int i = 2 * ci + a % 3, j = 2 * cj + (a / 3) % 3, k = 2 * ck + a / 9;
                        const bool bnd = i == 0 || j == 0 || k == 0 || i == M - 1 || j == M - 1 || k == M - 1;
                        dof[27 * c + a] = size_t(c) * nodes + size_t(i) + size_t(M) * (j + size_t(M) * k);
                        x[27 * c + a] = bnd ? 0.0 : src_u[dof[27 * c + a]];
                    }
                const double ps = 25.0 * h / m;
                for (int v = 0; v < kNp; ++v) {
                    vtx[v] = size_t(ci + (v & 1)) + size_t(P) * (cj + ((v >> 1) & 1) + size_t(P) * (ck + (v >> 2)));
                    x[kNu + v] = ps * src_p[vtx[v]];
                }
                // one digit set against x's largest magnitude; the pressure rows of the same
                // products, or the double-float moments where x exceeds u by more than 2^kMaxGap
                int Ex = kNoExp, Eu = kNoExp;
                for (int k = 0; k < kNx; ++k) {
                    const int b = binade(x[k]);
                    Ex = b > Ex ? b : Ex;
                    if (k < kNu) Eu = b > Eu ? b : Eu;
                }
                if (Ex == kNoExp) continue;
                static int dx[kNx][kDigits];
                for (int k = 0; k < kNx; ++k) digits(to_fixed(x[k], Ex), dx[k]);
                static float DX[kNu][kDigits], DU[kNp][kDigits];
                slice_products<kNu, kNx>(KX, dx, DX);
                slice_products<kNp, kNu>(KU, dx, DU);   // the first 81 digit rows: u's
                const q2::df64 sA = q2::split_double(m * h / kScaleA), sB = q2::split_double(h * h / kScaleB);
                const int shift = Ex - kFrac + kCombineShift;
                for (int r = 0; r < kNu; ++r) dst_u[dof[r]] += compose(combine(DX[r]) * sA, shift);
                if (Eu != kNoExp && Ex - Eu > kMaxGap) {
                    q2::df64 ud[kNu], bu[kNp];
                    for (int k = 0; k < kNu; ++k) ud[k] = q2::split_double(x[k]);
                    bu_moments(ud, bu);
                    for (int v = 0; v < kNp; ++v) dst_p[vtx[v]] += -h * h * bu[v].to_double();
                } else {
                    for (int v = 0; v < kNp; ++v) dst_p[vtx[v]] += compose(combine(DU[v]) * sB, shift);
                }
            }
    for (int k = 0; k < M; ++k)
        for (int j = 0; j < M; ++j)
            for (int i = 0; i < M; ++i)
                if (i == 0 || j == 0 || k == 0 || i == M - 1 || j == M - 1 || k == M - 1) {
                    const size_t node = size_t(i) + size_t(M) * (j + size_t(M) * k);
                    for (int c = 0; c < 3; ++c) dst_u[c * nodes + node] = src_u[c * nodes + node];
                }
    return 0;
}
