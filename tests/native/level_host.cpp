// Host run of the V-cycle level operator's cell computation (csrc/brick.cuh, brick_compute with a
// one-cell brick, as k_cell_atomic uses it): gather with constrained entries read as 0, the
// sum-factorised cell operator, the mu h scaling, then the kernel's scatter rule (no adds into
// boundary rows) and identity rows. Test support only: tests/test_outer_host.py builds this file
// with the host compiler and compares the result with the oracle's A in FP64 and FP32.
#include <cstddef>

#include "brick.cuh"

template <typename T>
static void level_apply(int n, const T* mu, const T* src, T* dst) {
    using namespace stk;
    const int M = 2 * n + 1;
    const size_t nodes = size_t(M) * M * M;
    BrickArgs<T> a{};
    a.n = n;
    a.M = M;
    a.nodes = nodes;
    a.h = T(1.0 / n);
    a.mu = mu;
    a.src = src;
    for (size_t i = 0; i < 3 * nodes; ++i) dst[i] = T(0);
    for (int ck = 0; ck < n; ++ck)
        for (int cj = 0; cj < n; ++cj)
            for (int ci = 0; ci < n; ++ci) {
                T w[3][27];
                if (!brick_compute<T, 1, 1, 1>(a, ci, cj, ck, 0, w)) continue;
                for (int k = 0; k < 3; ++k)
                    for (int j = 0; j < 3; ++j)
                        for (int i = 0; i < 3; ++i) {
                            const int gi = 2 * ci + i, gj = 2 * cj + j, gk = 2 * ck + k;
                            if (gi == 0 || gj == 0 || gk == 0 || gi == M - 1 || gj == M - 1 || gk == M - 1) continue;
                            const size_t node = size_t(gi) + size_t(M) * (gj + size_t(M) * gk);
                            for (int c = 0; c < 3; ++c) dst[c * nodes + node] += w[c][i + 3 * j + 9 * k];
                        }
            }
    for (int k = 0; k < M; ++k)
        for (int j = 0; j < M; ++j)
            for (int i = 0; i < M; ++i)
                if (i == 0 || j == 0 || k == 0 || i == M - 1 || j == M - 1 || k == M - 1) {
                    const size_t node = size_t(i) + size_t(M) * (j + size_t(M) * k);
                    for (int c = 0; c < 3; ++c) dst[c * nodes + node] = src[c * nodes + node];
                }
}

extern "C" int level_apply_f64(int n, const double* mu, const double* src, double* dst) {
    level_apply<double>(n, mu, src, dst);
    return 0;
}
extern "C" int level_apply_f32(int n, const float* mu, const float* src, float* dst) {
    level_apply<float>(n, mu, src, dst);
    return 0;
}
