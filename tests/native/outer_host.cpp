// Host run of the double-float outer Stokes kernel (csrc/outer.cuh): the phase functions are
// plain functions of the thread index, so one CTA is emulated by running phase 1 for its 96
// threads, then phase 1b, then phase 2 (the two barriers of the kernel), with the atomic adds as
// plain adds. Boundary rows get the identity afterwards, as in launch_stokes_blocks. Test
// support only: tests/test_outer_host.py builds this file with the host compiler and compares
// the result with the oracle's Stokes operator.
#include <cstddef>
#include <vector>

#include "outer.cuh"

extern "C" int outer_apply_host(int n, const double* mu, const double* src_u, const double* src_p, double* dst_u,
                                double* dst_p) {
    using namespace stk;
    const int M = 2 * n + 1;
    const size_t nodes = size_t(M) * M * M, np = size_t(n + 1) * (n + 1) * (n + 1), cells = size_t(n) * n * n;
    for (size_t i = 0; i < 3 * nodes; ++i) dst_u[i] = 0.0;
    for (size_t i = 0; i < np; ++i) dst_p[i] = 0.0;
    OuterArgs a{n, M, nodes, 1.0 / n, mu, src_u, src_p, dst_u, dst_p};
    std::vector<OuterShared> sh(1);
    static q2::df64 T2[kOuterThreads][27];
    const int blocks = int((cells + kOuterCells - 1) / kOuterCells);
    for (int b = 0; b < blocks; ++b) {
        for (int t = 0; t < kOuterThreads; ++t) {
            q2::df64 U[27];
            outer_phase1<true, true>(a, t / kOuterCells, b, t % kOuterCells, sh[0], U, T2[t]);
        }
        for (int t = 0; t < kOuterThreads; ++t) outer_phase1b<true>(a, t / kOuterCells, b, t % kOuterCells, sh[0], T2[t]);
        for (int t = 0; t < kOuterThreads; ++t) {
            q2::df64 W[27];
            outer_phase2<true, true>(a, t / kOuterCells, b, t % kOuterCells, sh[0], W);
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
