// Host run of the pressure-side gathers of the preconditioner (csrc/pressure.cuh): B^T p line by
// line as k_bt_gather runs it (weights, then t_e for every vertex of the line, then the line's
// nodes), and one S_hat^-1 Chebyshev step vertex by vertex as k_schur_cheb runs it. Test support
// only: tests/test_kernels_host.py builds this file with the host compiler and compares the
// results with the oracle's B^T and M_p.
#include <cstddef>
#include <vector>

#include "pressure.cuh"

template <int C>
static void bt_component(int n, double s, const double* p, double* out) {
    const int P = n + 1, M = 2 * n + 1;
    std::vector<q2::df64> t(P);
    q2::df64 w[9];
    for (int K = 0; K < M; ++K)
        for (int J = 0; J < M; ++J) {
            double* o = out + size_t(C) * size_t(M) * M * M + size_t(M) * (J + size_t(M) * K);
            if (J == 0 || J == M - 1 || K == 0 || K == M - 1) {
                for (int i = 0; i < M; ++i) o[i] = 0.0;
                continue;
            }
            for (int q = 0; q < 9; ++q) w[q] = stk::bt_weight<C>(J, K, q);
            for (int e = 0; e < P; ++e) t[e] = stk::bt_t<C>(n, p, J, K, e, w);
            for (int e = 0; e < P; ++e) stk::bt_out<C>(n, s, o, e, t.data());
        }
}

extern "C" int bt_apply_host(int n, double h, const double* p, double* out) {
    const double s = -h * h;
    bt_component<0>(n, s, p, out);
    bt_component<1>(n, s, p, out);
    bt_component<2>(n, s, p, out);
    return 0;
}

extern "C" int schur_step_host(int n, const double* scale, const double* r, const double* dinv, const double* z,
                               const double* d, double* z_new, double* d_new, double c1, double c2) {
    const size_t np = size_t(n + 1) * (n + 1) * (n + 1);
    for (size_t v = 0; v < np; ++v) stk::schur_vertex(n, scale, r, dinv, z, d, z_new, d_new, c1, c2, v);
    return 0;
}
