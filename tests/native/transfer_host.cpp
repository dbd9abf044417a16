// Host run of the cell-wise level transfers (csrc/transfer.cuh): prolongation plane by plane and
// restriction cell by cell, over every (component, plane, cell) k_prolong_cells and
// k_restrict_cells launch a thread for. Test support only: tests/test_kernels_host.py builds this
// file with the host compiler and compares the results with the oracle's P and P^T.
#include <cstddef>

#include "transfer.cuh"

template <typename T>
static void prolong(int nc, const T* coarse, T* fine, int add) {
    const size_t ncell = size_t(nc) * nc * nc;
    for (int c = 0; c < 3; ++c)
        for (int z = 0; z < 5; ++z)
            for (size_t cell = 0; cell < ncell; ++cell) stk::prolong_cell_plane<T>(nc, coarse, fine, add != 0, c, z, cell);
}

template <typename T>
static void restrict_(int nc, const T* fine, T* coarse) {
    const size_t Mc = size_t(2 * nc + 1);
    for (size_t i = 0; i < 3 * Mc * Mc * Mc; ++i) coarse[i] = T(0);
    const size_t ncell = size_t(nc) * nc * nc;
    for (int c = 0; c < 3; ++c)
        for (size_t cell = 0; cell < ncell; ++cell) stk::restrict_cell<T>(nc, fine, coarse, c, cell);
}

extern "C" int prolong_host_f64(int nc, const double* coarse, double* fine, int add) {
    prolong<double>(nc, coarse, fine, add);
    return 0;
}
extern "C" int prolong_host_f32(int nc, const float* coarse, float* fine, int add) {
    prolong<float>(nc, coarse, fine, add);
    return 0;
}
extern "C" int restrict_host_f64(int nc, const double* fine, double* coarse) {
    restrict_<double>(nc, fine, coarse);
    return 0;
}
extern "C" int restrict_host_f32(int nc, const float* fine, float* coarse) {
    restrict_<float>(nc, fine, coarse);
    return 0;
}
