// outer.cu -- launcher of the component-split double-float outer Stokes blocks (outer.cuh).
#include "internal.cuh"
#include "outer.cuh"
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

template <bool DO_A, bool DO_BT, bool DO_B>
__global__ void __launch_bounds__(kOuterThreads, 2) k_outer_df64(OuterArgs a) {
    __shared__ OuterShared sh;
    const int c = threadIdx.x / kOuterCells, g = threadIdx.x % kOuterCells;
    q2::df64 U[27], W[27];
    if (c == 0) outer_phase1<0, DO_A, DO_B>(a, blockIdx.x, g, sh, U, W);
    else if (c == 1) outer_phase1<1, DO_A, DO_B>(a, blockIdx.x, g, sh, U, W);
    else outer_phase1<2, DO_A, DO_B>(a, blockIdx.x, g, sh, U, W);
    __syncthreads();
    if (c == 0) outer_phase2<0, DO_A, DO_BT>(a, blockIdx.x, g, sh, W);
    else if (c == 1) outer_phase2<1, DO_A, DO_BT>(a, blockIdx.x, g, sh, W);
    else outer_phase2<2, DO_A, DO_BT>(a, blockIdx.x, g, sh, W);
}

}  // namespace

cudaError_t launch_outer_df64(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                              double* dst_u, double* dst_p, bool do_a, bool do_bt, bool do_b, cudaStream_t s) {
    OuterArgs a{g.n, g.M, g.nodes, g.h, mu, src_u, src_p, dst_u, dst_p};
    const unsigned nb = unsigned((g.cells + kOuterCells - 1) / kOuterCells);
    if (do_a && do_bt && do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_outer_df64<true, true, true><<<nb, kOuterThreads, 0, s>>>(a)));
    else if (do_a && !do_bt && !do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_outer_df64<true, false, false><<<nb, kOuterThreads, 0, s>>>(a)));
    else if (!do_a && do_bt && !do_b)
        LAUNCH(PROF_BT_F64, s, (k_outer_df64<false, true, false><<<nb, kOuterThreads, 0, s>>>(a)));
    else if (!do_a && !do_bt && do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_outer_df64<false, false, true><<<nb, kOuterThreads, 0, s>>>(a)));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace stk
