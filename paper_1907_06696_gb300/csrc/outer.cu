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
__global__ void __launch_bounds__(kOuterThreads, 4) k_outer_df64(OuterArgs a) {
    extern __shared__ __align__(16) unsigned char outer_smem[];
    OuterShared& sh = *reinterpret_cast<OuterShared*>(outer_smem);
    const int c = threadIdx.x / kOuterCells, g = threadIdx.x % kOuterCells;
    {
        q2::df64 T2[27];
        {
            q2::df64 U[27];
            outer_phase1<DO_A, DO_B>(a, c, blockIdx.x, g, sh, U, T2);
        }
        __syncthreads();
        outer_phase1b<DO_A>(a, c, blockIdx.x, g, sh, T2);
    }
    __syncthreads();
    q2::df64 W[27];
    outer_phase2<DO_A, DO_BT>(a, c, blockIdx.x, g, sh, W);
}

}  // namespace

cudaError_t launch_outer_df64(const LevelGeom& g, const double* mu, const double* src_u, const double* src_p,
                              double* dst_u, double* dst_p, bool do_a, bool do_bt, bool do_b, cudaStream_t s) {
    OuterArgs a{g.n, g.M, g.nodes, g.h, mu, src_u, src_p, dst_u, dst_p};
    static bool configured = false;
    constexpr int smem = int(sizeof(OuterShared));
    if (!configured) {   // first call happens in set-up or a solve, never inside a stream capture
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_outer_df64<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_outer_df64<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_outer_df64<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_outer_df64<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return e;
        configured = true;
    }
    const unsigned nb = unsigned((g.cells + kOuterCells - 1) / kOuterCells);
    if (do_a && do_bt && do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_outer_df64<true, true, true><<<nb, kOuterThreads, smem, s>>>(a)));
    else if (do_a && !do_bt && !do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_outer_df64<true, false, false><<<nb, kOuterThreads, smem, s>>>(a)));
    else if (!do_a && do_bt && !do_b)
        LAUNCH(PROF_BT_F64, s, (k_outer_df64<false, true, false><<<nb, kOuterThreads, smem, s>>>(a)));
    else if (!do_a && !do_bt && do_b)
        LAUNCH(PROF_STOKES_F64, s, (k_outer_df64<false, false, true><<<nb, kOuterThreads, smem, s>>>(a)));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace stk
