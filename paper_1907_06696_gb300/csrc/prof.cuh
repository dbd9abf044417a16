// prof.cuh -- optional per-kernel-class timing with CUDA events, and a count
// of every kernel launch the library issues. Off by default; enabled through
// stokes_profile(). Classes are listed in include/stokes.h.
#pragma once

#include <cuda_runtime.h>

namespace stk {

enum ProfClass {
    PROF_VMULT_F32 = 0,   // velocity cell kernel, FP32
    PROF_VMULT_F64 = 1,   // velocity cell kernel, FP64
    PROF_STOKES_F64 = 2,  // fused A + B^T + B cell kernel (outer operator)
    PROF_BT_F64 = 3,      // B^T cell kernel (preconditioner)
    PROF_MASS_P = 4,      // pressure mass cell kernel
    PROF_TRANSFER = 5,    // prolongation / restriction
    PROF_SMOOTH_VEC = 6,  // Chebyshev updates, residuals, boundary copies, memsets of level vectors
    PROF_KRYLOV = 7,      // multi-dot, multi-axpy, axpby, norms
    PROF_COARSE = 8,      // coarse solve
    PROF_CAST = 9,        // precision casts
    PROF_RESID_F64 = 10,  // outer operator for the solvers' restart and final residuals (native FP64)
    PROF_NCLASS = 11
};

// Called around each launch; cheap no-ops unless profiling is enabled.
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s);
void prof_count(int launches);
// Launches of this host thread are recorded under class cls instead of their own while cls >= 0.
void prof_override(int cls);
bool prof_enabled();
long long launch_total();

}  // namespace stk
