// batch.cuh -- the FP32 V-cycle of many independent problems in one persistent launch.
//
// Every problem keeps its own level hierarchy (uniform n^3 meshes of any size and level count);
// one cooperative kernel runs the V-cycle of Section 2.2.1 (Jacobi-Chebyshev smoothing of a given
// degree, residual, restriction, exact coarse solve, prolongation, post-smoothing) for all active
// problems at once. The recursion is laid out as a fixed list of phases by depth below each
// problem's finest level (depth d acts on level L_p - 1 - d of problem p, so problems with fewer
// levels reach their coarse solve earlier and idle at the deeper depths); consecutive phases are
// separated by a grid barrier. Within a phase the blocks take work items (problem, tile of cells
// or nodes) from a device work queue (one atomic counter per phase); problems whose mask entry is
// 0 (converged) are skipped. Grid barriers are bounded by %globaltimer: a barrier that runs out
// records STOKES_TIMEOUT in the status word and every block leaves the kernel.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace stk {

constexpr int kBatchMaxLevels = 12;
constexpr int kBatchMaxDegree = 8;

// One level of one problem: geometry, FP32 level vectors, Chebyshev coefficients of step k
// (d <- c1[k] d + c2[k] D^-1 (b - A x); step 0 of the zero-guess smoothing uses no operator).
struct BatchLevel {
    int n, M;
    size_t nodes, n_u;
    float h;
    const float* mu;
    const float* dinv;
    float *b, *x, *r, *d, *acc;
    float c1[kBatchMaxDegree], c2[kBatchMaxDegree];
};

struct BatchProblem {
    int L;                               // levels, index 0 = coarsest
    int nf;                              // free DoFs of the coarsest level
    const int* free_idx;                 // their indices in the coarsest level vector
    const double* Ainv;                  // dense inverse of the coarsest free block (FP64)
    BatchLevel lev[kBatchMaxLevels];
};

enum BatchOp {
    BOP_ZERO = 0,          // coarsest x = 0
    BOP_COARSE = 1,        // coarsest x[free] = Ainv b[free] (one warp per row)
    BOP_CHEB0 = 2,         // first smoothing step with zero guess: d = c2[0] D^-1 b, x = d
    BOP_LEVELOP = 3,       // acc += A x (one thread per cell, atomic adds)
    BOP_CONSUME_CHEB = 4,  // d = c1[k] d + c2[k] D^-1 (b - acc), x += d, acc = 0
    BOP_CONSUME_RESID = 5, // r = b - acc, acc = 0
    BOP_RESTRICT = 6,      // b_{l-1} = P^T r_l (one thread per coarse node)
    BOP_PROLONG = 7        // x_l += P x_{l-1} (one thread per fine node)
};

struct BatchPhase {
    int op, depth, k;
};

// Schedule of one V-cycle for problems with the given level counts and smoother degree.
int batch_build_phases(const int* levels, int n_problems, int degree, BatchPhase* out, int capacity);
// Work items of phase ph for problem p (0 if the problem has no part in it).
size_t batch_items(const BatchProblem& p, const BatchPhase& ph);

struct BatchLaunch {
    const BatchProblem* problems;   // device, n_problems
    int n_problems;
    const BatchPhase* phases;       // device, n_phases
    int n_phases;
    const unsigned* tile_prefix;    // device, n_phases x (n_problems + 1): first tile of each problem
    unsigned* counters;             // device, n_phases + 2 (work-queue counters, barrier count and generation)
    const int* active;              // device, n_problems (0 = skip)
    unsigned* status;               // device status word (bit 1: a grid barrier gave up)
    unsigned long long wait_ns;     // bound of each grid-barrier wait
};

constexpr int kBatchThreads = 384;   // threads per block

// Work items per thread in one tile of a phase (a tile = kBatchThreads x this many items): one
// cell for the operator and one warp-row for the coarse solve, more for the light vector passes.
__host__ __device__ constexpr int batch_items_per_thread(int op) {
    return op == BOP_LEVELOP || op == BOP_COARSE ? 1 : (op == BOP_RESTRICT || op == BOP_PROLONG ? 4 : 16);
}

// Most blocks the cooperative launch can keep resident; 0 if the device cannot run it.
int batch_grid_blocks();
// One V-cycle of the batch with `blocks` blocks (clamped to 1..batch_grid_blocks()).
cudaError_t launch_batch_vcycle(const BatchLaunch& bl, int blocks, cudaStream_t s);

}  // namespace stk
