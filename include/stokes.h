/*
 * stokes.h -- C ABI of the GB300 matrix-free GMG Stokes library.
 *
 * Method: Clevenger & Heister, "Comparison between algebraic and matrix-free
 * geometric multigrid for a Stokes problem on adaptive meshes with variable
 * viscosity" (arXiv 1907.06696).
 *   - Stokes problem with variable viscosity and homogeneous Dirichlet
 *     velocity: Section 2, eq. (stokes).
 *   - Taylor-Hood Q2-Q1 on hexahedra and the blocks A, B, B^T, F:
 *     Section 2.1, eq. (stokes_linear_system).
 *   - Block-triangular preconditioner P = [[A, B^T], [0, -S]]:
 *     Section 2.2, eq. (stokes_precond).
 *   - A^-1 ~ one matrix-free GMG V-cycle on the fully coupled A with a
 *     degree-4 Chebyshev smoother, one smoothing step per level: Section 2.2.1.
 *   - S^-1 ~ Chebyshev iteration on the 1/mu-weighted pressure mass matrix,
 *     outer FGMRES: Section 2.2.2.
 *   - Harmonic cell averaging of the viscosity and its Q0 restriction to the
 *     level hierarchy: Section 2.3.
 *   - Sinker benchmark coefficients: Section 3.2.
 *
 * Mesh and vector layout (every entry point):
 *   Uniform n^3 cube cells on [0,1]^3, h = 1/n. Level l (0 = coarsest) has
 *   n_l = n / 2^(L-1-l) cells per axis. Q2 nodes form an M^3 lattice,
 *   M = 2 n_l + 1, node (i,j,k) -> i + M j + M^2 k. A velocity vector is
 *   component-blocked: entry c*M^3 + node, length N_u = 3 M^3 (boundary nodes
 *   included). A pressure vector holds the (n+1)^3 Q1 vertex values,
 *   vertex (i,j,k) -> i + (n+1) j + (n+1)^2 k. A Stokes vector is [u; p],
 *   length N_u + N_p, FP64.
 *   All six walls are no-slip: velocity entries on boundary nodes are
 *   constrained. Every operator IGNORES the constrained entries of its input
 *   (treats them as 0) and acts as the IDENTITY on them in its output, i.e.
 *   the constrained operator is [[A_ff, 0], [0, I]].
 *
 * Memory: every pointer named *_dev is a device pointer owned by the caller
 * (for example a torch tensor's data_ptr()); the library never frees it. The
 * library owns its tables and workspace (allocated in stokes_setup and, for
 * the Krylov basis, on the first stokes_solve; freed by stokes_destroy).
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Calls are asynchronous on that stream unless stated otherwise. One context
 * must not be used from two streams at the same time (its workspace is shared).
 *
 * Errors: every call returns a stokes_status; no C++ exception crosses the
 * ABI. stokes_last_error() gives a message for the calling thread's last error.
 */
#ifndef STOKES_GB300_H
#define STOKES_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stokes_ctx stokes_ctx;

typedef enum {
    STOKES_OK = 0,
    STOKES_EINVAL = 1,          /* bad argument (size, level, precision, null pointer) */
    STOKES_ENOMEM = 2,          /* device or host allocation failed */
    STOKES_ECUDA = 3,           /* a CUDA runtime call or kernel launch failed */
    STOKES_NOT_CONVERGED = 4,   /* a solve ended with its true residual above rtol */
    STOKES_BREAKDOWN = 5,       /* NaN/Inf or a zero Krylov norm in stokes_solve */
    STOKES_TIMEOUT = 6,         /* a bounded wait inside a kernel gave up (options.wait_limit_s) */
    STOKES_EMESH = 7            /* unsupported mesh description */
} stokes_status;

typedef enum { STOKES_FP64 = 0, STOKES_FP32 = 1 } stokes_prec;

typedef enum {
    STOKES_BLOCK_A = 0,         /* u -> A_c u            (N_u -> N_u) */
    STOKES_BLOCK_B = 1,         /* u -> B u              (N_u -> N_p) */
    STOKES_BLOCK_BT = 2,        /* p -> B^T p            (N_p -> N_u, zero on constrained rows) */
    STOKES_BLOCK_MP = 3,        /* p -> M_p p            (N_p -> N_p) */
    STOKES_BLOCK_STOKES = 4     /* [u;p] -> [A_c u + B^T p; B u]  (N_u+N_p -> N_u+N_p) */
} stokes_block;

typedef struct {
    int kind;                   /* 0 = uniform n^3 grid of the unit cube (the only kind) */
    int n;                      /* cells per axis on the finest level, n = c * 2^(n_levels-1), 1 <= c <= 6 */
    int n_levels;               /* multigrid levels, >= 1 */
} stokes_mesh;

typedef struct {
    int kind;                   /* 0 = sinker formula (Section 3.2); 1 = values at quadrature points */
    int n_sinkers;              /* kind 0 */
    const double* centres;      /* kind 0: host, 3*n_sinkers (x,y,z per sinker) */
    double mu_min, mu_max;      /* kind 0: mu = X mu_min + (1 - X) mu_max */
    double delta, omega;        /* kind 0: decay (200) and sinker diameter (0.1) */
    double beta;                /* kind 0: forcing f = (0, 0, beta (X - 1)) (10) */
    const double* mu_q;         /* kind 1: host, n^3 * 27 values; cell-major (cell index
                                   ci + n cj + n^2 ck), then Gauss point qx + 3 qy + 9 qz */
} stokes_mu;

typedef struct {
    uint32_t noslip_faces;      /* bit f = face f is no-slip; must be 0x3F (all walls, eq. stokes) */
} stokes_bc;

typedef struct {
    int cheb_degree;            /* Chebyshev smoother degree per smoothing step (4, Section 2.2.1) */
    double smoothing_range;     /* eigenvalue interval [lam_hi / range, lam_hi] (15) */
    double eig_safety;          /* lam_hi = safety * Lanczos estimate of lambda_max(D^-1 A) (1.2) */
    int lanczos_steps;          /* Lanczos steps for lambda_max (12) */
    int schur_degree;           /* Chebyshev degree of S_hat^-1 on M_p, interval [1/8, 27/8] (5); 0 = S_hat =
                                   diag(M_p) itself (Section 3.4; degree 1 is (4/7) diag(M_p)^-1) */
    int restart;                /* FGMRES restart length (50, Section 3.4) */
    int outer_arith;            /* arithmetic of the FP64-interface outer operator: 0 = native FP64;
                                   1 = double-float (pairs of floats, ~48-bit significand) on the FP32
                                   units for every block (default; GB300's FP64 rate is 1/72 of FP32: the
                                   Stokes block takes 0.83 vs 1.95 ms, B^T alone 0.15 vs 0.22 ms at
                                   64^3). Both match the FP64 oracle to 1e-12.
                                   2 = the whole operator [A B^T; B 0] of uniform meshes on the tensor
                                   cores, exactly: each cell's FP64 inputs in fixed point against their
                                   largest magnitude, split into 7 digit slices of 8 bits, times the
                                   integer element table [[5400 A_ref, -216 R^T], [-216 R, 0]] (f16,
                                   tcgen05.mma with FP32 accumulation, exact because every partial sum
                                   is an integer below 2^24), recombined in double-float and written
                                   as FP64 with integer instructions; every other block and the
                                   Krylov basis as in 1. Not yet the default: its speed is unmeasured. */
    int vmult_kernel;           /* level operator of the V-cycle: 0 = one thread per cell with atomic adds
                                   and a separate epilogue pass (default); 1 = brick-tiled, atomic-free
                                   and deterministic, epilogue fused; 2 = FP32 levels: the brick-tiled
                                   scatter of 1 with the cell products on the tensor cores (A_cell =
                                   mu_c h A_hat with 5400 A_hat exact in f16; each cell's values scaled
                                   by a power of two and split into two f16 terms, 22 significant bits;
                                   f32 accumulation), FP64 levels as 0; 3 = FP32 levels: three
                                   threads per cell, one per output component, cross derivatives
                                   exchanged in shared memory (by default 0 uses it on the FP32
                                   levels of at most 16^3 cells, where a level operator's time is
                                   one thread's serial work), FP64 levels as 0 */
    int graphs;                 /* 1 = capture the V-cycle's level recursion once per precision as a CUDA
                                   graph and replay it on a library stream ordered with the caller's
                                   stream by events (default); 0 = launch kernel by kernel. The first
                                   V-cycle of each precision performs the capture. */
    int precond_kind;           /* 0 = block-triangular P of eq. stokes_precond (default): z_p = -S_hat^-1 r_p,
                                   z_u = A_hat^-1 (r_u - B^T z_p); 1 = block-diagonal P_D = diag(A, S) of
                                   Section 2.2 / Table 1: z_u = A_hat^-1 r_u, z_p = S_hat^-1 r_p */
    int outer_solver;           /* 0 = FGMRES(restart) (default); 1 = IDR(idr_s), the memory-light solver of
                                   Section 3.4 (van Gijzen & Sonneveld's bi-orthogonal IDR(s) with right
                                   preconditioning, 3 idr_s + 4 vectors; shadow space from splitmix64
                                   seeds 1907100 + i, orthonormalised). Not for stokes_batch_solve.
                                   2 = GMRES(restart) with the preconditioner as one fixed linear map
                                   (Section 3.4: the V-cycle and S_hat^-1 are fixed polynomials and an
                                   exact coarse solve): restart + 2 vectors instead of 2 restart + 2; a
                                   cycle ends with x += P^-1 (V y) (one preconditioner application more
                                   per cycle, not counted in iterations) and the solve ends when the
                                   true residual b - K x, recomputed after the cycle, meets rtol.
                                   3 = MINRES (method (ii)(b) of Section 2.2; Paige & Saunders) with
                                   the symmetric positive definite P_D: requires precond_kind = 1
                                   (EINVAL at set-up otherwise); 11 vectors; the 2-norm residual is
                                   carried by the recurrence and checked against b - K x (a drift
                                   restarts MINRES from x, at most 10 times). Not for batches. */
    int idr_s;                  /* shadow-space dimension of IDR(s), 1..8 (2) */
    int gram_schmidt;           /* FGMRES orthogonalisation with the double-float basis (outer_arith 1 or 2,
                                   restart <= 64): 1 = classical Gram-Schmidt twice with the second
                                   projection of each basis vector delayed into the next step, two
                                   passes over the basis per iteration (default: the FGMRES vector
                                   kernels take 20% less time at 64^3 and 96^3, the same iterations);
                                   0 = the same two projections in three passes. Same Krylov space; the preconditioner
                                   receives the once-projected vector. GMRES (outer_solver 2) and the
                                   native FP64 basis always take three passes. */
    double wait_limit_s;        /* bound, in seconds of the GPU's global timer, of every wait inside the
                                   library's kernels (the tensor-core operator's wait for its MMAs; 1.0).
                                   A wait that runs out records STOKES_TIMEOUT in the context's device
                                   status word (see stokes_device_status) and its kernel leaves, with
                                   undefined output; 0 gives up at once (exercises that path). */
    int batch_vcycle;           /* stokes_batch_solve with FP32 V-cycles inside FGMRES: 0 = one captured
                                   V-cycle graph per problem, replayed on the problem's own stream
                                   (default; measured faster); 1 = in a round where at least eight
                                   problems reach their preconditioner, their V-cycles run as one
                                   persistent cooperative launch (work queue of (problem, tile) items
                                   per phase, grid barriers bounded by wait_limit_s, the other problems
                                   masked out), other rounds as 0. Read from the first context of the
                                   batch. */
    int fused_smoother;         /* 1 = each Jacobi-Chebyshev step's vector update is carried by the
                                   next product on the level (the cell and component-split operators,
                                   vmult_kernel 0 and 3): each node's operand x' = x + c1 d + c2
                                   D^-1 (b - A x) is formed where the product gathers it, the owner
                                   cell stores the new (d, x), and the pre-smoothing's last update
                                   rides on its residual's product, so a degree-k smoothing takes k
                                   products and one vector pass instead of k of each; 0 = a separate
                                   vector pass after every product (default: on GB300 the products
                                   are bound by issue and latency, and gathering five vectors at every
                                   node of every cell costs them more than the streaming pass saves:
                                   a degree-4 smoothing at 64^3 takes 374 us fused, 268 us separate).
                                   Same arithmetic. */
} stokes_options;

typedef struct {
    int iterations;             /* Krylov iterations: FGMRES / GMRES Arnoldi steps, IDR(s) preconditioned
                                   operator applications */
    double rel_residual;        /* final recurrence estimate |g_k| / ||b|| */
    double rel_residual_true;   /* ||b - K x|| / ||b|| recomputed in FP64 after the solve */
    double seconds;             /* wall time of the solve on the host clock */
    int status;                 /* the stokes_status returned */
} stokes_solve_info;

/* Fill `opt` with the defaults listed above. */
void stokes_default_options(stokes_options* opt);

/* Build the level hierarchy (Section 2.2.1) for a uniform mesh: per-level cell
 * viscosity (harmonic average of mu at the 27 Gauss points of each finest cell,
 * parent = mean of its 8 children, Section 2.3), inverse diagonals of A_l,
 * Lanczos estimates of lambda_max(D_l^-1 A_l) (start vector: splitmix64 with
 * seed 1907000 + l, value u01 - 1/2 per DoF index, constrained entries 0),
 * the dense FP64 inverse of the coarsest A_0 on its free DoFs, the diagonal of
 * M_p, and the right-hand side F (kind 0 only; F = 0 for kind 1).
 * Synchronous on `stream`. On success *out owns all of it. Errors: EINVAL
 * (null pointer, n or n_levels out of range), EMESH (kind != 0, n not
 * c*2^(L-1) with c <= 6, bc != 0x3F), ENOMEM, ECUDA. */
stokes_status stokes_setup(const stokes_mesh* mesh, const stokes_mu* mu, const stokes_bc* bc,
                           const stokes_options* opt /* NULL = defaults */, void* stream,
                           stokes_ctx** out);

/* ---- Adaptive octree meshes (Abstract; local smoothing by citation in Section 2.2.1) ----
 *
 * A cell of level l (side 2^-l) at integer position (i, j, k), 0 <= i, j, k < 2^l, l <= 15, is
 * the key  l << 48 | k << 32 | j << 16 | i.  Leaves must tile the unit cube and be 2:1
 * balanced across faces, edges and vertices. Points are keyed on the lattice of spacing
 * 2^-(lmax+1) (lmax = finest leaf level): key = x + Mx (y + Mx z), Mx = 2^(lmax+1) + 1.
 *
 * Active space (what stokes_solve, stokes_vmult level -1 and gmg_vcycle act on): the Q2
 * nodes of the leaves that are not hanging, in increasing key order, component-blocked
 * velocity [3][nodes]; the Q1 vertices that are not hanging, in increasing key order. A
 * node of a leaf that lies on a face or edge of a coarser neighbouring leaf, and is not one
 * of its nodes, is hanging: its value is the coarser leaf's Q2 (velocity) or Q1 (pressure)
 * interpolant there, resolved inside the operators. Nodes on the cube boundary are
 * Dirichlet (identity rows, as on uniform meshes).
 *
 * Multigrid levels: index 0 = the uniform grid 2^coarsest_level, index li = refinement
 * level coarsest_level + li, holding every cell of that level (leaf or refined) and its Q2
 * nodes in increasing key order. Nodes on the boundary of those cells' union but inside the
 * cube (refinement edge) are ordinary rows of the level operator and are never smoothed.
 * One V-cycle: the active right-hand side goes to the level of each node's coarsest leaf;
 * down: degree-k Chebyshev smoothing from zero, residual (edge rows included), restriction
 * added to the coarser level; dense FP64 solve on level 0; up: prolongation added on every
 * node, Chebyshev smoothing; each active node takes its value on its level. */
typedef struct {
    int coarsest_level;         /* coarsest multigrid level (uniform), <= every leaf's level; its
                                   free velocity DoFs (dense solve) must number at most 4000 */
    int64_t n_leaves;
    const uint64_t* leaf_keys;  /* host, n_leaves keys (any order) */
} stokes_octree;

/* Leaves of the adaptive sinker mesh: start from the uniform grid 2^base_level; split a leaf
 * while its level is below the maximum level of a sinker (max_levels[s]) and its distance
 * interval [min, max |x - c_s|] over the cell meets (shell_radius - shell_half_width,
 * shell_radius + shell_half_width); then 2:1-balance (faces, edges, vertices). Writes up to
 * `capacity` sorted keys to `keys` (host; may be NULL with capacity 0 to query the count) and
 * the count to *n_leaves. Errors: EINVAL (bad argument, or capacity below the count while
 * keys is given; *n_leaves is set), ENOMEM. */
stokes_status stokes_octree_sinker_mesh(int base_level, int n_sinkers, const double* centres,
                                        const int* max_levels, double shell_radius, double shell_half_width,
                                        uint64_t* keys, int64_t capacity, int64_t* n_leaves);

/* Set up an octree problem: host tables (active DoFs, constraints, levels, copy lists), cell
 * viscosity (leaf: harmonic average over its Gauss points; refined cell: mean of its
 * children, Section 2.3), level diagonals, Lanczos estimates per level li >= 1 (start vector
 * splitmix64 with seed 1907000 + li on the smoothed nodes), the dense inverse of level 0 and
 * the right-hand side. mu must be kind 0. Synchronous. Errors: EINVAL, EMESH (unbalanced or
 * malformed leaves, constraint chains), ENOMEM, ECUDA. The context then serves stokes_size,
 * stokes_vmult, gmg_vcycle, stokes_solve, stokes_solve_host, stokes_get_rhs,
 * stokes_get_viscosity (level -1: leaves), stokes_get_inv_diagonal, stokes_get_lambda_max,
 * stokes_precondition, stokes_schur_inverse and stokes_octree_table; the uniform-only entry
 * points (autotune, batch solve, smooth, transfers, coarse solve) return EMESH. */
stokes_status stokes_setup_octree(const stokes_octree* mesh, const stokes_mu* mu, const stokes_bc* bc,
                                  const stokes_options* opt, void* stream, stokes_ctx** out);

/* Adaptive refinement by a gradient indicator (Section 3.3: each new mesh refines about 1/7 of the
 * cells chosen by a gradient-based estimator, so that the cell count about doubles; the estimator
 * is not specified). Indicator of leaf K of side h: eta_K = h^(5/2) |grad u_h(x_K)|_F, the
 * Frobenius norm of the Q2 velocity's gradient at the leaf centre (there d/dx u is the difference
 * of the two face-centre values over h), the leaf's values taken from the active vector through
 * the hanging-node constraints with Dirichlet values read as 0. The floor(n fraction + 1/2) leaves
 * with the largest eta (equal eta: smaller key first) are split into their 8 children; the result
 * is 2:1 balanced. mesh: the current leaves (any order) and coarsest level; u_host: host, the
 * active velocity [3][active nodes] of that mesh (the first 3 x nodes entries of a stokes_solve
 * result on a context set up from it); fraction in (0, 1] (1/7 in the paper). eta (host, may be
 * NULL): n_leaves indicators in increasing key order. Writes up to `capacity` sorted new keys to
 * `keys` (may be NULL with capacity 0 to query the count) and the count to *n_leaves. Host only,
 * synchronous. Errors: EINVAL (bad argument, non-finite velocity, a leaf beyond level 15, capacity
 * below the count while keys is given; *n_leaves is set), EMESH (leaves not a balanced tiling),
 * ENOMEM. */
stokes_status stokes_octree_refine_gradient(const stokes_octree* mesh, const double* u_host, double fraction,
                                            double* eta, uint64_t* keys, int64_t capacity, int64_t* n_leaves);

/* Host copy of a table of an octree context; returns the entry count (0 for a bad argument)
 * and writes min(count, capacity) entries to `out` (host; may be NULL):
 *   0 leaf keys (uint64)                   1 active velocity node keys (uint64)
 *   2 active pressure vertex keys (uint64) 3 node keys of multigrid level `level` (uint64)
 *   4 node flags of level `level` (uint8: 1 boundary, 2 refinement edge)
 *   5 per active velocity node: the multigrid level index it is copied to (int32)
 *   6 number of hanging velocity nodes, 7 number of hanging pressure vertices (count only) */
size_t stokes_octree_table(const stokes_ctx* ctx, int which, int level, void* out, size_t capacity);

/* Free everything the context owns (synchronises the device first). NULL is a no-op. */
void stokes_destroy(stokes_ctx* ctx);

const char* stokes_strerror(stokes_status s);
/* Message for the calling thread's last failed call ("" if none). */
const char* stokes_last_error(void);

/* Sizes: what = 0 N_u, 1 N_p, 2 cells, 3 cells per axis, 4 number of levels.
 * level -1 = finest. Returns 0 for a bad argument. Octree contexts: level -1 = the active
 * space (N_u, N_p, leaves; what 3 = finest leaf level), level li = multigrid level li
 * (3 * nodes, 0, cells; what 3 = its refinement level). */
size_t stokes_size(const stokes_ctx* ctx, int level, int what);

/* dst = block * src on one level (Section 2.1, eq. stokes_linear_system),
 * matrix-free, sum-factorised on Q2 cells with the level's cell viscosity.
 * level -1 = finest. prec FP32 is available for block A only; the B, B^T,
 * M_p and Stokes blocks are FP64 and finest-level only. src and dst must not
 * overlap. Errors: EINVAL (bad level/block/precision, null pointer), ECUDA.
 * Octree contexts: level -1 is the active space with hanging-node constraints (FP64, all
 * blocks, native FP64 arithmetic); level li >= 0 is multigrid level li (block A, FP32 or
 * FP64; refinement-edge rows are ordinary rows). */
stokes_status stokes_vmult(stokes_ctx* ctx, int level, int block, int prec,
                           const void* src_dev, void* dst_dev, void* stream);

/* x = V(rhs): one GMG V-cycle with zero initial guess on the finest level
 * (Section 2.2.1): per level one pre- and one post-smoothing step of the
 * degree-k Jacobi-Chebyshev smoother, residual, restriction, recursion,
 * prolongation; exact FP64 solve on level 0. prec selects the arithmetic of
 * the whole cycle (FP32: vectors and kernels in FP32, coarse solve in FP64);
 * rhs and x have that precision and length N_u. x holds rhs on constrained
 * entries. rhs and x must not overlap. Octree contexts: rhs and x are FP64 active velocity
 * vectors whatever prec (prec selects the arithmetic of the local-smoothing cycle). */
stokes_status gmg_vcycle(stokes_ctx* ctx, int prec, const void* rhs_dev, void* x_dev, void* stream);

/* Solve [[A, B^T], [B, 0]] [u; p] = [rhs_u; rhs_p] with right-preconditioned
 * FP64 FGMRES(restart) (Section 2.2.2) and P^-1 of eq. stokes_precond:
 * z_p = -S_hat^-1 r_p, z_u = V(r_u - B^T z_p), the V-cycle in `vcycle_prec`
 * (options outer_solver and precond_kind select GMRES, IDR(s) or MINRES and the
 * block-diagonal P_D instead). rhs_dev = NULL uses the sinker right-hand side
 * [F; 0]. up_dev: in = initial guess, out = solution with zero-mean pressure.
 * Stops when the recurrence residual <= rtol ||b|| and the true residual
 * b - K x, recomputed with the native FP64 operator, is too; otherwise the
 * method restarts from x (at most 10 times). The returned status follows that
 * true residual: OK only if it is <= rtol ||b||, NOT_CONVERGED otherwise
 * (max_it reached, or the restarts used up; up holds the last iterate and
 * info->rel_residual_true its true residual). Host-synchronous (small
 * device->host reads per iteration). Errors: NOT_CONVERGED, BREAKDOWN, EINVAL,
 * ENOMEM, ECUDA. */
stokes_status stokes_solve(stokes_ctx* ctx, int vcycle_prec, const double* rhs_dev, double* up_dev,
                           double rtol, int max_it, stokes_solve_info* info, void* stream);

/* Solve n_problems independent Stokes systems together (each context from its own stokes_setup,
 * any sizes): the same FGMRES (or GMRES, per context option outer_solver 0 or 2) as stokes_solve,
 * with the iterations of all unconverged problems advancing in lock step; contexts set up for IDR(s)
 * or MINRES are EINVAL. Each problem's kernels run on its own stream (streams[i]; streams = NULL:
 * library-created streams), so small problems share the GPU, and each problem's V-cycle is replayed
 * as its captured graph. rhs_devs = NULL or rhs_devs[i] = NULL: the sinker right-hand side [F; 0].
 * up_devs[i]: in = initial guess, out = solution (zero-mean pressure). infos[i] (optional) per
 * problem; seconds = wall time of the whole batch. Host-synchronous. A context may appear only once.
 * Errors: EINVAL, ENOMEM, ECUDA; NOT_CONVERGED or BREAKDOWN if any problem ended so (the others
 * are still solved). No counterpart in the paper: batching is the GPU's way to fill the device with
 * many small problems. */
stokes_status stokes_batch_solve(int n_problems, stokes_ctx* const* ctxs, int vcycle_prec,
                                 const double* const* rhs_devs, double* const* up_devs, double rtol, int max_it,
                                 stokes_solve_info* infos, void* const* streams);

/* Same as stokes_solve with HOST buffers: copies rhs_host (or uses the sinker
 * F when NULL) to library-owned device memory, solves from a zero initial
 * guess and copies the solution to up_host (length N_u + N_p). */
stokes_status stokes_solve_host(stokes_ctx* ctx, int vcycle_prec, const double* rhs_host, double* up_host,
                                double rtol, int max_it, stokes_solve_info* info, void* stream);

/* ---- single steps of the path (each is what the V-cycle / solve runs) ---- */

/* Copy the cell viscosity of `level` (n_l^3 doubles, cell ci + n cj + n^2 ck) (Section 2.3). */
stokes_status stokes_get_viscosity(stokes_ctx* ctx, int level, double* mu_dev, void* stream);
/* Copy 1/diag(A_l) (N_u doubles, 0 on constrained entries). */
stokes_status stokes_get_inv_diagonal(stokes_ctx* ctx, int level, double* dinv_dev, void* stream);
/* Lanczos estimate of lambda_max(D_l^-1 A_l) (host double; 0 for level 0). */
stokes_status stokes_get_lambda_max(stokes_ctx* ctx, int level, double* lam_host);
/* Copy the assembled right-hand side F (N_u doubles, Section 2.1, def. of F). */
stokes_status stokes_get_rhs(stokes_ctx* ctx, double* F_dev, void* stream);
/* fine = P coarse (add = 0) or fine += P coarse (add = 1): Q2 embedding from
 * level fine_level-1 to fine_level, constrained fine entries left 0 / unchanged. */
stokes_status stokes_prolongate(stokes_ctx* ctx, int fine_level, int prec, const void* coarse_dev,
                                void* fine_dev, int add, void* stream);
/* coarse = P^T fine, constrained coarse entries set to 0. */
stokes_status stokes_restrict(stokes_ctx* ctx, int fine_level, int prec, const void* fine_dev,
                              void* coarse_dev, void* stream);
/* One smoothing step of degree k on level >= 1: x <- x + q(D^-1 A) D^-1 (b - A x)
 * (zero_guess = 1: x is output only). Constrained entries of b must be 0. */
stokes_status stokes_smooth(stokes_ctx* ctx, int level, int prec, const void* b_dev, void* x_dev,
                            int zero_guess, void* stream);
/* x = A_0^-1 b on the coarsest level's free DoFs (FP64 arithmetic), 0 elsewhere. */
stokes_status stokes_coarse_solve(stokes_ctx* ctx, int prec, const void* b_dev, void* x_dev, void* stream);
/* z_p = S_hat^-1 r_p: Jacobi-Chebyshev of degree schur_degree on M_p, interval [1/8, 27/8]. */
stokes_status stokes_schur_inverse(stokes_ctx* ctx, const double* rp_dev, double* zp_dev, void* stream);
/* z = P^-1 r for a Stokes vector (eq. stokes_precond), V-cycle in vcycle_prec. */
stokes_status stokes_precondition(stokes_ctx* ctx, int vcycle_prec, const double* r_dev, double* z_dev,
                                  void* stream);

/* Autotuner (no counterpart in the paper). what = 1: threads per block of the cell-parallel level
 * operator (64, 128 or 256; the fastest FP32 product on the finest level); what = 2: the Chebyshev
 * degree (3..6) with the shortest wall time of an FGMRES solve to relative residual 1e-3 with the
 * FP32 V-cycle and the context's own right-hand side; what = 3: both. The choice is kept in the
 * context for later V-cycles and solves (captured graphs are dropped and recaptured). Outputs may
 * be NULL. Synchronous; allocates work vectors (and the Krylov basis) on first use.
 * Note: the paper's smoother degree is 4; a tuned degree trades smoothing work per V-cycle against
 * the outer iteration count. */
stokes_status stokes_autotune(stokes_ctx* ctx, int what, void* stream, int* block_out, int* degree_out);

/* Change options.batch_vcycle of a context (0 or 1; see stokes_options): how stokes_batch_solve
 * runs the FP32 V-cycles when this context comes first in the batch. Errors: EINVAL. No counterpart
 * in the paper. */
stokes_status stokes_set_batch_vcycle(stokes_ctx* ctx, int mode);

/* Synchronise `stream`, then read and clear the context's device status word: TIMEOUT if a
 * bounded wait inside one of the library's kernels gave up since the last check (the output of
 * that call is undefined; the context stays usable), OK otherwise. stokes_solve checks the word
 * itself before it returns. No counterpart in the paper. */
stokes_status stokes_device_status(stokes_ctx* ctx, void* stream);

/* ---- allocation-free entry point (no counterpart in the paper) ---- */

/* Largest pressure space stokes_schur_inverse_noalloc accepts: the (n+1)^3 Q1
 * vertices of a 32^3 mesh. */
#define STOKES_NOALLOC_MAX_NP 35937
/* z_p = S_hat^-1 r_p exactly as stokes_schur_inverse computes it (Jacobi-
 * Chebyshev of the given degree on the 1/mu-weighted pressure mass matrix,
 * interval [1/8, 27/8]), for callers that cannot allocate device memory and so
 * cannot create a context: it takes the uniform mesh size n and the caller's
 * cell viscosity mu_dev (n^3 doubles, cell ci + n cj + n^2 ck), needs no
 * stokes_ctx, and calls no cudaMalloc/cudaFree. Its three work vectors live in
 * one fixed device array of 3 * STOKES_NOALLOC_MAX_NP doubles (~0.86 MB) that
 * every GPU loading the library holds until exit. The first call on a device
 * looks up that array's address (make it before any stream capture); later
 * calls on a stream that is not capturing look it up again. All calls share
 * the array: calls that overlap on the GPU race; serialise them. degree 0 is
 * S_hat = diag(M_p), as for the context's schur_degree = 0. rp_dev and zp_dev
 * hold (n+1)^3 doubles and must not overlap. Errors: EINVAL (null pointer,
 * n < 1, n > 32, i.e. (n+1)^3 > STOKES_NOALLOC_MAX_NP, degree < 0), ECUDA. */
stokes_status stokes_schur_inverse_noalloc(int n, const double* mu_dev, const double* rp_dev, double* zp_dev,
                                           int degree, void* stream);

/* ---- instrumentation (no counterpart in the paper; used by the benchmark) ---- */

/* Kernel classes timed by stokes_profile: 0 velocity cell kernel FP32, 1 velocity
 * cell kernel FP64, 2 fused A+B^T+B cell kernel, 3 B^T cell kernel, 4 pressure mass
 * cell kernel, 5 transfers, 6 smoother / residual vector kernels, 7 Krylov vector
 * kernels, 8 coarse solve, 9 precision casts, 10 the outer operator applied in native FP64
 * for the solvers' restart and final residuals (uniform meshes). */
#define STOKES_PROF_NCLASS 11
/* enable = 1: record a CUDA event pair around every kernel launch the library
 * issues from now on (adds two event records per launch); 0: stop. Process-wide,
 * for single-threaded use. */
stokes_status stokes_profile(int enable);
/* Milliseconds and launches accumulated for class `cls` (synchronises the device);
 * reset = 1 clears all classes afterwards. */
stokes_status stokes_profile_read(int cls, double* ms, long long* launches, int reset);
/* Test hook: from now on the library's device allocations fail with ENOMEM once they would take
 * more than `bytes` in total (freed bytes are not counted back); bytes < 0 removes the limit.
 * Exercises the allocation-failure paths of set-up and solve (a failed set-up frees what it had
 * allocated). Process-wide, for single-threaded use. */
stokes_status stokes_debug_alloc_limit(long long bytes);
/* 1 if this library was built with STOKES_DEBUG (index-map checks), else 0. In such a build
 * every kernel of the octree path checks each entry it reads from a host-built index map
 * (table numbers: 0 cell -> level nodes, 1 node -> parent cell, 2 node -> position in the parent,
 * 3 leaf -> velocity nodes or constraints, 4 velocity constraint -> nodes, 5 leaf -> pressure
 * vertices or constraints, 6 pressure constraint -> vertices, 7 copy list -> active node,
 * 8 copy list -> level node) against the size of what it indexes. A bad entry is skipped, never
 * trapped on, and recorded in the context's status words; the call that ran the kernel
 * (stokes_setup_octree, stokes_vmult, gmg_vcycle, stokes_schur_inverse, stokes_precondition,
 * stokes_solve; each synchronises its stream in such a build) then returns STOKES_EMESH and
 * stokes_last_error() names the table and the entry's position in it. */
int stokes_debug_build(void);
/* Test hook of STOKES_DEBUG builds: from now on the checks of `table` on this octree context
 * accept only entries below (true bound - cut), so that the last `cut` valid entries read as bad
 * and exercise the path above without any out-of-range access. Drops the captured V-cycle
 * graphs. Errors: EINVAL (release build, uniform-mesh context, bad table, cut < 0), ECUDA. */
stokes_status stokes_debug_index_cut(stokes_ctx* ctx, int table, long long cut);
/* Number of kernel launches the library has issued since it was loaded. */
long long stokes_launch_count(void);
/* FP32 and FP64 FMA throughput of the current device in TFLOP/s (eight independent FMA
 * chains per thread, 8 CTAs of 256 threads per SM, ~10 ms each; synchronous). */
stokes_status stokes_probe_fma(double* fp32_tflops, double* fp64_tflops);

#ifdef __cplusplus
}
#endif

#endif /* STOKES_GB300_H */
