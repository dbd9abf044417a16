// octree.cuh -- adaptive octree meshes: host tables (octree_host.cpp) and device kernels
// (octree.cu) for the constrained active operator and the local-smoothing level hierarchy.
//
// A cell is packed as key = l << 48 | k << 32 | j << 16 | i (level l <= 15, 0 <= i,j,k < 2^l),
// side 2^-l. Points lie on the lattice of spacing 2^-(lmax+1): a level-l cell has
// S = 2^(lmax+1-l) lattice units per side and its Q2 nodes at (i S, j S, k S) + (a, b, c) S/2.
// Point key = x + Mx (y + Mx z), Mx = 2^(lmax+1) + 1; nodes are numbered in increasing key
// order on the active mesh and on every level, cells in increasing cell key.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "internal.cuh"

namespace stk {

inline uint64_t oct_key(int l, int i, int j, int k) {
    return (uint64_t(l) << 48) | (uint64_t(k) << 32) | (uint64_t(j) << 16) | uint64_t(i);
}
inline int oct_l(uint64_t c) { return int(c >> 48); }
inline int oct_i(uint64_t c) { return int(c & 0xFFFF); }
inline int oct_j(uint64_t c) { return int((c >> 16) & 0xFFFF); }
inline int oct_k(uint64_t c) { return int((c >> 32) & 0xFFFF); }

// Refinement around the sinkers (see stokes_octree_sinker_mesh) and full 2:1 balance.
std::vector<uint64_t> oct_refine_shells(int base_level, int n_sinkers, const double* centres,
                                        const int* max_levels, double radius, double half_width);
std::vector<uint64_t> oct_balance(const std::vector<uint64_t>& leaves);

// One multigrid level of the local-smoothing hierarchy (all cells of level l).
struct OctLevelHost {
    int l = 0;
    std::vector<uint64_t> cells;       // sorted cell keys
    std::vector<uint64_t> nodes;       // sorted node keys
    std::vector<int32_t> cell_nodes;   // [cells][27] level node indices
    std::vector<uint8_t> flags;        // per node: 1 = cube boundary, 2 = refinement edge
    std::vector<double> mu;            // per cell
    std::vector<uint32_t> parent;      // per node, l > coarsest: parent cell (index on level l-1)
    std::vector<uint16_t> pos;         // per node: position in the parent, px + 5 py + 25 pz, p in 0..4
};

constexpr int kOctUCon = 9;            // terms of a velocity (Q2) hanging-node constraint
constexpr int kOctPCon = 4;            // terms of a pressure (Q1) hanging-node constraint

struct OctHost {
    int base = 0, coarsest = 0, lmax = 0;
    uint64_t Mx = 0;
    std::vector<uint64_t> leaves;      // sorted
    std::vector<double> leaf_mu, leaf_h;
    // velocity: active Q2 nodes, hanging constraints, per-leaf references
    std::vector<uint64_t> unodes;
    std::vector<uint8_t> ubnd;
    std::vector<int32_t> leaf_u;       // [leaves][27]: node index, or -(constraint + 1)
    std::vector<int32_t> ucon_node;    // [constraints][kOctUCon], -1 = unused
    std::vector<double> ucon_w;
    // pressure: active Q1 vertices
    std::vector<uint64_t> pverts;
    std::vector<int32_t> leaf_p;       // [leaves][8]
    std::vector<int32_t> pcon_node;    // [constraints][kOctPCon]
    std::vector<double> pcon_w;
    // local smoothing
    std::vector<OctLevelHost> levels;  // levels coarsest .. lmax
    std::vector<int32_t> copy_level;   // per active velocity node: level of its coarsest leaf
    std::vector<int32_t> copy_index;   // its index on that level
    // right-hand side, pressure mass diagonal and weights
    std::vector<double> F;             // 3 * unodes, component-blocked
    std::vector<double> mp_diag, p_weights;
};

struct OctSinkers {
    int n = 0;
    const double* centres = nullptr;
    double mu_min = 1, mu_max = 1, delta = 200, omega = 0.1, beta = 10;
};

// Builds every table from a 2:1-balanced leaf set (active_only: the sorted leaves, their sizes
// and the velocity space with its constraints only). Returns an empty string on success, else
// the reason (unbalanced mesh, constraint chain, bad keys).
std::string oct_build(const std::vector<uint64_t>& leaves, int coarsest, const OctSinkers& sk, OctHost& out,
                      bool active_only = false);

// Gradient indicator of every leaf (sorted order): eta_K = h^(5/2) |grad u_h(x_K)|_F from the active
// velocity u (component-blocked [3][unodes], Dirichlet values read as 0); and the refinement that
// splits the floor(n fraction + 1/2) leaves with the largest eta (ties: smaller key), then 2:1
// balances (Section 3.3, gradient-based adaptive refinement).
void oct_gradient_indicator(const OctHost& o, const double* u, std::vector<double>& eta);
std::vector<uint64_t> oct_refine_by_indicator(const std::vector<uint64_t>& leaves, const std::vector<double>& eta,
                                              double fraction);

// ---- device side (octree.cu) ----

// Index-map checks of STOKES_DEBUG builds. Every entry a kernel reads from one of these host-built
// tables is compared with the size of what it indexes; a bad entry is skipped (its gather reads 0,
// its scatter is dropped) and recorded in the context's status word (kStatusBadIndex, then the
// table and the entry's position in it, first one wins), which the next read of the status word
// turns into STOKES_EMESH. Nothing traps. Release builds compile the checks away.
enum OctTable {
    OCT_CELL_NODES = 0,   // level cell -> 27 level nodes
    OCT_PARENT,           // level node -> parent cell on the next coarser level
    OCT_POS,              // level node -> position in its parent (< 125)
    OCT_LEAF_U,           // leaf -> 27 active velocity nodes or constraints
    OCT_UCON_NODE,        // velocity constraint -> its terms' nodes
    OCT_LEAF_P,           // leaf -> 8 active pressure vertices or constraints
    OCT_PCON_NODE,        // pressure constraint -> its terms' vertices
    OCT_COPY_ACTIVE,      // copy list -> active velocity node
    OCT_COPY_LEVEL,       // copy list -> level node
    OCT_NTABLES
};
const char* oct_table_name(int table);

// Status word bits and layout (4 unsigned: flags, table + 1 of the first bad entry, its position
// low and high word); bits 1 and 2 are the bounded waits' time-outs.
constexpr unsigned kStatusBadIndex = 4u;
constexpr int kStatusWords = 4;

struct OctDebug {
    unsigned* status = nullptr;          // the context's status words
    long long cut[OCT_NTABLES] = {};     // test hook: bound lowered by cut[t] for table t
};

struct OctLevelDev {
    int n_cells = 0;
    size_t nn = 0;                      // level nodes; vectors hold 3 nn entries
    double h = 0;
    const int32_t* cell_nodes = nullptr;
    const uint8_t* flags = nullptr;
    const uint32_t* parent = nullptr;
    const uint16_t* pos = nullptr;
    OctDebug dbg;
};

struct OctActiveDev {
    int n_leaves = 0;
    size_t nu_nodes = 0, np = 0;
    const int32_t* leaf_u = nullptr;
    const int32_t* leaf_p = nullptr;
    const int32_t* ucon_node = nullptr;
    const double* ucon_w = nullptr;
    const int32_t* pcon_node = nullptr;
    const double* pcon_w = nullptr;
    const uint8_t* ubnd = nullptr;
    const double* mu = nullptr;         // per leaf
    const uint8_t* level = nullptr;     // per leaf
    size_t n_ucon = 0, n_pcon = 0;      // constraint records
    OctDebug dbg;
};

// acc (+)= A_l src over the level's cells (src boundary entries read as 0, boundary rows of acc
// untouched); the caller zeroes acc first.
template <typename T>
cudaError_t launch_oct_level_cells(const OctLevelDev& L, const T* mu, const T* src, T* acc, cudaStream_t s);
// dst = src on boundary nodes (identity rows).
template <typename T>
cudaError_t launch_oct_copy_boundary(const OctLevelDev& L, const T* src, T* dst, cudaStream_t s);
// diag[c][node] = sum over cells of mu h A_hat[c*27+a][c*27+a]; then inverse with 0 on boundary
// and refinement-edge nodes.
cudaError_t launch_oct_inv_diag(const OctLevelDev& L, const double* mu, const double* ref_diag81, double* tmp,
                                double* dinv, cudaStream_t s);
// Level transfers between level l (fine, with parent/pos) and level l-1 (coarse cells).
template <typename T>
cudaError_t launch_oct_prolongate(const OctLevelDev& F, const OctLevelDev& C, const T* coarse, T* fine, bool add,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_oct_restrict_add(const OctLevelDev& F, const OctLevelDev& C, const T* fine, T* coarse,
                                    cudaStream_t s);
// Copies between an active velocity vector (FP64) and the level vectors of one level.
template <typename T>
cudaError_t launch_oct_copy_to_level(size_t n_copy, const int32_t* active_idx, const int32_t* level_idx,
                                     size_t nu_nodes, size_t level_nn, const double* active, T* level,
                                     const OctDebug& dbg, cudaStream_t s);
template <typename T>
cudaError_t launch_oct_copy_from_level(size_t n_copy, const int32_t* active_idx, const int32_t* level_idx,
                                       size_t nu_nodes, size_t level_nn, const T* level, double* active,
                                       const OctDebug& dbg, cudaStream_t s);
// Active blocks with hanging-node constraints (FP64): dst_u = A u + B^T p, dst_p = B u by flags;
// dst parts are overwritten; Dirichlet rows of dst_u hold src_u (DO_A) or 0 (B^T only).
cudaError_t launch_oct_active(const OctActiveDev& a, const double* src_u, const double* src_p, double* dst_u,
                              double* dst_p, bool do_a, bool do_bt, bool do_b, cudaStream_t s);
// dst_u = src_u on the Dirichlet rows of the active velocity space.
cudaError_t launch_oct_identity_rows(const OctActiveDev& a, const double* src_u, double* dst_u, cudaStream_t s);
// dst = M_p src on the active pressure space (FP64).
cudaError_t launch_oct_mass_p(const OctActiveDev& a, const double* src, double* dst, cudaStream_t s);

// Chebyshev consumers of a level product accumulated in acc (brick.cu):
// EPI 1: r = b - acc; EPI 2: d = c1 d + c2 dinv (b - acc), x += d; both clear acc.
template <typename T>
cudaError_t launch_consume(int epi, size_t n, T* acc, const T* b, const T* dinv, T* d, T* x_or_r, double c1,
                           double c2, cudaStream_t s);

}  // namespace stk
