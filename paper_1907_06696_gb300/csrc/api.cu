// api.cu -- context, set-up, V-cycle, FGMRES and the C ABI (include/stokes.h).
//
// V-cycle (Section 2.2.1): per level l >= 1, one degree-k Jacobi-Chebyshev
// pre-smoothing step from a zero guess, residual, restriction, recursion,
// prolongation and one post-smoothing step; level 0 is solved exactly with
// the dense FP64 inverse of its free block. Chebyshev recurrence: Y. Saad,
// Iterative Methods for Sparse Linear Systems, 2nd ed., Alg. 12.1, with the
// Jacobi-preconditioned residual; interval [lam_hi / range, lam_hi],
// lam_hi = safety * Lanczos estimate of lambda_max(D^-1 A).
// Outer solve (Section 2.2.2): right-preconditioned FGMRES(restart) in FP64
// with P^-1 of eq. (stokes_precond); classical Gram-Schmidt applied twice,
// each pass one fused multi-dot and one fused multi-axpy, one host
// synchronisation per iteration.
#include "../../include/stokes.h"
#include "batch.cuh"
#include "brick.cuh"
#include "internal.cuh"
#include "octree.cuh"
#include "prof.cuh"

#include <algorithm>
#include <chrono>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

using namespace stk;

namespace stk {

// Process-wide launch counter and optional event timing (single host thread).
namespace {
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};
bool g_prof_on = false;
long long g_launches = 0;
std::vector<cudaEvent_t> g_pool;
std::vector<ProfRec> g_recs;
cudaEvent_t g_open = nullptr;
double g_ms[PROF_NCLASS] = {};
long long g_cnt[PROF_NCLASS] = {};

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain() {
    if (g_recs.empty()) return;
    cudaDeviceSynchronize();
    for (const ProfRec& r : g_recs) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) g_ms[r.cls] += ms;
        g_cnt[r.cls] += 1;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}
}  // namespace

void prof_begin(int, cudaStream_t s) {
    if (!g_prof_on) return;
    g_open = take_event();
    cudaEventRecord(g_open, s);
}
thread_local int t_override = -1;
void prof_override(int cls) { t_override = cls; }
void prof_end(int cls, cudaStream_t s) {
    if (!g_prof_on || !g_open) return;
    cudaEvent_t e = take_event();
    cudaEventRecord(e, s);
    g_recs.push_back({t_override >= 0 ? t_override : cls, g_open, e});
    g_open = nullptr;
    if (g_recs.size() > 200000) drain();
}
void prof_count(int k) { g_launches += k; }
bool prof_enabled() { return g_prof_on; }
long long launch_total() { return g_launches; }

}  // namespace stk

namespace {

thread_local std::string g_last_error;

stokes_status fail(stokes_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

#define CK(expr)                                                                                         \
    do {                                                                                                 \
        cudaError_t _e = (expr);                                                                         \
        if (_e != cudaSuccess)                                                                           \
            return fail(_e == cudaErrorMemoryAllocation ? STOKES_ENOMEM : STOKES_ECUDA,                  \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                             \
    } while (0)

#define CKS(expr)                                                                                        \
    do {                                                                                                 \
        stokes_status _s = (expr);                                                                       \
        if (_s != STOKES_OK) return _s;                                                                  \
    } while (0)

template <typename T>
struct LevelVecs {
    T* b = nullptr;   // right-hand side of the level problem
    T* x = nullptr;   // level solution / correction
    T* r = nullptr;   // residual
    T* d = nullptr;   // Chebyshev direction
    T* t = nullptr;   // operator output
    T* mu = nullptr;  // cell viscosity
    T* dinv = nullptr;
    T* acc = nullptr; // operator accumulator of the cell-parallel kernel (kept at zero between uses)
    // the fused smoother's second (d, x) pair and its two further accumulators (zero between uses)
    T* x2 = nullptr;
    T* d2 = nullptr;
    T* acc2 = nullptr;
    T* acc3 = nullptr;
};

struct Level {
    LevelGeom g;
    LevelVecs<double> v64;
    LevelVecs<float> v32;
    PlaneLayout planes{};        // brick-plane slots of the tiled operator
    double* slots64 = nullptr;
    float* slots32 = nullptr;
    double lam_max = 0.0, lo = 0.0, hi = 0.0;
};

template <typename T> LevelVecs<T>& vecs(Level& L);
template <> LevelVecs<double>& vecs<double>(Level& L) { return L.v64; }
template <> LevelVecs<float>& vecs<float>(Level& L) { return L.v32; }
template <typename T> T* slots(Level& L);
template <> double* slots<double>(Level& L) { return L.slots64; }
template <> float* slots<float>(Level& L) { return L.slots32; }

// One level of the local-smoothing hierarchy of an octree mesh (index 0 = coarsest).
struct OctLevel {
    OctLevelDev g;
    LevelVecs<double> v64;
    LevelVecs<float> v32;
    double lam_max = 0.0, lo = 0.0, hi = 0.0;
    size_t n_copy = 0;                 // active nodes copied to / from this level
    int32_t* copy_a = nullptr;         // their active indices
    int32_t* copy_l = nullptr;         // their level indices
};

// Adaptive (octree) mesh: active space with hanging-node constraints and the level hierarchy.
struct OctCtx {
    OctHost host;
    OctActiveDev act;
    std::vector<OctLevel> lev;
    double* leaf_mu = nullptr;
};

template <typename T> LevelVecs<T>& ovecs(OctLevel& L);
template <> LevelVecs<double>& ovecs<double>(OctLevel& L) { return L.v64; }
template <> LevelVecs<float>& ovecs<float>(OctLevel& L) { return L.v32; }

}  // namespace

struct stokes_ctx {
    int n = 0, L = 0;
    stokes_options opt{};
    std::vector<Level> lev;
    std::vector<void*> allocs;
    double* ref_diag = nullptr;
    double* F = nullptr;          // finest right-hand side (N_u)
    double* mp_dinv = nullptr;    // 1 / diag(M_p)
    double* p_weights = nullptr;  // int psi_l
    double p_wsum = 1.0;
    // Schur Chebyshev work (N_p each)
    double *sp_d = nullptr, *sp_t = nullptr;
    double *sp_z2 = nullptr, *sp_d2 = nullptr;   // second (z, d) pair of the gathered S_hat^-1 steps
    double* mp_scale = nullptr;                 // h^3 / mu per finest cell
    // preconditioner / operator work (N_u)
    double* tu = nullptr;
    float *stage_in = nullptr, *stage_out = nullptr;   // FP32 V-cycle input / output
    // coarse level
    int nf = 0;
    int* free_idx = nullptr;
    double* Ainv = nullptr;
    // reductions
    double* partials = nullptr;
    double* dots = nullptr;       // device results (up to 2*restart+8)
    double* dots_host = nullptr;  // pinned
    // Krylov workspace (allocated on first solve)
    size_t N = 0;
    size_t ldv = 0;   // row stride of V (N rounded up to even)
    double *V = nullptr, *Z = nullptr, *w = nullptr, *bvec = nullptr, *hdev = nullptr;
    int krylov_restart = 0;
    // host-buffer solve
    double *h_rhs_dev = nullptr, *h_up_dev = nullptr;
    // V-cycle replayed as a captured CUDA graph on a library stream (per precision)
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // [FP64, FP32]
    long long glaunches[2] = {0, 0};                 // kernel launches inside each graph
    int cell_block = 128;                            // threads per block of the cell kernel (autotuned)
    float *tune_x = nullptr, *tune_r = nullptr, *tune_b = nullptr;   // autotuner work (FP32, finest level)
    double* tune_up = nullptr;                                        // autotuner solution vector
    OctCtx* oct = nullptr;                           // set for octree meshes (stokes_setup_octree)
    // IDR(s) workspace (allocated on the first IDR solve): G, U, P (s vectors each), r, v, t, tmp
    int idr_alloc_s = 0;
    double *idr_G = nullptr, *idr_U = nullptr, *idr_P = nullptr, *idr_r = nullptr, *idr_v = nullptr,
           *idr_t = nullptr, *idr_tmp = nullptr, *idr_c = nullptr;
    cudaStream_t idr_stream = nullptr;
    double* mr[11] = {};   // MINRES work vectors
    // tensor-core level operator: f16 table of 5400 A_hat; device status word (bit 0: a bounded
    // wait inside a kernel gave up), checked by stokes_device_status and at the end of a solve
    void* tc_table = nullptr;
    void* outer_tc_table = nullptr;   // outer_arith 2: the f16 integer element table
    unsigned* dev_status = nullptr;
    TcArgs tc{};
};

namespace {

// Test hook (stokes_debug_alloc_limit): bytes the library may still allocate on the device; < 0 =
// no limit.
long long g_alloc_left = -1;

template <typename T>
stokes_status dalloc(stokes_ctx* c, T** p, size_t count) {
    const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
    if (g_alloc_left >= 0) {
        if ((long long)bytes > g_alloc_left) return fail(STOKES_ENOMEM, "device allocation limit reached (test hook)");
        g_alloc_left -= (long long)bytes;
    }
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return fail(STOKES_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return STOKES_OK;
}

// Host reductions: copy k device scalars to host (synchronous on the stream).
stokes_status fetch(stokes_ctx* c, int k, cudaStream_t s, double* out) {
    CK(cudaMemcpyAsync(c->dots_host, c->dots, size_t(k) * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < k; ++i) out[i] = c->dots_host[i];
    return STOKES_OK;
}

stokes_status dot(stokes_ctx* c, size_t n, const double* a, const double* b, cudaStream_t s, double* out) {
    CK(launch_multidot(n, 1, a, n, b, c->partials, c->dots, s));
    return fetch(c, 1, s, out);
}

// Largest eigenvalue of the symmetric tridiagonal matrix (alpha, beta) by Sturm bisection.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
    const int k = int(a.size());
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
        double r = 0.0;
        if (i > 0) r += std::fabs(b[i - 1]);
        if (i < k - 1) r += std::fabs(b[i]);
        lo = std::fmin(lo, a[i] - r);
        hi = std::fmax(hi, a[i] + r);
    }
    auto count_below = [&](double x) {  // number of eigenvalues < x
        int cnt = 0;
        double q = a[0] - x;
        if (q < 0) ++cnt;
        for (int i = 1; i < k; ++i) {
            if (q == 0.0) q = 1e-300;
            q = a[i] - x - b[i - 1] * b[i - 1] / q;
            if (q < 0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (count_below(mid) >= k) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Level-operator selector for launch_level_op: 1 = brick kernel, 2 = tensor-core brick kernel,
// 3 = component-split kernel (FP32 levels), else the cell kernel's block size. By default the
// FP32 levels of at most kSplitMaxN^3 cells take the component-split kernel: there a level
// operator is one short wave and its time one thread's serial work, which the split divides by 3.
constexpr int kSplitMaxN = 16;

template <typename T>
int level_kernel(const stokes_ctx* c, int l) {
    const int k = c->opt.vmult_kernel;
    if (k == 1 || k == 2 || k == 3) return k;
    if (sizeof(T) == 4 && c->lev[l].g.n <= kSplitMaxN) return 3;
    return c->cell_block;
}

template <typename T>
stokes_status vmult_level(stokes_ctx* c, int l, const T* src, T* dst, cudaStream_t s) {
    Level& L = c->lev[l];
    CK(launch_level_op<T>(level_kernel<T>(c, l), L.g, L.planes, EPI_PLAIN, vecs<T>(L).mu, src, dst, nullptr, nullptr,
                          nullptr, 0.0, 0.0, slots<T>(L), vecs<T>(L).acc, s, &c->tc));
    return STOKES_OK;
}

// Chebyshev step fused into the operator: d = c1 d + c2 D^-1 (b - A x); x += d (x in place).
template <typename T>
stokes_status cheb_step(stokes_ctx* c, int l, const T* b, T* x, double c1, double c2, cudaStream_t s) {
    Level& L = c->lev[l];
    LevelVecs<T>& v = vecs<T>(L);
    CK(launch_level_op<T>(level_kernel<T>(c, l), L.g, L.planes, EPI_CHEB, v.mu, x, nullptr, b, v.dinv, v.d, c1, c2,
                          slots<T>(L), v.acc, s, &c->tc));
    return STOKES_OK;
}

// One degree-k Chebyshev smoothing step on level l (x, b caller buffers of the level size).
template <typename T>
stokes_status smooth(stokes_ctx* c, int l, const T* b, T* x, bool zero_guess, cudaStream_t s) {
    Level& L = c->lev[l];
    LevelVecs<T>& v = vecs<T>(L);
    const double theta = 0.5 * (L.hi + L.lo), delta = 0.5 * (L.hi - L.lo);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    const size_t n = L.g.n_u;
    if (zero_guess) {
        CK(launch_cheb_update<T>(n, b, nullptr, v.dinv, v.d, x, 0.0, 1.0 / theta, false, s));
    } else {
        CKS(cheb_step<T>(c, l, b, x, 0.0, 1.0 / theta, s));
    }
    for (int it = 1; it < c->opt.cheb_degree; ++it) {
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        CKS(cheb_step<T>(c, l, b, x, rho_new * rho, 2.0 * rho_new / delta, s));
        rho = rho_new;
    }
    return STOKES_OK;
}

// Whether level l smooths with each Chebyshev step carried by the next product (the cell and
// component-split operators; the level has the second (d, x) pair and the extra accumulators).
template <typename T>
bool fused_level(const stokes_ctx* c, int l) {
    const int k = level_kernel<T>(c, l);
    return c->opt.fused_smoother == 1 && k != 1 && k != 2 && vecs<T>(const_cast<Level&>(c->lev[l])).x2 != nullptr;
}

// Degree-k smoothing with each step's update carried by the next product (ChebGather); with r
// given also r = b - A x_k, whose product then carries the last update. The iterates alternate
// between (x, d) and the level's (x2, d2); the accumulators rotate over acc, acc2, acc3 (all zero
// again on return). x receives the result.
template <typename T>
stokes_status smooth_fused(stokes_ctx* c, int l, const T* b, T* x, bool zero_guess, T* r, cudaStream_t s) {
    Level& L = c->lev[l];
    LevelVecs<T>& v = vecs<T>(L);
    const int kern = level_kernel<T>(c, l);
    const int deg = c->opt.cheb_degree;
    const double theta = 0.5 * (L.hi + L.lo), delta = 0.5 * (L.hi - L.lo);
    const double sigma = theta / delta;
    // coefficients of step j: d <- c1[j] d + c2[j] D^-1 (b - A x), x <- x + d (as smooth())
    std::vector<double> c1(deg), c2(deg);
    double rho = 1.0 / sigma;
    c1[0] = 0.0;
    c2[0] = 1.0 / theta;
    for (int j = 1; j < deg; ++j) {
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        c1[j] = rho_new * rho;
        c2[j] = 2.0 * rho_new / delta;
        rho = rho_new;
    }
    T* X[2] = {x, v.x2};
    T* Dv[2] = {v.d, v.d2};
    T* A[3] = {v.acc, v.acc2, v.acc3};
    const size_t n = L.g.n_u;
    // products of the iterates first .. last: the first plain, the others carrying a step
    const int first = zero_guess ? 1 : 0;
    const int last = r ? deg : deg - 1;
    const int m = last - first + 1;
    const int fused = m > 1 ? m - 1 : 0;
    // with r the last carried step writes x_k, which must land in x: start in pair (fused mod 2)
    const int p0 = (r && (fused & 1)) ? 1 : 0;
    if (zero_guess) {
        CK(launch_cheb_update<T>(n, b, nullptr, v.dinv, Dv[p0], X[p0], 0.0, c2[0], false, s));
    } else if (p0 == 1) {
        CK(cudaMemcpyAsync(X[1], x, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    if (m <= 0) return STOKES_OK;
    int cur = p0;
    CK(launch_accumulate<T>(kern, L.g, v.mu, X[cur], A[0], s));
    for (int j = 2; j <= m; ++j) {
        const int step = first + j - 2;   // the update from iterate `step` to `step + 1`
        ChebGather<T> g;
        g.acc_prev = A[(j - 2) % 3];
        g.b = b;
        g.dinv = v.dinv;
        g.d_old = Dv[cur];
        g.x_old = X[cur];
        g.d_new = Dv[cur ^ 1];
        g.x_new = X[cur ^ 1];
        g.acc_zero = j == 2 ? nullptr : A[j % 3];
        g.c1 = T(c1[step]);
        g.c2 = T(c2[step]);
        CK(launch_cell_cheb<T>(kern, L.g, v.mu, g, A[(j - 1) % 3], s));
        cur ^= 1;
    }
    T* zero2 = m >= 2 ? A[(m - 2) % 3] : nullptr;
    if (r) {
        CK(launch_consume2<T>(EPI_RESID, n, A[(m - 1) % 3], b, nullptr, nullptr, nullptr, nullptr, r, zero2, 0.0, 0.0, s));
    } else {
        CK(launch_consume2<T>(EPI_CHEB, n, A[(m - 1) % 3], b, v.dinv, Dv[cur], X[cur], Dv[0], X[0], zero2, c1[deg - 1],
                              c2[deg - 1], s));
    }
    return STOKES_OK;
}

template <typename T>
stokes_status coarse_solve(stokes_ctx* c, const T* b, T* x, cudaStream_t s) {
    Level& L0 = c->lev[0];
    CK(cudaMemsetAsync(x, 0, L0.g.n_u * sizeof(T), s));
    CK(launch_coarse_solve<T>(c->nf, c->free_idx, c->Ainv, b, x, s));
    return STOKES_OK;
}

// x_l = V_l(b_l) with zero initial guess, level buffers.
template <typename T>
stokes_status vcycle_level(stokes_ctx* c, int l, cudaStream_t s) {
    Level& L = c->lev[l];
    LevelVecs<T>& v = vecs<T>(L);
    if (l == 0) return coarse_solve<T>(c, v.b, v.x, s);
    LevelVecs<T>& vc = vecs<T>(c->lev[l - 1]);
    const bool fused = fused_level<T>(c, l);
    if (fused) {
        CKS(smooth_fused<T>(c, l, v.b, v.x, true, v.r, s));   // pre-smoothing and its residual
        CK(launch_restrict<T>(L.g, v.r, vc.b, s));
    } else {
        CKS(smooth<T>(c, l, v.b, v.x, true, s));
        // the residual in a pass of its own: forming it inside the restriction (reading b and the
        // accumulator at every owned fine node and clearing it there) measured slower at 64^3 and
        // 128^3 (V-cycle 890 vs 865 us, 5.25 vs 5.19 ms)
        const int kern = level_kernel<T>(c, l);
        CK(launch_level_op<T>(kern, L.g, L.planes, EPI_RESID, v.mu, v.x, v.r, v.b, nullptr, nullptr, 0.0, 0.0,
                              slots<T>(L), v.acc, s, &c->tc));
        CK(launch_restrict<T>(L.g, v.r, vc.b, s, kern == 1));   // the brick operator's cycle stays deterministic
    }
    CKS(vcycle_level<T>(c, l - 1, s));
    CK(launch_prolongate<T>(L.g, vc.x, v.x, true, s));
    if (fused) CKS(smooth_fused<T>(c, l, v.b, v.x, false, nullptr, s));
    else CKS(smooth<T>(c, l, v.b, v.x, false, s));
    return STOKES_OK;
}

// The level recursion of one V-cycle. It touches only the context's level buffers, so it is
// captured once per precision as a CUDA graph and replayed on the library stream (ordered
// after and before the caller's stream by events). Profiling runs it launch by launch.
template <typename T>
stokes_status run_levels(stokes_ctx* c, cudaStream_t s) {
    if (!c->opt.graphs || prof_enabled()) return vcycle_level<T>(c, c->L - 1, s);
    const int p = sizeof(T) == 4 ? 1 : 0;
    if (!c->gstream) {
        CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->gev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->gev_out, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(c->gev_in, s));
    CK(cudaStreamWaitEvent(c->gstream, c->gev_in, 0));
    if (!c->gexec[p]) {
        cudaGraph_t graph = nullptr;
        const long long before = launch_total();
        CK(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
        stokes_status st = vcycle_level<T>(c, c->L - 1, c->gstream);
        cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
        if (st != STOKES_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CK(e);
        e = cudaGraphInstantiate(&c->gexec[p], graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        c->glaunches[p] = launch_total() - before;
    }
    CK(cudaGraphLaunch(c->gexec[p], c->gstream));
    prof_count(int(c->glaunches[p]));
    CK(cudaEventRecord(c->gev_out, c->gstream));
    CK(cudaStreamWaitEvent(s, c->gev_out, 0));
    return STOKES_OK;
}

template <typename T>
stokes_status vcycle(stokes_ctx* c, const T* rhs, T* x, cudaStream_t s) {
    Level& F = c->lev[c->L - 1];
    LevelVecs<T>& v = vecs<T>(F);
    CK(cudaMemcpyAsync(v.b, rhs, F.g.n_u * sizeof(T), cudaMemcpyDeviceToDevice, s));
    CK(launch_zero_boundary<T>(F.g, v.b, s));
    CKS(run_levels<T>(c, s));
    CK(cudaMemcpyAsync(x, v.x, F.g.n_u * sizeof(T), cudaMemcpyDeviceToDevice, s));
    CK(launch_copy_boundary<T>(F.g, rhs, x, s));
    return STOKES_OK;
}

// ---------------------------------------------------------------- octree meshes
// Local smoothing (Section 2.2.1 by citation): level li (0 = coarsest) holds all cells of its
// refinement level; edge nodes are ordinary rows and columns of A_li but are never smoothed
// (D^-1 = 0 there), boundary nodes are identity rows.

size_t active_nu(const stokes_ctx* c) { return c->oct ? 3 * c->oct->act.nu_nodes : c->lev[c->L - 1].g.n_u; }
size_t active_np(const stokes_ctx* c) { return c->oct ? c->oct->act.np : c->lev[c->L - 1].g.n_p; }

// dst = A_li src (boundary rows: identity; boundary entries of src ignored).
template <typename T>
stokes_status oct_vmult_level(stokes_ctx* c, int li, const T* src, T* dst, cudaStream_t s) {
    OctLevel& L = c->oct->lev[li];
    CK(cudaMemsetAsync(dst, 0, 3 * L.g.nn * sizeof(T), s));
    CK(launch_oct_level_cells<T>(L.g, ovecs<T>(L).mu, src, dst, s));
    CK(launch_oct_copy_boundary<T>(L.g, src, dst, s));
    return STOKES_OK;
}

template <typename T>
stokes_status oct_smooth(stokes_ctx* c, int li, const T* b, T* x, bool zero_guess, cudaStream_t s) {
    OctLevel& L = c->oct->lev[li];
    LevelVecs<T>& v = ovecs<T>(L);
    const double theta = 0.5 * (L.hi + L.lo), delta = 0.5 * (L.hi - L.lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    const size_t n = 3 * L.g.nn;
    auto step = [&](double c1, double c2) -> stokes_status {
        CK(launch_oct_level_cells<T>(L.g, v.mu, x, v.acc, s));
        CK(launch_consume<T>(2, n, v.acc, b, v.dinv, v.d, x, c1, c2, s));
        return STOKES_OK;
    };
    if (zero_guess) {
        CK(launch_cheb_update<T>(n, b, nullptr, v.dinv, v.d, x, 0.0, 1.0 / theta, false, s));
    } else {
        CKS(step(0.0, 1.0 / theta));
    }
    for (int it = 1; it < c->opt.cheb_degree; ++it) {
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        CKS(step(rho_new * rho, 2.0 * rho_new / delta));
        rho = rho_new;
    }
    return STOKES_OK;
}

template <typename T>
stokes_status oct_vcycle_level(stokes_ctx* c, int li, cudaStream_t s) {
    OctLevel& L = c->oct->lev[li];
    LevelVecs<T>& v = ovecs<T>(L);
    if (li == 0) {
        CK(cudaMemsetAsync(v.x, 0, 3 * L.g.nn * sizeof(T), s));
        CK(launch_coarse_solve<T>(c->nf, c->free_idx, c->Ainv, v.b, v.x, s));
        return STOKES_OK;
    }
    OctLevel& C = c->oct->lev[li - 1];
    CKS(oct_smooth<T>(c, li, v.b, v.x, true, s));
    CK(launch_oct_level_cells<T>(L.g, v.mu, v.x, v.acc, s));
    CK(launch_consume<T>(1, 3 * L.g.nn, v.acc, v.b, nullptr, nullptr, v.r, 0.0, 0.0, s));   // r = b - A x
    CK(launch_oct_restrict_add<T>(L.g, C.g, v.r, ovecs<T>(C).b, s));
    CKS(oct_vcycle_level<T>(c, li - 1, s));
    CK(launch_oct_prolongate<T>(L.g, C.g, ovecs<T>(C).x, v.x, true, s));
    CKS(oct_smooth<T>(c, li, v.b, v.x, false, s));
    return STOKES_OK;
}

// x = V(rhs) on the active velocity space (FP64 vectors, V-cycle arithmetic T); Dirichlet
// rows act as the identity.
template <typename T>
stokes_status oct_vcycle(stokes_ctx* c, const double* rhs, double* x, cudaStream_t s) {
    OctCtx& o = *c->oct;
    const size_t nu = o.act.nu_nodes;
    for (OctLevel& L : o.lev) {
        CK(cudaMemsetAsync(ovecs<T>(L).b, 0, 3 * L.g.nn * sizeof(T), s));
        CK(launch_oct_copy_to_level<T>(L.n_copy, L.copy_a, L.copy_l, nu, L.g.nn, rhs, ovecs<T>(L).b, L.g.dbg, s));
    }
    CKS(oct_vcycle_level<T>(c, int(o.lev.size()) - 1, s));
    for (OctLevel& L : o.lev)
        CK(launch_oct_copy_from_level<T>(L.n_copy, L.copy_a, L.copy_l, nu, L.g.nn, ovecs<T>(L).x, x, L.g.dbg, s));
    CK(launch_oct_identity_rows(o.act, rhs, x, s));
    return STOKES_OK;
}

stokes_status oct_schur_inverse(stokes_ctx* c, const double* rp, double* zp, cudaStream_t s) {
    const size_t np = c->oct->act.np;
    const double lo = 1.0 / 8.0, hi = 27.0 / 8.0;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    // degree 0: S_hat = diag(M_p) itself (Section 3.4); otherwise the first Chebyshev step
    const double c0 = c->opt.schur_degree == 0 ? 1.0 : 1.0 / theta;
    CK(launch_cheb_update<double>(np, rp, nullptr, c->mp_dinv, c->sp_d, zp, 0.0, c0, false, s));
    for (int it = 1; it < c->opt.schur_degree; ++it) {
        CK(launch_oct_mass_p(c->oct->act, zp, c->sp_t, s));
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        CK(launch_cheb_update<double>(np, rp, c->sp_t, c->mp_dinv, c->sp_d, zp, rho_new * rho, 2.0 * rho_new / delta,
                                      true, s));
        rho = rho_new;
    }
    return STOKES_OK;
}

stokes_status oct_precondition(stokes_ctx* c, int prec, const double* r, double* z, cudaStream_t s) {
    OctCtx& o = *c->oct;
    const size_t nu = 3 * o.act.nu_nodes, np = o.act.np;
    double* zp = z + nu;
    CKS(oct_schur_inverse(c, r + nu, zp, s));
    if (c->opt.precond_kind == 1) {   // P_D: z_p = S_hat^-1 r_p, z_u = A_hat^-1 r_u
        if (prec == STOKES_FP64) return oct_vcycle<double>(c, r, z, s);
        return oct_vcycle<float>(c, r, z, s);
    }
    CK(launch_axpby(np, -1.0, zp, 0.0, zp, s));                               // z_p = -S^-1 r_p
    CK(launch_oct_active(o.act, nullptr, zp, c->tu, nullptr, false, true, false, s));
    CK(launch_axpby(nu, 1.0, r, -1.0, c->tu, s));                            // t = r_u - B^T z_p
    if (prec == STOKES_FP64) return oct_vcycle<double>(c, c->tu, z, s);
    return oct_vcycle<float>(c, c->tu, z, s);
}

// z_p = S_hat^-1 r_p: Jacobi-Chebyshev on M_p, interval [1/8, 27/8], zero guess.
stokes_status schur_inverse(stokes_ctx* c, const double* rp, double* zp, cudaStream_t s) {
    if (c->oct) return oct_schur_inverse(c, rp, zp, s);
    const LevelGeom& g = c->lev[c->L - 1].g;
    const double lo = 1.0 / 8.0, hi = 27.0 / 8.0;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    // degree 0: S_hat = diag(M_p) itself (Section 3.4); otherwise the first Chebyshev step
    const int deg = c->opt.schur_degree;
    const double c0 = deg == 0 ? 1.0 : 1.0 / theta;
    // the later steps form M_p z per vertex and update in the same kernel, alternating between
    // (zp, sp_d) and (sp_z2, sp_d2); the first step starts in the pair the last one ends in zp
    double* Z[2] = {zp, c->sp_z2};
    double* D[2] = {c->sp_d, c->sp_d2};
    int cur = deg > 1 ? (deg - 1) & 1 : 0;
    CK(launch_cheb_update<double>(g.n_p, rp, nullptr, c->mp_dinv, D[cur], Z[cur], 0.0, c0, false, s));
    for (int it = 1; it < deg; ++it) {
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        CK(launch_schur_cheb(g, c->mp_scale, rp, c->mp_dinv, Z[cur], D[cur], Z[cur ^ 1], D[cur ^ 1], rho_new * rho,
                             2.0 * rho_new / delta, s));
        cur ^= 1;
        rho = rho_new;
    }
    return STOKES_OK;
}

// dst = K src. native: FP64 arithmetic whatever outer_arith says; the solvers use it for the
// residuals b - K x they restart from and report, so that the ~2^-47 relative rounding of the
// double-float operator (amplified by the viscosity contrast) enters only the Krylov recurrences,
// which the restarts correct like iterative refinement.
stokes_status apply_stokes(stokes_ctx* c, const double* src, double* dst, cudaStream_t s, bool native = false) {
    if (c->oct) {
        const size_t nu = 3 * c->oct->act.nu_nodes;
        CK(launch_oct_active(c->oct->act, src, src + nu, dst, dst + nu, true, true, true, s));
        return STOKES_OK;
    }
    Level& F = c->lev[c->L - 1];
    if (!native && c->opt.outer_arith == 2 && c->outer_tc_table) {   // exact digit slices on the tensor cores
        CK(cudaMemsetAsync(dst, 0, (F.g.n_u + F.g.n_p) * sizeof(double), s));
        CK(launch_outer_tc(F.g, F.v64.mu, src, src + F.g.n_u, dst, dst + F.g.n_u, c->outer_tc_table, c->tc.status,
                           c->tc.wait_ns, s));
        CK(launch_copy_boundary<double>(F.g, src, dst, s));   // identity rows
        return STOKES_OK;
    }
    if (native) prof_override(PROF_RESID_F64);
    const cudaError_t e = launch_stokes_blocks(F.g, F.v64.mu, src, src + F.g.n_u, dst, dst + F.g.n_u, true, true,
                                               true, c->opt.outer_arith >= 1 && !native, s);
    prof_override(-1);
    CK(e);
    return STOKES_OK;
}

// z = P^-1 r (eq. stokes_precond).
// Parts of the preconditioner for the batched driver (uniform meshes, FP32 V-cycle): PREC_PRE
// runs everything up to the right-hand side of the finest FP32 level, PREC_POST everything after
// the level recursion (which the batched kernel runs for many problems at once); PREC_ALL both
// with the recursion in between.
enum PrecPart { PREC_ALL = 0, PREC_PRE = 1, PREC_POST = 2 };

stokes_status precondition(stokes_ctx* c, int prec, const double* r, double* z, cudaStream_t s,
                           int part = PREC_ALL) {
    if (c->oct) return oct_precondition(c, prec, r, z, s);
    Level& F = c->lev[c->L - 1];
    const size_t nu = F.g.n_u, np = F.g.n_p;
    double* zp = z + nu;
    const double* rin = c->opt.precond_kind == 1 ? r : c->tu;   // the V-cycle's right-hand side
    if (part == PREC_POST) {   // the tail of vcycle<float>, then back to FP64
        CK(cudaMemcpyAsync(c->stage_out, F.v32.x, nu * sizeof(float), cudaMemcpyDeviceToDevice, s));
        CK(launch_copy_boundary<float>(F.g, c->stage_in, c->stage_out, s));
        CK(launch_cast_f2d(nu, c->stage_out, z, s));
        CK(launch_copy_boundary<double>(F.g, rin, z, s));
        return STOKES_OK;
    }
    CKS(schur_inverse(c, r + nu, zp, s));
    if (c->opt.precond_kind != 1) {
        CK(launch_axpby(np, -1.0, zp, 0.0, zp, s));                           // z_p = -S^-1 r_p
        CK(launch_stokes_blocks(F.g, F.v64.mu, nullptr, zp, c->tu, nullptr, false, true, false,
                                c->opt.outer_arith >= 1, s));
        CK(launch_axpby(nu, 1.0, r, -1.0, c->tu, s));                        // t = r_u - B^T z_p
    }   // else P_D: z_p = S_hat^-1 r_p, z_u = A_hat^-1 r_u
    if (prec == STOKES_FP64) return vcycle<double>(c, rin, z, s);
    CK(launch_cast_d2f(nu, rin, c->stage_in, s));
    if (part == PREC_PRE) {    // the head of vcycle<float>
        CK(cudaMemcpyAsync(F.v32.b, c->stage_in, nu * sizeof(float), cudaMemcpyDeviceToDevice, s));
        CK(launch_zero_boundary<float>(F.g, F.v32.b, s));
        return STOKES_OK;
    }
    CKS(vcycle<float>(c, c->stage_in, c->stage_out, s));
    CK(launch_cast_f2d(nu, c->stage_out, z, s));
    CK(launch_copy_boundary<double>(F.g, rin, z, s));
    return STOKES_OK;
}

stokes_status ensure_krylov(stokes_ctx* c) {
    const int m = c->opt.restart;
    if (c->V && c->krylov_restart == m) return STOKES_OK;
    c->N = active_nu(c) + active_np(c);
    c->ldv = c->N + (c->N & 1);   // even row stride: 16-byte aligned entry pairs (krylov.cu)
    CKS(dalloc(c, &c->V, size_t(m + 1) * c->ldv));
    // flexible GMRES keeps the m preconditioned vectors; GMRES (outer_solver 2) one work vector
    CKS(dalloc(c, &c->Z, c->opt.outer_solver == 2 ? c->ldv : size_t(m) * c->N));
    CKS(dalloc(c, &c->w, c->N));
    CKS(dalloc(c, &c->bvec, c->N));
    CKS(dalloc(c, &c->hdev, size_t(3 * (m + 4))));   // h1, and two step records of the delayed passes
    c->krylov_restart = m;
    return STOKES_OK;
}

stokes_status remove_pressure_mean(stokes_ctx* c, double* up, cudaStream_t s) {
    const size_t nu = active_nu(c), np = active_np(c);
    double wp = 0.0;
    CKS(dot(c, np, c->p_weights, up + nu, s, &wp));
    CK(launch_add_scalar(np, -wp / c->p_wsum, up + nu, s));
    return STOKES_OK;
}

// Right-preconditioned FGMRES(restart) as a resumable state machine: enqueue() issues one
// phase's kernels on the run's stream and a small device->host copy; complete() runs the host
// part once that stream has finished. One problem (stokes_solve) or many in lock step
// (stokes_batch_solve) use the same code.
// With flexible = false it is GMRES(restart) with a fixed preconditioner (outer_solver 2,
// Section 3.4): P^-1 V_j goes to one work vector instead of the stored Z_j, and a cycle ends with
// x += P^-1 (V y).
// The solve ends only when the true residual b - K x, recomputed in the final phase, meets the
// tolerance; otherwise a new cycle starts from it. The recurrence can run ahead of the true
// residual: with the FP32 V-cycle P^-1 (V y) differs slightly from the combination GMRES assumed,
// and at large sizes and viscosity contrasts rounding in K Z = V H lets FGMRES drift too.
struct FgmresRun {
    enum Phase { P_BNORM, P_RESTART, P_ITER, P_FINAL, P_DONE };
    stokes_ctx* c = nullptr;
    int prec = 0;
    const double* b = nullptr;
    double* x = nullptr;
    double rtol = 1e-8;
    int max_it = 1;
    cudaStream_t s = nullptr;
    stokes_solve_info* info = nullptr;
    Phase phase = P_BNORM;
    stokes_status st = STOKES_NOT_CONVERGED;
    int its = 0, j = 0, m = 0;
    double bnorm = 0.0, est = 1.0, hn_prev = 0.0;
    bool next_v = false;   // V_{j} = w / hn_prev still to be formed before iteration j
    bool flexible = true;
    bool lag = false;           // delayed re-orthogonalisation (two passes over V per step)
    double inv_sqrt_s = 1.0;    // 1 / |u_j| for the preconditioner input u_j / |u_j|
    bool force_cycle = false;   // the final check sent the run back: iterate at least once
    int verify_left = 10;       // such returns left
    bool batched = false;       // the batched driver runs the FP32 level recursion of P^-1
    int batch_stage = 0;        // 1: P_ITER stopped before the level recursion (pin, zj kept)
    const double* pin = nullptr;
    double* zj = nullptr;
    std::vector<double> H, cs, sn, g, y;
    double& Hij(int i, int jj) { return H[size_t(i) * m + jj]; }
};

// Batched driver: P_ITER runs the preconditioner up to the finest FP32 right-hand side and stops
// (batch_stage 1); the driver runs the level recursion of every such problem in one launch; the
// next enqueue resumes after it.
stokes_status fgmres_stop_before_levels(FgmresRun& r, const double* pin, double* zj) {
    CKS(precondition(r.c, r.prec, pin, zj, r.s, PREC_PRE));
    r.pin = pin;
    r.zj = zj;
    r.batch_stage = 1;
    return STOKES_OK;
}

stokes_status fgmres_resume_after_levels(FgmresRun& r) {
    CKS(precondition(r.c, r.prec, r.pin, r.zj, r.s, PREC_POST));
    r.batch_stage = 0;
    return STOKES_OK;
}

stokes_status fgmres_enqueue(FgmresRun& r) {
    stokes_ctx* c = r.c;
    const size_t N = c->N;
    const int m = r.m;
    cudaStream_t s = r.s;
    switch (r.phase) {
        case FgmresRun::P_BNORM:
            CK(launch_multidot(N, 1, r.b, N, r.b, c->partials, c->dots, s));
            CK(cudaMemcpyAsync(c->dots_host, c->dots, sizeof(double), cudaMemcpyDeviceToHost, s));
            return STOKES_OK;
        case FgmresRun::P_RESTART:
            CKS(apply_stokes(c, r.x, c->w, s, true));
            CK(launch_axpby(N, 1.0, r.b, -1.0, c->w, s));                              // w = b - K x
            CK(launch_multidot(N, 1, c->w, N, c->w, c->partials, c->dots, s));
            CK(cudaMemcpyAsync(c->dots_host, c->dots, sizeof(double), cudaMemcpyDeviceToHost, s));
            return STOKES_OK;
        case FgmresRun::P_ITER: {
            const int j = r.j;
            double* V = c->V;
            const size_t ldv = c->ldv;
            double* vj = V + size_t(j) * ldv;
            double* zj = r.flexible ? c->Z + size_t(j) * N : c->Z;
            if (r.lag) {
                // Delayed re-orthogonalisation: row j holds u_j, w of the previous step after one
                // projection; the preconditioner takes u_j / |u_j| (FGMRES allows any z_j: the
                // relation K z_j = V H e_j holds for the z_j used). Pass A: V^T w with the dot of
                // row j corrected on the device to v_j . w; pass B: writes the twice-projected
                // v_j over row j and u_{j+1} = w - V h to row j + 1, with the dots of the record.
                if (r.batch_stage == 0) {
                    if (r.next_v) CK(launch_df_store_scaled(N, c->w, 1.0 / r.hn_prev, vj, s));   // V_0
                    CK(launch_df_to_double(N, vj, c->w, s, j == 0 ? 1.0 : r.inv_sqrt_s));
                    if (r.batched) return fgmres_stop_before_levels(r, c->w, zj);
                    CKS(precondition(c, r.prec, c->w, zj, s));
                } else {
                    CKS(fgmres_resume_after_levels(r));
                }
                CKS(apply_stokes(c, zj, c->w, s));
                double* h1d = c->hdev;
                const double* prev = j > 0 ? c->hdev + size_t(m + 4) * (1 + (j & 1)) : nullptr;
                double* cur = c->hdev + size_t(m + 4) * (1 + ((j + 1) & 1));
                CK(launch_gs_dot_lag(N, j + 1, V, ldv, c->w, c->partials, h1d, prev, s));
                CK(launch_gs_lag_project(N, j + 1, V, ldv, h1d, prev, c->w, c->partials, cur, s));
                CK(cudaMemcpyAsync(c->dots_host, c->hdev, size_t(3 * (m + 4)) * sizeof(double), cudaMemcpyDeviceToHost, s));
                return STOKES_OK;
            }
            const bool df = c->opt.outer_arith >= 1 && m <= gs_max_k();   // V as double-float pairs (krylov.cu)
            if (r.batch_stage == 1) {
                CKS(fgmres_resume_after_levels(r));
            } else if (df) {
                if (r.next_v) CK(launch_df_store_scaled(N, c->w, 1.0 / r.hn_prev, vj, s));   // V_j = w / |w|
                CK(launch_df_to_double(N, vj, c->w, s));
                if (r.batched) return fgmres_stop_before_levels(r, c->w, zj);
                CKS(precondition(c, r.prec, c->w, zj, s));
            } else {
                if (r.next_v) CK(launch_axpby(N, 1.0 / r.hn_prev, c->w, 0.0, vj, s));
                if (r.batched) return fgmres_stop_before_levels(r, vj, zj);
                CKS(precondition(c, r.prec, vj, zj, s));
            }
            CKS(apply_stokes(c, zj, c->w, s));
            // classical Gram-Schmidt applied twice ("twice is enough") in three passes over V:
            // h1 = V^T w; w1 = w - V h1 with h2 = V^T w1 and |w1|^2 in the same sweep;
            // V_{j+1} = (w1 - V h2) / hn with hn = sqrt(|w1|^2 - |h2|^2) computed on the device
            // (no cancellation: h2 is small after the first pass). The last vector of a cycle is
            // not needed (the restart recomputes the residual).
            double* h1d = c->hdev;
            double* h2d = c->hdev + (m + 4);
            CK(launch_gs_dot(N, j + 1, V, ldv, c->w, c->partials, h1d, df, s));
            CK(launch_gs_project_dot(N, j + 1, V, ldv, h1d, c->w, c->partials, h2d, df, s));
            if (j + 1 < m) CK(launch_gs_project_scale(N, j + 1, V, ldv, h2d, c->w, h2d + j + 3, vj + ldv, df, s));
            CK(cudaMemcpyAsync(c->dots_host, c->hdev, size_t(2 * (m + 4)) * sizeof(double), cudaMemcpyDeviceToHost, s));
            return STOKES_OK;
        }
        case FgmresRun::P_FINAL:
            CKS(remove_pressure_mean(c, r.x, s));   // synchronous (one dot)
            CKS(apply_stokes(c, r.x, c->w, s, true));
            CK(launch_axpby(N, 1.0, r.b, -1.0, c->w, s));
            CK(launch_multidot(N, 1, c->w, N, c->w, c->partials, c->dots, s));
            CK(cudaMemcpyAsync(c->dots_host, c->dots, sizeof(double), cudaMemcpyDeviceToHost, s));
            return STOKES_OK;
        case FgmresRun::P_DONE:
            return STOKES_OK;
    }
    return STOKES_OK;
}

// x += Z y for the finished cycle (y from the upper-triangular solve on the host); without the
// stored Z: x += P^-1 (V y), with V y formed in w (double-float V: by the projection pass with
// w = 0 and coefficients -y into the free basis row V_k, then converted to FP64).
stokes_status fgmres_update_x(FgmresRun& r, int k) {
    stokes_ctx* c = r.c;
    const size_t N = c->N;
    for (int i = k - 1; i >= 0; --i) {
        double t = r.g[i];
        for (int l = i + 1; l < k; ++l) t -= r.Hij(i, l) * r.y[l];
        r.y[i] = t / r.Hij(i, i);
    }
    if (r.flexible) {
        CK(cudaMemcpyAsync(c->hdev, r.y.data(), size_t(k) * sizeof(double), cudaMemcpyHostToDevice, r.s));
        CK(launch_multiaxpy(N, k, c->Z, N, c->hdev, r.x, 1.0, r.s));
    } else {
        const bool df = c->opt.outer_arith >= 1 && r.m <= gs_max_k();
        CK(cudaMemsetAsync(c->w, 0, N * sizeof(double), r.s));
        if (df) {
            for (int i = 0; i < k; ++i) r.y[i] = -r.y[i];
            r.y[k] = 1.0;                                                          // scale
            CK(cudaMemcpyAsync(c->hdev, r.y.data(), size_t(k + 1) * sizeof(double), cudaMemcpyHostToDevice, r.s));
            double* vk = c->V + size_t(k) * c->ldv;                               // unused after the cycle
            CK(launch_gs_project_scale(N, k, c->V, c->ldv, c->hdev, c->w, c->hdev + k, vk, true, r.s));
            CK(launch_df_to_double(N, vk, c->w, r.s));
        } else {
            CK(cudaMemcpyAsync(c->hdev, r.y.data(), size_t(k) * sizeof(double), cudaMemcpyHostToDevice, r.s));
            CK(launch_multiaxpy(N, k, c->V, c->ldv, c->hdev, c->w, 1.0, r.s));
        }
        CKS(precondition(c, r.prec, c->w, c->Z, r.s));
        CK(launch_axpby(N, 1.0, c->Z, 1.0, r.x, r.s));
    }
    CK(cudaStreamSynchronize(r.s));   // r.y is pageable host memory
    return STOKES_OK;
}

// Host part of the phase just finished (the run's stream is idle); chooses the next phase.
stokes_status fgmres_complete(FgmresRun& r) {
    stokes_ctx* c = r.c;
    const int m = r.m;
    const double* hd = c->dots_host;
    switch (r.phase) {
        case FgmresRun::P_BNORM:
            r.bnorm = std::sqrt(hd[0]);
            if (r.bnorm == 0.0) {
                CK(cudaMemsetAsync(r.x, 0, c->N * sizeof(double), r.s));
                r.est = 0.0;
                r.st = STOKES_OK;
                r.phase = FgmresRun::P_FINAL;
            } else {
                r.phase = FgmresRun::P_RESTART;
            }
            return STOKES_OK;
        case FgmresRun::P_RESTART: {
            const double beta = std::sqrt(hd[0]);
            if (!std::isfinite(beta)) { r.st = STOKES_BREAKDOWN; r.phase = FgmresRun::P_FINAL; return STOKES_OK; }
            r.est = beta / r.bnorm;
            if (beta <= r.rtol * r.bnorm && !r.force_cycle) {
                r.st = STOKES_OK;
                r.phase = FgmresRun::P_FINAL;
                return STOKES_OK;
            }
            r.force_cycle = false;
            if (r.its >= r.max_it) { r.phase = FgmresRun::P_FINAL; return STOKES_OK; }
            std::fill(r.g.begin(), r.g.end(), 0.0);
            r.g[0] = beta;
            r.j = 0;
            r.hn_prev = beta;      // V_0 = (b - K x) / beta
            r.next_v = true;
            r.phase = FgmresRun::P_ITER;
            return STOKES_OK;
        }
        case FgmresRun::P_ITER: {
            const int j = r.j;
            double hn = 0.0;
            if (r.lag) {
                const double* rec = hd + size_t(m + 4) * (1 + ((j + 1) & 1));
                for (int i = 0; i <= j; ++i) r.Hij(i, j) = hd[i] + rec[i];
                hn = rec[j + 2];                              // |u_{j+1} - V c|
                r.inv_sqrt_s = 1.0 / std::sqrt(rec[j + 1]);
            } else {
                for (int i = 0; i <= j; ++i) r.Hij(i, j) = hd[i] + hd[m + 4 + i];
                hn = hd[m + 4 + j + 2];   // the norm V_{j+1} was scaled with
            }
            if (!std::isfinite(hn)) { r.st = STOKES_BREAKDOWN; r.phase = FgmresRun::P_FINAL; return STOKES_OK; }
            r.Hij(j + 1, j) = hn;
            for (int i = 0; i < j; ++i) {
                const double t = r.cs[i] * r.Hij(i, j) + r.sn[i] * r.Hij(i + 1, j);
                r.Hij(i + 1, j) = -r.sn[i] * r.Hij(i, j) + r.cs[i] * r.Hij(i + 1, j);
                r.Hij(i, j) = t;
            }
            const double den = std::hypot(r.Hij(j, j), r.Hij(j + 1, j));
            r.cs[j] = r.Hij(j, j) / den;
            r.sn[j] = r.Hij(j + 1, j) / den;
            r.Hij(j, j) = den;
            r.Hij(j + 1, j) = 0.0;
            r.g[j + 1] = -r.sn[j] * r.g[j];
            r.g[j] = r.cs[j] * r.g[j];
            ++r.its;
            r.est = std::fabs(r.g[j + 1]) / r.bnorm;
            const bool conv = std::fabs(r.g[j + 1]) <= r.rtol * r.bnorm || hn == 0.0;
            if (conv || j + 1 == m || r.its >= r.max_it) {
                CKS(fgmres_update_x(r, j + 1));
                if (conv) { r.st = STOKES_OK; r.phase = FgmresRun::P_FINAL; }
                else if (r.its >= r.max_it) r.phase = FgmresRun::P_FINAL;
                else r.phase = FgmresRun::P_RESTART;
            } else {
                r.next_v = false;   // V_{j+1} was formed on the device
                r.j = j + 1;
            }
            return STOKES_OK;
        }
        case FgmresRun::P_FINAL: {
            const double rt = std::sqrt(hd[0]);
            if (r.st == STOKES_OK && r.bnorm > 0.0 && rt > r.rtol * r.bnorm && r.its < r.max_it && r.verify_left > 0) {
                --r.verify_left;
                r.force_cycle = true;
                r.st = STOKES_NOT_CONVERGED;   // the recurrence ran ahead: continue from b - K x
                r.phase = FgmresRun::P_RESTART;
                return STOKES_OK;
            }
            // the status follows the true residual, whatever ended the iteration (max_it, the
            // recurrence, or no verification returns left); only a breakdown keeps its own status
            if (r.st != STOKES_BREAKDOWN && r.bnorm > 0.0)
                r.st = rt <= r.rtol * r.bnorm ? STOKES_OK : STOKES_NOT_CONVERGED;
            if (r.info) {
                r.info->iterations = r.its;
                r.info->rel_residual = r.est;
                r.info->rel_residual_true = r.bnorm > 0 ? rt / r.bnorm : 0.0;
                r.info->status = r.st;
            }
            r.phase = FgmresRun::P_DONE;
            return STOKES_OK;
        }
        case FgmresRun::P_DONE:
            return STOKES_OK;
    }
    return STOKES_OK;
}

stokes_status fgmres_init(FgmresRun& r, stokes_ctx* c, int prec, const double* b, double* x, double rtol,
                          int max_it, stokes_solve_info* info, cudaStream_t s) {
    CKS(ensure_krylov(c));
    r.c = c;
    r.prec = prec;
    r.b = b;
    r.x = x;
    r.rtol = rtol;
    r.max_it = max_it;
    r.s = s;
    r.info = info;
    r.m = c->opt.restart;
    r.flexible = c->opt.outer_solver != 2;
    r.lag = r.flexible && c->opt.gram_schmidt == 1 && c->opt.outer_arith >= 1 && r.m <= gs_max_k();
    r.H.assign(size_t(r.m + 1) * r.m, 0.0);
    r.cs.assign(r.m, 0.0);
    r.sn.assign(r.m, 0.0);
    r.g.assign(r.m + 1, 0.0);
    r.y.assign(r.m + 1, 0.0);
    r.phase = FgmresRun::P_BNORM;
    return STOKES_OK;
}

// Advance all runs in lock step until every one is done (one host synchronisation per run per round).
stokes_status fgmres_drive(std::vector<FgmresRun>& runs) {
    bool active = true;
    while (active) {
        active = false;
        for (FgmresRun& r : runs)
            if (r.phase != FgmresRun::P_DONE) CKS(fgmres_enqueue(r));
        for (FgmresRun& r : runs) {
            if (r.phase == FgmresRun::P_DONE) continue;
            CK(cudaStreamSynchronize(r.s));
            CKS(fgmres_complete(r));
            if (r.phase != FgmresRun::P_DONE) active = true;
        }
    }
    return STOKES_OK;
}

// Device state of the batched V-cycle: the problems' level tables, the phase list and per-phase
// tile offsets of the work queue (rebuilt each round for the problems that take part), the queue
// counters, the mask of those problems, the status word; a stream for the launch and events that
// order it with the problems' streams.
struct BatchVcycle {
    std::vector<void*> mem;
    BatchLaunch bl{};
    std::vector<BatchProblem> probs;   // host copy (sizes for the tile counts)
    std::vector<int> levels;
    int degree = 0, max_phases = 0;
    int* active_host = nullptr;          // pinned, with the round's phases and tile offsets
    BatchPhase* phases_host = nullptr;
    unsigned* prefix_host = nullptr;
    int* active_dev = nullptr;
    BatchPhase* phases_dev = nullptr;
    unsigned* prefix_dev = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev_out = nullptr;
    std::vector<cudaEvent_t> ev_in;
    ~BatchVcycle() {
        for (cudaEvent_t e : ev_in) cudaEventDestroy(e);
        if (ev_out) cudaEventDestroy(ev_out);
        if (s) cudaStreamDestroy(s);
        for (void* h : {static_cast<void*>(active_host), static_cast<void*>(phases_host),
                        static_cast<void*>(prefix_host)})
            if (h) cudaFreeHost(h);
        for (void* p : mem) cudaFree(p);
    }
    template <typename T>
    stokes_status upload(T** dev, const T* host, size_t count) {
        void* p = nullptr;
        CK(cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16)));
        mem.push_back(p);
        if (host && count) CK(cudaMemcpy(p, host, count * sizeof(T), cudaMemcpyHostToDevice));
        *dev = static_cast<T*>(p);
        return STOKES_OK;
    }
};

// Rounds with fewer problems at their preconditioner than this replay each problem's own captured
// V-cycle graph instead (a launch with few items still pays every grid barrier).
constexpr int kBatchKernelMinProblems = 8;

// True if the runs can share one batched V-cycle launch: FP32 V-cycles of uniform meshes inside
// FGMRES, one smoother degree, supported level counts, a device that runs cooperative launches.
bool batch_vcycle_eligible(const std::vector<FgmresRun>& runs) {
    if (runs.empty() || runs[0].prec != STOKES_FP32 || runs[0].c->opt.batch_vcycle != 1) return false;
    const int deg = runs[0].c->opt.cheb_degree;
    if (deg > kBatchMaxDegree) return false;
    for (const FgmresRun& r : runs)
        if (r.c->oct || !r.flexible || r.c->L > kBatchMaxLevels || r.c->opt.cheb_degree != deg) return false;
    return batch_grid_blocks() > 0;
}

stokes_status batch_vcycle_setup(BatchVcycle& B, const std::vector<FgmresRun>& runs) {
    const int P = int(runs.size());
    const int deg = runs[0].c->opt.cheb_degree;
    B.degree = deg;
    B.probs.assign(P, BatchProblem{});
    B.levels.assign(P, 0);
    double wait_s = 1e6;
    for (int p = 0; p < P; ++p) {
        stokes_ctx* c = runs[p].c;
        BatchProblem& bp = B.probs[p];
        bp.L = c->L;
        bp.nf = c->nf;
        bp.free_idx = c->free_idx;
        bp.Ainv = c->Ainv;
        for (int l = 0; l < c->L; ++l) {
            const Level& Lv = c->lev[l];
            BatchLevel& bl = bp.lev[l];
            bl.n = Lv.g.n;
            bl.M = Lv.g.M;
            bl.nodes = Lv.g.nodes;
            bl.n_u = Lv.g.n_u;
            bl.h = float(Lv.g.h);
            bl.mu = Lv.v32.mu;
            bl.dinv = Lv.v32.dinv;
            bl.b = Lv.v32.b;
            bl.x = Lv.v32.x;
            bl.r = Lv.v32.r;
            bl.d = Lv.v32.d;
            bl.acc = Lv.v32.acc;
            // the coefficients smooth() uses: step 0 (0, 1/theta), then the three-term recurrence
            const double theta = 0.5 * (Lv.hi + Lv.lo), delta = 0.5 * (Lv.hi - Lv.lo), sigma = theta / delta;
            double rho = 1.0 / sigma;
            bl.c1[0] = 0.0f;
            bl.c2[0] = float(1.0 / theta);
            for (int k = 1; k < deg; ++k) {
                const double rho_new = 1.0 / (2.0 * sigma - rho);
                bl.c1[k] = float(rho_new * rho);
                bl.c2[k] = float(2.0 * rho_new / delta);
                rho = rho_new;
            }
        }
        B.levels[p] = c->L;
        wait_s = std::min(wait_s, c->opt.wait_limit_s);
    }
    // every round's phase list (a subset of the problems) is no longer than the full batch's
    B.max_phases = batch_build_phases(B.levels.data(), P, deg, nullptr, 0);
    BatchProblem* dprob = nullptr;
    unsigned* dctr = nullptr;
    unsigned* dstatus = nullptr;
    CKS(B.upload(&dprob, B.probs.data(), size_t(P)));
    CKS(B.upload(&B.phases_dev, static_cast<const BatchPhase*>(nullptr), size_t(B.max_phases)));
    CKS(B.upload(&B.prefix_dev, static_cast<const unsigned*>(nullptr), size_t(B.max_phases) * (P + 1)));
    CKS(B.upload(&dctr, static_cast<const unsigned*>(nullptr), size_t(B.max_phases + 2)));
    CKS(B.upload(&dstatus, static_cast<const unsigned*>(nullptr), 1));
    CK(cudaMemset(dstatus, 0, sizeof(unsigned)));
    CKS(B.upload(&B.active_dev, static_cast<const int*>(nullptr), size_t(P)));
    CK(cudaMallocHost(reinterpret_cast<void**>(&B.active_host), sizeof(int) * P));
    CK(cudaMallocHost(reinterpret_cast<void**>(&B.phases_host), sizeof(BatchPhase) * B.max_phases));
    CK(cudaMallocHost(reinterpret_cast<void**>(&B.prefix_host), sizeof(unsigned) * B.max_phases * (P + 1)));
    CK(cudaStreamCreateWithFlags(&B.s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&B.ev_out, cudaEventDisableTiming));
    B.ev_in.resize(P, nullptr);
    for (cudaEvent_t& e : B.ev_in) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    B.bl = BatchLaunch{dprob, P, B.phases_dev, 0, B.prefix_dev, dctr, B.active_dev, dstatus,
                       (unsigned long long)(wait_s * 1e9)};
    return STOKES_OK;
}

// Phase list and tile offsets of one round for the problems in the mask (pinned host buffers,
// copied on the batch stream); returns the number of tiles of the largest phase.
stokes_status batch_vcycle_round(BatchVcycle& B, unsigned* widest) {
    const int P = int(B.probs.size());
    std::vector<int> lv;
    for (int p = 0; p < P; ++p)
        if (B.active_host[p]) lv.push_back(B.levels[p]);
    const int nph = batch_build_phases(lv.data(), int(lv.size()), B.degree, B.phases_host, B.max_phases);
    if (nph > B.max_phases) return fail(STOKES_ECUDA, "batched V-cycle: phase list overflow");
    *widest = 0;
    for (int i = 0; i < nph; ++i) {
        const size_t per_tile = size_t(kBatchThreads) * batch_items_per_thread(B.phases_host[i].op);
        unsigned t = 0;
        unsigned* pre = B.prefix_host + size_t(i) * (P + 1);
        for (int p = 0; p < P; ++p) {
            pre[p] = t;
            if (!B.active_host[p]) continue;
            const size_t tiles = (batch_items(B.probs[p], B.phases_host[i]) + per_tile - 1) / per_tile;
            if (size_t(t) + tiles > 0xFFFFFFF0u) return fail(STOKES_EINVAL, "batch too large for the work queue");
            *widest = std::max(*widest, unsigned(tiles));
            t += unsigned(tiles);
        }
        pre[P] = t;
        *widest = std::max(*widest, t);
    }
    B.bl.n_phases = nph;
    CK(cudaMemcpyAsync(B.active_dev, B.active_host, sizeof(int) * P, cudaMemcpyHostToDevice, B.s));
    CK(cudaMemcpyAsync(B.phases_dev, B.phases_host, sizeof(BatchPhase) * nph, cudaMemcpyHostToDevice, B.s));
    CK(cudaMemcpyAsync(B.prefix_dev, B.prefix_host, sizeof(unsigned) * size_t(nph) * (P + 1),
                       cudaMemcpyHostToDevice, B.s));
    return STOKES_OK;
}

// Lock-step FGMRES of all runs. In a round where at least kBatchKernelMinProblems runs reached
// their preconditioner, one batched V-cycle launch runs all of their level recursions; in other
// rounds each replays its own captured V-cycle graph on its stream. Returns TIMEOUT if a grid
// barrier of the batched kernel gave up.
stokes_status fgmres_drive_batched(std::vector<FgmresRun>& runs, BatchVcycle& B) {
    const int P = int(runs.size());
    bool active = true;
    while (active) {
        active = false;
        for (FgmresRun& r : runs)
            if (r.phase != FgmresRun::P_DONE) CKS(fgmres_enqueue(r));
        int count = 0;
        for (int p = 0; p < P; ++p) {
            B.active_host[p] = runs[p].phase != FgmresRun::P_DONE && runs[p].batch_stage == 1;
            count += B.active_host[p];
        }
        if (count >= kBatchKernelMinProblems) {
            unsigned widest = 0;
            CKS(batch_vcycle_round(B, &widest));
            for (int p = 0; p < P; ++p)
                if (B.active_host[p]) {
                    CK(cudaEventRecord(B.ev_in[p], runs[p].s));
                    CK(cudaStreamWaitEvent(B.s, B.ev_in[p], 0));
                }
            CK(launch_batch_vcycle(B.bl, int(widest), B.s));
            CK(cudaEventRecord(B.ev_out, B.s));
            for (int p = 0; p < P; ++p)
                if (B.active_host[p]) {
                    CK(cudaStreamWaitEvent(runs[p].s, B.ev_out, 0));
                    CKS(fgmres_enqueue(runs[p]));   // resumes after the level recursion
                }
            // the pinned round buffers are rewritten next round: their copies must have run
            CK(cudaStreamSynchronize(B.s));
        } else if (count > 0) {
            for (int p = 0; p < P; ++p)
                if (B.active_host[p]) {
                    CKS(run_levels<float>(runs[p].c, runs[p].s));
                    CKS(fgmres_enqueue(runs[p]));
                }
        }
        for (FgmresRun& r : runs) {
            if (r.phase == FgmresRun::P_DONE) continue;
            CK(cudaStreamSynchronize(r.s));
            CKS(fgmres_complete(r));
            if (r.phase != FgmresRun::P_DONE) active = true;
        }
    }
    unsigned w = 0;
    CK(cudaMemcpy(&w, B.bl.status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (w != 0) return fail(STOKES_TIMEOUT, "a grid barrier of the batched V-cycle gave up (wait_limit_s)");
    return STOKES_OK;
}

stokes_status fgmres(stokes_ctx* c, int prec, const double* b, double* x, double rtol, int max_it,
                     stokes_solve_info* info, cudaStream_t s) {
    std::vector<FgmresRun> runs(1);
    stokes_solve_info local{};
    CKS(fgmres_init(runs[0], c, prec, b, x, rtol, max_it, info ? info : &local, s));
    CKS(fgmres_drive(runs));
    const stokes_status st = runs[0].st;
    if (st != STOKES_OK) return fail(st, st == STOKES_BREAKDOWN ? "(F)GMRES breakdown (non-finite norm)"
                                                                 : "(F)GMRES: true residual above rtol (max_it or restarts used up)");
    return STOKES_OK;
}

// ---------------------------------------------------------------- IDR(s)
// The memory-light outer solver of Section 3.4: IDR(s) with bi-orthogonalisation and right
// preconditioning by P^-1 (M. B. van Gijzen, P. Sonneveld, ACM TOMS 38 (2011), Alg. 913), omega
// by "maintaining the convergence" (kappa = 0.7). 3s + 4 vectors of N instead of FGMRES's 2 m + 1.
// The shadow space: splitmix64 uniforms u01 - 1/2 with seeds 1907100 + i, orthonormalised.
// Iterations count preconditioned operator applications, as for FGMRES.
stokes_status ensure_idr(stokes_ctx* c, int sdim) {
    c->N = active_nu(c) + active_np(c);
    const size_t N = c->N;
    if (c->idr_alloc_s < sdim) {
        CKS(dalloc(c, &c->idr_G, size_t(sdim) * N));
        CKS(dalloc(c, &c->idr_U, size_t(sdim) * N));
        CKS(dalloc(c, &c->idr_P, size_t(sdim) * N));
        if (!c->idr_r) {
            for (double** q : {&c->idr_r, &c->idr_v, &c->idr_t, &c->idr_tmp}) CKS(dalloc(c, q, N));
            CKS(dalloc(c, &c->idr_c, 16));
        }
        c->idr_alloc_s = sdim;
    }
    if (!c->bvec) CKS(dalloc(c, &c->bvec, N));
    // shadow space (rebuilt every solve: cheap, and independent of earlier calls)
    for (int i = 0; i < sdim; ++i) {
        double* pi = c->idr_P + size_t(i) * N;
        CK(launch_splitmix_vector(N, uint64_t(1907100 + i), nullptr, pi, c->idr_stream));
        for (int j = 0; j < i; ++j) {
            double d = 0.0;
            CKS(dot(c, N, c->idr_P + size_t(j) * N, pi, c->idr_stream, &d));
            CK(launch_axpby(N, -d, c->idr_P + size_t(j) * N, 1.0, pi, c->idr_stream));
        }
        double nn = 0.0;
        CKS(dot(c, N, pi, pi, c->idr_stream, &nn));
        CK(launch_axpby(N, 1.0 / std::sqrt(nn), pi, 0.0, pi, c->idr_stream));
    }
    return STOKES_OK;
}

stokes_status idr_solve(stokes_ctx* c, int prec, const double* b, double* x, double rtol, int max_it,
                        stokes_solve_info* info, cudaStream_t s) {
    const int sd = c->opt.idr_s;   // workspace and shadow space: ensure_idr (stokes_solve)
    const size_t N = c->N;
    double *G = c->idr_G, *U = c->idr_U, *P = c->idr_P, *r = c->idr_r, *v = c->idr_v, *t = c->idr_t,
           *tmp = c->idr_tmp;
    auto col = [&](double* A, int i) { return A + size_t(i) * N; };
    double bnorm2 = 0.0;
    CKS(dot(c, N, b, b, s, &bnorm2));
    const double bnorm = std::sqrt(bnorm2);
    stokes_status st = STOKES_NOT_CONVERGED;
    int its = 0;
    double rnorm = 0.0;
    if (bnorm == 0.0) {
        CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        st = STOKES_OK;
    } else {
      // passes: IDR(s) from r = b - K x; a new pass starts when the recursively updated residual met
      // the tolerance but the true one did not (at most 10 restarts)
      const double tol = rtol * bnorm;
      for (int pass = 0; pass < 11; ++pass) {
        CKS(apply_stokes(c, x, r, s, true));
        CK(launch_axpby(N, 1.0, b, -1.0, r, s));                              // r = b - K x
        double rr = 0.0;
        CKS(dot(c, N, r, r, s, &rr));
        rnorm = std::sqrt(rr);
        if (!std::isfinite(rnorm)) { st = STOKES_BREAKDOWN; break; }
        if (rnorm <= tol) { st = STOKES_OK; break; }
        if (its >= max_it) { st = STOKES_NOT_CONVERGED; break; }
        st = STOKES_NOT_CONVERGED;
        CK(cudaMemsetAsync(G, 0, size_t(sd) * N * sizeof(double), s));
        CK(cudaMemsetAsync(U, 0, size_t(sd) * N * sizeof(double), s));
        std::vector<double> Ms(size_t(sd) * sd, 0.0), f(sd), cc(sd), dots(sd + 1);
        for (int i = 0; i < sd; ++i) Ms[size_t(i) * sd + i] = 1.0;
        auto M = [&](int i, int j) -> double& { return Ms[size_t(i) * sd + j]; };
        double om = 1.0;
        auto multidot = [&](int k, const double* V, const double* w, double* out) -> stokes_status {
            CK(launch_multidot(N, k, V, N, w, c->partials, c->dots, s));
            return fetch(c, k, s, out);
        };
        bool done = false;
        while (!done && its < max_it) {
            CKS(multidot(sd, P, r, f.data()));                                    // f = P^T r
            for (int k = 0; k < sd && !done; ++k) {
                // c = M[k:, k:]^-1 f[k:] (lower triangular)
                for (int i = k; i < sd; ++i) {
                    double acc = f[i];
                    for (int j = k; j < i; ++j) acc -= M(i, j) * cc[j - k];
                    cc[i - k] = acc / M(i, i);
                }
                CK(cudaMemcpyAsync(c->idr_c, cc.data(), sizeof(double) * (sd - k), cudaMemcpyHostToDevice, s));
                CK(launch_lincomb(N, sd - k, col(G, k), N, c->idr_c, 1.0, r, v, -1.0, s));   // v = r - G c
                CKS(precondition(c, prec, v, tmp, s));                                     // tmp = P^-1 v
                // U_k = U[:, k:] c + om P^-1 v, in place (each entry of U_k read before written)
                CK(launch_lincomb(N, sd - k, col(U, k), N, c->idr_c, om, tmp, col(U, k), 1.0, s));
                CKS(apply_stokes(c, col(U, k), col(G, k), s));                                // G_k = K U_k
                ++its;
                for (int i = 0; i < k; ++i) {
                    double pg = 0.0;
                    CKS(dot(c, N, col(P, i), col(G, k), s, &pg));
                    const double alpha = pg / M(i, i);
                    // G_k -= alpha G_i and U_k -= alpha U_i in one pass
                    CK(launch_axpy2(N, -alpha, col(G, i), col(G, k), -alpha, col(U, i), col(U, k), nullptr, nullptr,
                                    s));
                }
                CKS(multidot(sd - k, col(P, k), col(G, k), dots.data()));              // M[k:, k] = P^T G_k
                for (int i = k; i < sd; ++i) M(i, k) = dots[i - k];
                if (!std::isfinite(M(k, k)) || M(k, k) == 0.0) { st = STOKES_BREAKDOWN; done = true; break; }
                const double beta = f[k] / M(k, k);
                // r -= beta G_k, x += beta U_k and |r|^2 in one pass
                CK(launch_axpy2(N, -beta, col(G, k), r, beta, col(U, k), x, c->partials, c->dots, s));
                CKS(fetch(c, 1, s, &rr));
                rnorm = std::sqrt(rr);
                if (!std::isfinite(rnorm)) { st = STOKES_BREAKDOWN; done = true; break; }
                if (rnorm <= tol) { st = STOKES_OK; done = true; break; }
                if (its >= max_it) { done = true; break; }
                for (int i = k + 1; i < sd; ++i) f[i] -= beta * M(i, k);
            }
            if (done || its >= max_it) break;
            // dimension-reduction step
            CKS(precondition(c, prec, r, v, s));
            CKS(apply_stokes(c, v, t, s));
            ++its;
            double t2[2] = {0.0, 0.0};
            CK(launch_dot2(N, t, t, r, c->partials, c->dots, s));   // t . t and t . r in one pass
            CKS(fetch(c, 2, s, t2));
            const double tt = t2[0], tr = t2[1];
            if (!(tt > 0.0) || !std::isfinite(tt)) { st = STOKES_BREAKDOWN; break; }
            om = tr / tt;
            const double rho = std::fabs(tr) / (std::sqrt(tt) * rnorm);
            if (rho < 0.7) om = om * 0.7 / rho;
            CK(launch_axpy2(N, -om, t, r, om, v, x, c->partials, c->dots, s));   // r -= om t, x += om v, |r|^2
            CKS(fetch(c, 1, s, &rr));
            rnorm = std::sqrt(rr);
            if (!std::isfinite(rnorm)) { st = STOKES_BREAKDOWN; break; }
            if (rnorm <= tol) { st = STOKES_OK; break; }
        }
        if (st == STOKES_BREAKDOWN) break;
      }
    }
    // pressure with zero mean, true residual
    CKS(remove_pressure_mean(c, x, s));
    CKS(apply_stokes(c, x, r, s, true));
    CK(launch_axpby(N, 1.0, b, -1.0, r, s));
    double rt = 0.0;
    CKS(dot(c, N, r, r, s, &rt));
    // the status follows the true residual (a recurrence that met the tolerance on the last
    // allowed restart is not enough); only a breakdown keeps its own status
    if (st != STOKES_BREAKDOWN && bnorm > 0.0) st = std::sqrt(rt) <= rtol * bnorm ? STOKES_OK : STOKES_NOT_CONVERGED;
    if (info) {
        info->iterations = its;
        info->rel_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
        info->rel_residual_true = bnorm > 0 ? std::sqrt(rt) / bnorm : 0.0;
        info->status = st;
    }
    if (st != STOKES_OK)
        return fail(st, st == STOKES_BREAKDOWN ? "IDR(s) breakdown" : "IDR(s): true residual above rtol (max_it or restarts used up)");
    return STOKES_OK;
}

// ---------------------------------------------------------------- MINRES
// Method (ii)(b) of Section 2.2: MINRES (Paige & Saunders, SIAM J. Numer. Anal. 12 (1975)) with
// the symmetric positive definite block-diagonal P_D = diag(A_hat, S_hat) (precond_kind 1): the
// Lanczos process of P^-1 K in the P-inner product, its tridiagonal matrix reduced by Givens
// rotations, x updated every step along three-term directions w. The 2-norm residual is carried
// by the same recurrence (K w from K z) and checked against b - K x as in IDR(s): a drifted
// residual restarts MINRES from x (at most 10 times). 11 vectors of N.
stokes_status minres_solve(stokes_ctx* c, int prec, const double* b, double* x, double rtol, int max_it,
                           stokes_solve_info* info, cudaStream_t s) {
    const size_t N = c->N;
    for (double*& q : c->mr)
        if (!q) CKS(dalloc(c, &q, N));
    double *v_old = c->mr[0], *v = c->mr[1], *z = c->mr[2], *q = c->mr[3], *w_old = c->mr[4], *w = c->mr[5],
           *Kw_old = c->mr[6], *Kw = c->mr[7], *r = c->mr[8];
    double bnorm2 = 0.0;
    CKS(dot(c, N, b, b, s, &bnorm2));
    const double bnorm = std::sqrt(bnorm2);
    stokes_status st = STOKES_NOT_CONVERGED;
    int its = 0;
    double rnorm = 0.0;
    if (bnorm == 0.0) {
        CK(cudaMemsetAsync(x, 0, N * sizeof(double), s));
        st = STOKES_OK;
    } else {
      const double tol = rtol * bnorm;
      for (int pass = 0; pass < 11; ++pass) {
        CKS(apply_stokes(c, x, r, s, true));
        CK(launch_axpby(N, 1.0, b, -1.0, r, s));                               // r = b - K x
        double rr = 0.0;
        CKS(dot(c, N, r, r, s, &rr));
        rnorm = std::sqrt(rr);
        if (!std::isfinite(rnorm)) { st = STOKES_BREAKDOWN; break; }
        if (rnorm <= tol) { st = STOKES_OK; break; }
        if (its >= max_it) { st = STOKES_NOT_CONVERGED; break; }
        st = STOKES_NOT_CONVERGED;
        for (double* t : {v_old, w_old, w, Kw_old, Kw}) CK(cudaMemsetAsync(t, 0, N * sizeof(double), s));
        CK(cudaMemcpyAsync(v, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CKS(precondition(c, prec, v, z, s));
        double g2 = 0.0;
        CKS(dot(c, N, v, z, s, &g2));
        if (!(g2 > 0.0) || !std::isfinite(g2)) { st = STOKES_BREAKDOWN; break; }
        double gamma_old = 1.0, gamma = std::sqrt(g2), eta = gamma;
        double c_old = 1.0, cs = 1.0, s_old = 0.0, sn = 0.0;
        bool done = false;
        while (its < max_it) {
            CK(launch_axpby(N, 0.0, z, 1.0 / gamma, z, s));                    // z /= gamma
            CKS(apply_stokes(c, z, q, s));                                        // q = K z
            double delta = 0.0;
            CKS(dot(c, N, q, z, s, &delta));
            // rotations of the previous two steps applied to the new column (delta, gamma)
            const double a0 = cs * delta - c_old * sn * gamma;
            const double a2 = sn * delta + c_old * cs * gamma;
            const double a3 = s_old * gamma;
            // next Lanczos vector (scaled by gamma_new) into v_old; unnormalised w and K w
            // the three recurrences in one pass (each the two axpby steps of the unfused form)
            CK(launch_minres_dirs(N, q, z, v_old, v, -gamma / gamma_old, -delta / gamma, Kw_old, Kw, -a3, -a2, w_old,
                                  w, -a3, -a2, s));
            CKS(precondition(c, prec, v_old, q, s));                             // z_new into q
            CKS(dot(c, N, v_old, q, s, &g2));
            if (!(g2 >= 0.0) || !std::isfinite(g2)) { st = STOKES_BREAKDOWN; done = true; break; }
            const double gamma_new = std::sqrt(g2);
            const double a1 = std::hypot(a0, gamma_new);
            c_old = cs;
            s_old = sn;
            cs = a0 / a1;
            sn = gamma_new / a1;
            // w_new = w_old / a1, K w_new likewise, x += cs eta w_new, r -= cs eta K w_new, |r|^2
            CK(launch_minres_update(N, 1.0 / a1, w_old, Kw_old, cs * eta, x, r, c->partials, c->dots, s));
            eta = -sn * eta;
            ++its;
            std::swap(v_old, v);      // v <- v_new, v_old <- v
            std::swap(z, q);          // z <- z_new
            std::swap(w_old, w);      // w <- w_new, w_old <- w
            std::swap(Kw_old, Kw);
            gamma_old = gamma;
            gamma = gamma_new;
            CKS(fetch(c, 1, s, &rr));
            rnorm = std::sqrt(rr);
            if (!std::isfinite(rnorm)) { st = STOKES_BREAKDOWN; done = true; break; }
            if (rnorm <= tol || gamma == 0.0) break;
        }
        if (done) break;
      }
    }
    CKS(remove_pressure_mean(c, x, s));
    CKS(apply_stokes(c, x, r, s, true));
    CK(launch_axpby(N, 1.0, b, -1.0, r, s));
    double rt = 0.0;
    CKS(dot(c, N, r, r, s, &rt));
    // the status follows the true residual; only a breakdown keeps its own status
    if (st != STOKES_BREAKDOWN && bnorm > 0.0) st = std::sqrt(rt) <= rtol * bnorm ? STOKES_OK : STOKES_NOT_CONVERGED;
    if (info) {
        info->iterations = its;
        info->rel_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
        info->rel_residual_true = bnorm > 0 ? std::sqrt(rt) / bnorm : 0.0;
        info->status = st;
    }
    if (st != STOKES_OK) return fail(st, st == STOKES_BREAKDOWN ? "MINRES breakdown" : "MINRES: true residual above rtol (max_it or restarts used up)");
    return STOKES_OK;
}

// Viscosity description (Sections 2.3, 3.2), checked on the host before any device work: kind 0
// (sinker formula) needs finite sinker centres, 0 < mu_min, mu_max < inf and finite delta, omega,
// beta; kind 1 needs cells x 27 finite, positive quadrature-point values (the harmonic average
// and the 1/mu pressure mass need mu > 0).
stokes_status validate_mu(const stokes_mu* mu, size_t cells) {
    if (mu->kind == 0) {
        if (mu->n_sinkers < 0 || (mu->n_sinkers > 0 && !mu->centres)) return fail(STOKES_EINVAL, "bad sinker list");
        for (int i = 0; i < 3 * mu->n_sinkers; ++i)
            if (!std::isfinite(mu->centres[i])) return fail(STOKES_EINVAL, "non-finite sinker centre");
        if (!(mu->mu_min > 0.0) || !(mu->mu_max > 0.0) || !std::isfinite(mu->mu_min) || !std::isfinite(mu->mu_max))
            return fail(STOKES_EINVAL, "mu_min and mu_max must be finite and positive");
        if (!std::isfinite(mu->delta) || !std::isfinite(mu->omega) || !std::isfinite(mu->beta) || mu->delta < 0.0 ||
            mu->omega < 0.0)
            return fail(STOKES_EINVAL, "delta, omega must be finite and >= 0, beta finite");
        return STOKES_OK;
    }
    if (mu->kind == 1) {
        if (!mu->mu_q) return fail(STOKES_EINVAL, "mu_q is null");
        for (size_t i = 0; i < 27 * cells; ++i)
            if (!(mu->mu_q[i] > 0.0) || !std::isfinite(mu->mu_q[i]))
                return fail(STOKES_EINVAL, "quadrature-point viscosity must be finite and positive");
        return STOKES_OK;
    }
    return fail(STOKES_EINVAL, "unknown viscosity kind");
}

// The context's device status word, for outer_arith 2 the outer operator's f16 integer element
// table, and for vmult_kernel 2 the tensor-core level operator's f16 table (5400 A_hat from the
// library's own sum-factorised cell operator); both checked to be exact in f16.
stokes_status setup_device_status(stokes_ctx* c, cudaStream_t s) {
    CKS(dalloc(c, &c->dev_status, kStatusWords));
    CK(cudaMemsetAsync(c->dev_status, 0, kStatusWords * sizeof(unsigned), s));
    c->tc.status = c->dev_status;
    c->tc.wait_ns = (unsigned long long)(c->opt.wait_limit_s * 1e9);
    if (c->opt.outer_arith == 2) {
        unsigned char* table = nullptr;
        int* flag = nullptr;
        CKS(dalloc(c, &table, outer_tc_table_bytes()));
        CKS(dalloc(c, &flag, 1));
        CK(outer_tc_setup(table, flag, s));
        int hflag = 0;
        CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hflag != 0) return fail(STOKES_ECUDA, "the integer element table is not exact in f16 (outer_arith 2)");
        c->outer_tc_table = table;
    }
    if (c->opt.vmult_kernel != 2) return STOKES_OK;
    CK(tc_configure());
    unsigned char* table = nullptr;
    int* flag = nullptr;
    CKS(dalloc(c, &table, tc_table_bytes()));
    CKS(dalloc(c, &flag, 1));
    CK(tc_build_table(table, flag, s));
    int hflag = 0;
    CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hflag != 0) return fail(STOKES_ECUDA, "5400 A_hat is not exact in f16 (tensor-core operator)");
    c->tc_table = table;
    c->tc.table = table;
    return STOKES_OK;
}

// Read and clear the device status words (synchronises s): EMESH if a STOKES_DEBUG index check
// met a bad table entry, TIMEOUT if a bounded device wait gave up.
stokes_status take_device_status(stokes_ctx* c, cudaStream_t s) {
    if (!c->dev_status) return STOKES_OK;
    unsigned w[kStatusWords] = {};
    CK(cudaMemcpyAsync(w, c->dev_status, sizeof(w), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(c->dev_status, 0, sizeof(w), s));
    CK(cudaStreamSynchronize(s));
    if (w[0] & kStatusBadIndex) {
        const unsigned long long at = (static_cast<unsigned long long>(w[3]) << 32) | w[2];
        return fail(STOKES_EMESH, std::string("index map ") + oct_table_name(int(w[1]) - 1) + ": entry " +
                                      std::to_string(at) + " out of range");
    }
    if (w[0] != 0) return fail(STOKES_TIMEOUT, "a bounded wait inside a kernel gave up (wait_limit_s)");
    return STOKES_OK;
}

#ifdef STOKES_DEBUG
constexpr bool kDebugBuild = true;
#else
constexpr bool kDebugBuild = false;
#endif

// STOKES_DEBUG builds read the status words at the end of every call that ran index-map kernels
// (synchronising its stream), so the call that met a bad entry returns EMESH; release builds pass
// st through.
stokes_status debug_status(stokes_ctx* c, cudaStream_t s, stokes_status st) {
    if (!kDebugBuild || st != STOKES_OK || !c) return st;
    return take_device_status(c, s);
}

stokes_status validate_options(const stokes_options& o) {
    if (o.cheb_degree < 1 || o.smoothing_range <= 1.0 || o.eig_safety <= 0.0 || o.lanczos_steps < 1 ||
        o.schur_degree < 0 || o.restart < 1 || o.restart > 500 || (o.outer_arith < 0 || o.outer_arith > 2) ||
        o.vmult_kernel < 0 || o.vmult_kernel > 3 || (o.graphs != 0 && o.graphs != 1) || !(o.wait_limit_s >= 0.0) ||
        (o.batch_vcycle != 0 && o.batch_vcycle != 1) || (o.fused_smoother != 0 && o.fused_smoother != 1) ||
        o.wait_limit_s > 1e6 ||
        (o.precond_kind != 0 && o.precond_kind != 1) || o.outer_solver < 0 || o.outer_solver > 3 || (o.gram_schmidt != 0 && o.gram_schmidt != 1) ||
        (o.outer_solver == 3 && o.precond_kind != 1) ||
        o.idr_s < 1 || o.idr_s > 8)
        return fail(STOKES_EINVAL, "bad options");
    return STOKES_OK;
}

// Runs f(i) for i < n on the host threads, i interleaved over the threads (balances the
// triangular loops below).
template <typename F>
void host_parallel_rows(int n, F f) {
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt < 1 ? 1 : (nt > 32 ? 32 : nt);
    if (n < 64 || nt == 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            for (int i = int(t); i < n; i += int(nt)) f(i);
        });
    for (auto& x : th) x.join();
}

// Inverse of a dense symmetric positive definite matrix (row-major nf x nf): blocked Cholesky
// A = L L^T (row panels of kBlk columns; every inner loop a contiguous dot product), then
// W = L^-1 column by column (stored transposed, W[j][i] = (L^-1)_ij), then A^-1 = L^-T L^-1,
// entry (a, b) = sum_{i >= max(a, b)} W[a][i] W[b][i]. Rows and columns are spread over the
// host threads; the result does not depend on their number.
stokes_status spd_inverse(const std::vector<double>& A, int nf, std::vector<double>& Ainv) {
    constexpr int kBlk = 64;
    std::vector<double> L = A;   // lower triangle overwritten by the factor
    auto Lr = [&](int i) { return L.data() + size_t(i) * nf; };
    auto dotn = [](const double* x, const double* y, int n) {
        double t = 0.0;
        for (int k = 0; k < n; ++k) t += x[k] * y[k];
        return t;
    };
    for (int kb = 0; kb < nf; kb += kBlk) {
        const int ke = std::min(kb + kBlk, nf);
        // diagonal block (earlier panels already subtracted by the trailing updates)
        for (int j = kb; j < ke; ++j) {
            const double d = Lr(j)[j] - dotn(Lr(j) + kb, Lr(j) + kb, j - kb);
            if (!(d > 0.0)) return fail(STOKES_EINVAL, "coarse matrix is not positive definite");
            Lr(j)[j] = std::sqrt(d);
            for (int i = j + 1; i < ke; ++i) Lr(i)[j] = (Lr(i)[j] - dotn(Lr(i) + kb, Lr(j) + kb, j - kb)) / Lr(j)[j];
        }
        // panel below the block, then the trailing lower triangle
        host_parallel_rows(nf - ke, [&](int t) {
            double* ri = Lr(ke + t);
            for (int j = kb; j < ke; ++j) ri[j] = (ri[j] - dotn(ri + kb, Lr(j) + kb, j - kb)) / Lr(j)[j];
        });
        host_parallel_rows(nf - ke, [&](int t) {
            const int i = ke + t;
            double* ri = Lr(i);
            for (int j = ke; j <= i; ++j) ri[j] -= dotn(ri + kb, Lr(j) + kb, ke - kb);
        });
    }
    std::vector<double> W(size_t(nf) * nf, 0.0);
    host_parallel_rows(nf, [&](int j) {
        double* x = W.data() + size_t(j) * nf;   // x[i] = (L^-1)_ij, i >= j
        x[j] = 1.0 / Lr(j)[j];
        for (int i = j + 1; i < nf; ++i) x[i] = -dotn(Lr(i) + j, x + j, i - j) / Lr(i)[i];
    });
    Ainv.assign(size_t(nf) * nf, 0.0);
    host_parallel_rows(nf, [&](int a) {
        const double* wa = W.data() + size_t(a) * nf;
        for (int b = 0; b <= a; ++b) {
            const double* wb = W.data() + size_t(b) * nf;
            Ainv[size_t(a) * nf + b] = dotn(wa + a, wb + a, nf - a);
        }
    });
    for (int a = 0; a < nf; ++a)
        for (int b = a + 1; b < nf; ++b) Ainv[size_t(a) * nf + b] = Ainv[size_t(b) * nf + a];
    return STOKES_OK;
}

stokes_status check_level(const stokes_ctx* c, int& level) {
    if (!c) return fail(STOKES_EINVAL, "null context");
    if (level == -1) level = c->L - 1;
    if (level < 0 || level >= c->L) return fail(STOKES_EINVAL, "level out of range");
    return STOKES_OK;
}

stokes_status setup_impl(const stokes_mesh* mesh, const stokes_mu* mu, const stokes_bc* bc,
                         const stokes_options* opt, cudaStream_t s, stokes_ctx* c) {
    if (opt) c->opt = *opt; else stokes_default_options(&c->opt);
    const stokes_options& o = c->opt;
    CKS(validate_options(o));
    CK(brick_configure());
    CK(gs_configure());
    c->n = mesh->n;
    c->L = mesh->n_levels;
    const int L = c->L;
    c->lev.resize(L);
    for (int l = 0; l < L; ++l) c->lev[l].g = make_geom(mesh->n >> (L - 1 - l));
    const LevelGeom& gf = c->lev[L - 1].g;
    CKS(setup_device_status(c, s));
    // ---- per-level storage
    for (int l = 0; l < L; ++l) {
        Level& Lv = c->lev[l];
        const size_t nu = Lv.g.n_u, nc = Lv.g.cells;
        for (auto* p : {&Lv.v64.b, &Lv.v64.x, &Lv.v64.r, &Lv.v64.d, &Lv.v64.t, &Lv.v64.dinv, &Lv.v64.acc})
            CKS(dalloc(c, p, nu));
        for (auto* p : {&Lv.v32.b, &Lv.v32.x, &Lv.v32.r, &Lv.v32.d, &Lv.v32.t, &Lv.v32.dinv, &Lv.v32.acc})
            CKS(dalloc(c, p, nu));
        CK(cudaMemsetAsync(Lv.v64.acc, 0, nu * sizeof(double), s));
        CK(cudaMemsetAsync(Lv.v32.acc, 0, nu * sizeof(float), s));
        if (o.fused_smoother == 1 && l > 0) {
            for (auto* p : {&Lv.v64.x2, &Lv.v64.d2, &Lv.v64.acc2, &Lv.v64.acc3}) {
                CKS(dalloc(c, p, nu));
                CK(cudaMemsetAsync(*p, 0, nu * sizeof(double), s));
            }
            for (auto* p : {&Lv.v32.x2, &Lv.v32.d2, &Lv.v32.acc2, &Lv.v32.acc3}) {
                CKS(dalloc(c, p, nu));
                CK(cudaMemsetAsync(*p, 0, nu * sizeof(float), s));
            }
        }
        CK(cudaMemsetAsync(Lv.v64.d, 0, nu * sizeof(double), s));
        CK(cudaMemsetAsync(Lv.v32.d, 0, nu * sizeof(float), s));
        CKS(dalloc(c, &Lv.v64.mu, nc));
        CKS(dalloc(c, &Lv.v32.mu, nc));
        Lv.planes = brick_layout(Lv.g.n);
        CKS(dalloc(c, &Lv.slots64, Lv.planes.total));
        CKS(dalloc(c, &Lv.slots32, Lv.planes.total));
    }
    CKS(dalloc(c, &c->ref_diag, 81));
    CKS(dalloc(c, &c->F, gf.n_u));
    CKS(dalloc(c, &c->mp_dinv, gf.n_p));
    CKS(dalloc(c, &c->p_weights, gf.n_p));
    CKS(dalloc(c, &c->sp_d, gf.n_p));
    CKS(dalloc(c, &c->sp_t, gf.n_p));
    CKS(dalloc(c, &c->sp_z2, gf.n_p));
    CKS(dalloc(c, &c->sp_d2, gf.n_p));
    CKS(dalloc(c, &c->mp_scale, gf.cells));
    CKS(dalloc(c, &c->tu, gf.n_u));
    CKS(dalloc(c, &c->stage_in, gf.n_u));
    CKS(dalloc(c, &c->stage_out, gf.n_u));
    CKS(dalloc(c, &c->partials, size_t(std::max(multidot_blocks(), gs_partials_blocks())) * (o.restart + 8)));
    CKS(dalloc(c, &c->dots, size_t(o.restart + 8)));
    CK(cudaMallocHost(&c->dots_host, size_t(3 * (o.restart + 8)) * sizeof(double)));
    // ---- viscosity (Section 2.3) and right-hand side (Section 3.2)
    double* centres = nullptr;
    if (mu->kind == 0) {
        const int ns = mu->n_sinkers;
        if (ns < 0 || (ns > 0 && !mu->centres)) return fail(STOKES_EINVAL, "bad sinker list");
        CKS(dalloc(c, &centres, size_t(3) * (ns > 0 ? ns : 1)));
        if (ns > 0) CK(cudaMemcpyAsync(centres, mu->centres, sizeof(double) * 3 * ns, cudaMemcpyHostToDevice, s));
        CK(launch_mu_sinker(gf, centres, ns, mu->mu_min, mu->mu_max, mu->delta, mu->omega, c->lev[L - 1].v64.mu, s));
        CK(launch_rhs_sinker(gf, centres, ns, mu->delta, mu->omega, mu->beta, c->F, s));
    } else if (mu->kind == 1) {
        if (!mu->mu_q) return fail(STOKES_EINVAL, "mu_q is null");
        double* q = nullptr;
        CKS(dalloc(c, &q, gf.cells * 27));
        CK(cudaMemcpyAsync(q, mu->mu_q, sizeof(double) * 27 * gf.cells, cudaMemcpyHostToDevice, s));
        CK(launch_mu_from_q(gf, q, c->lev[L - 1].v64.mu, s));
        CK(cudaMemsetAsync(c->F, 0, gf.n_u * sizeof(double), s));
    } else {
        return fail(STOKES_EINVAL, "unknown viscosity kind");
    }
    for (int l = L - 2; l >= 0; --l)
        CK(launch_mu_restrict(c->lev[l].g, c->lev[l + 1].v64.mu, c->lev[l].v64.mu, s));
    CK(launch_ref_diag(c->ref_diag, s));
    for (int l = 0; l < L; ++l) {
        Level& Lv = c->lev[l];
        CK(launch_cast_d2f(Lv.g.cells, Lv.v64.mu, Lv.v32.mu, s));
        CK(launch_inv_diag(Lv.g, Lv.v64.mu, c->ref_diag, Lv.v64.dinv, s));
        CK(launch_cast_d2f(Lv.g.n_u, Lv.v64.dinv, Lv.v32.dinv, s));
    }
    // ---- pressure mass diagonal and weights (Section 2.2.2)
    CK(launch_mass_p_diag(gf, c->lev[L - 1].v64.mu, c->sp_t, c->p_weights, s));
    CK(launch_mass_scale(gf, c->lev[L - 1].v64.mu, c->mp_scale, s));
    CK(launch_recip(gf.n_p, c->sp_t, c->mp_dinv, s));
    {
        double* ones = c->sp_d;
        CK(launch_fill(gf.n_p, 1.0, ones, s));
        CKS(dot(c, gf.n_p, c->p_weights, ones, s, &c->p_wsum));
    }
    // ---- Lanczos estimates of lambda_max(D^-1 A) per level >= 1
    for (int l = 1; l < L; ++l) {
        Level& Lv = c->lev[l];
        const size_t n = Lv.g.n_u;
        double *sq = Lv.v64.r, *v = Lv.v64.x, *vp = Lv.v64.d, *w = Lv.v64.t, *tmp = Lv.v64.b;
        CK(launch_sqrt_vec(n, Lv.v64.dinv, sq, s));
        CK(launch_splitmix_vector(n, uint64_t(1907000 + l), nullptr, v, s));
        CK(launch_zero_boundary<double>(Lv.g, v, s));
        double vv = 0.0;
        CKS(dot(c, n, v, v, s, &vv));
        CK(launch_axpby(n, 1.0 / std::sqrt(vv), v, 0.0, v, s));
        CK(cudaMemsetAsync(vp, 0, n * sizeof(double), s));
        double beta_prev = 0.0;
        std::vector<double> al, be;
        for (int it = 0; it < o.lanczos_steps; ++it) {
            CK(launch_mul(n, sq, v, tmp, s));
            CKS(vmult_level<double>(c, l, tmp, w, s));
            CK(launch_mul(n, sq, w, w, s));
            double alpha = 0.0;
            CKS(dot(c, n, w, v, s, &alpha));
            CK(launch_axpby(n, -alpha, v, 1.0, w, s));
            CK(launch_axpby(n, -beta_prev, vp, 1.0, w, s));
            double b2 = 0.0;
            CKS(dot(c, n, w, w, s, &b2));
            const double beta = std::sqrt(b2);
            al.push_back(alpha);
            if (beta <= 1e-12 * std::fabs(alpha)) break;
            be.push_back(beta);
            std::swap(vp, v);                                   // v_prev <- v
            CK(launch_axpby(n, 1.0 / beta, w, 0.0, v, s));      // v <- w / beta
            beta_prev = beta;
        }
        Lv.lam_max = tridiag_max_eig(al, be);
        Lv.hi = o.eig_safety * Lv.lam_max;
        Lv.lo = Lv.hi / o.smoothing_range;
    }
    // ---- dense inverse of the coarsest free block (FP64)
    {
        Level& L0 = c->lev[0];
        const int M = L0.g.M;
        std::vector<int> idx;
        for (int comp = 0; comp < 3; ++comp)
            for (int k = 1; k < M - 1; ++k)
                for (int j = 1; j < M - 1; ++j)
                    for (int i = 1; i < M - 1; ++i) idx.push_back(int(comp * L0.g.nodes + i + size_t(M) * (j + size_t(M) * k)));
        const int nf = int(idx.size());
        c->nf = nf;
        if (nf > 0) {
            CKS(dalloc(c, &c->free_idx, size_t(nf)));
            CK(cudaMemcpyAsync(c->free_idx, idx.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s));
            std::vector<double> A(size_t(nf) * nf), col(L0.g.n_u);
            double *e = L0.v64.b, *Ae = L0.v64.t;
            for (int j = 0; j < nf; ++j) {
                CK(cudaMemsetAsync(e, 0, L0.g.n_u * sizeof(double), s));
                const double one = 1.0;
                CK(cudaMemcpyAsync(e + idx[j], &one, sizeof(double), cudaMemcpyHostToDevice, s));
                CKS(vmult_level<double>(c, 0, e, Ae, s));
                CK(cudaMemcpyAsync(col.data(), Ae, L0.g.n_u * sizeof(double), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                for (int i = 0; i < nf; ++i) A[size_t(i) * nf + j] = col[idx[i]];
            }
            std::vector<double> Ainv;
            CKS(spd_inverse(A, nf, Ainv));
            CKS(dalloc(c, &c->Ainv, size_t(nf) * nf));
            CK(cudaMemcpyAsync(c->Ainv, Ainv.data(), sizeof(double) * nf * nf, cudaMemcpyHostToDevice, s));
        }
    }
    CK(cudaStreamSynchronize(s));
    return STOKES_OK;
}

template <typename T>
stokes_status upload(stokes_ctx* c, T** dev, const std::vector<T>& host, cudaStream_t s) {
    CKS(dalloc(c, dev, host.size()));
    if (!host.empty()) CK(cudaMemcpyAsync(*dev, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return STOKES_OK;
}

// Octree setup: host tables (octree_host.cpp), device copies, level diagonals, Lanczos
// estimates per level (start vector splitmix64(1907000 + li) on the smoothed nodes), the dense
// inverse of the coarsest (uniform) level, right-hand side and pressure mass diagonal.
stokes_status oct_setup_impl(const stokes_octree* mesh, const stokes_mu* mu, const stokes_options* opt,
                             cudaStream_t s, stokes_ctx* c) {
    if (opt) c->opt = *opt; else stokes_default_options(&c->opt);
    CKS(validate_options(c->opt));
    const stokes_options& o = c->opt;
    if (mu->kind != 0) return fail(STOKES_EINVAL, "octree meshes take the sinker viscosity (kind 0)");
    CKS(validate_mu(mu, 0));
    c->oct = new (std::nothrow) OctCtx();
    if (!c->oct) return fail(STOKES_ENOMEM, "host allocation failed");
    OctCtx& oc = *c->oct;
    std::vector<uint64_t> leaves(mesh->leaf_keys, mesh->leaf_keys + mesh->n_leaves);
    OctSinkers sk;
    sk.n = mu->n_sinkers;
    sk.centres = mu->centres;
    sk.mu_min = mu->mu_min;
    sk.mu_max = mu->mu_max;
    sk.delta = mu->delta;
    sk.omega = mu->omega;
    sk.beta = mu->beta;
    // host tables first: a malformed or unbalanced leaf set is refused before any device work
    const std::string err = oct_build(leaves, mesh->coarsest_level, sk, oc.host);
    if (!err.empty()) return fail(STOKES_EMESH, "octree: " + err);
    CK(brick_configure());
    CK(gs_configure());
    CKS(setup_device_status(c, s));
    const OctHost& H = oc.host;
    // ---- active space
    OctActiveDev& a = oc.act;
    a.n_leaves = int(H.leaves.size());
    a.nu_nodes = H.unodes.size();
    a.np = H.pverts.size();
    a.n_ucon = H.ucon_node.size() / kOctUCon;
    a.n_pcon = H.pcon_node.size() / kOctPCon;
    a.dbg.status = c->dev_status;
    // The active-space kernels visit leaves in Morton (z-curve) order of their lower corner on the
    // finest lattice, so that neighbouring threads share nodes in cache (the key order keeps the
    // leaves of different levels apart); numbering (key order) and results are unchanged up to the
    // order of the atomic additions.
    auto morton = [&](uint64_t cell) {
        const int sh = H.lmax - oct_l(cell);
        const uint64_t x = uint64_t(oct_i(cell)) << sh, y = uint64_t(oct_j(cell)) << sh, z = uint64_t(oct_k(cell)) << sh;
        uint64_t m = 0;
        for (int b = 0; b < 16; ++b)
            m |= (((x >> b) & 1) << (3 * b)) | (((y >> b) & 1) << (3 * b + 1)) | (((z >> b) & 1) << (3 * b + 2));
        return (m << 4) | uint64_t(oct_l(cell));
    };
    auto z_order = [&](const std::vector<uint64_t>& cells) {
        std::vector<uint64_t> key(cells.size());
        for (size_t n = 0; n < cells.size(); ++n) key[n] = morton(cells[n]);
        std::vector<uint32_t> perm(cells.size());
        for (size_t n = 0; n < perm.size(); ++n) perm[n] = uint32_t(n);
        std::sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return key[a] < key[b]; });
        return perm;   // perm[new position] = index in key order
    };
    {
        int32_t *lu, *lp, *un, *pn;
        double *uw, *pw, *lm;
        uint8_t *ub, *lv;
        const size_t nl = H.leaves.size();
        const std::vector<uint32_t> perm = z_order(H.leaves);
        std::vector<uint8_t> lev8(nl);
        std::vector<int32_t> zu(nl * 27), zp(nl * 8);
        std::vector<double> zmu(nl);
        for (size_t n = 0; n < nl; ++n) {
            const size_t o = perm[n];
            lev8[n] = uint8_t(oct_l(H.leaves[o]));
            zmu[n] = H.leaf_mu[o];
            std::copy(H.leaf_u.begin() + o * 27, H.leaf_u.begin() + o * 27 + 27, zu.begin() + n * 27);
            std::copy(H.leaf_p.begin() + o * 8, H.leaf_p.begin() + o * 8 + 8, zp.begin() + n * 8);
        }
        CKS(upload(c, &lu, zu, s));
        CKS(upload(c, &lp, zp, s));
        CKS(upload(c, &un, H.ucon_node, s));
        CKS(upload(c, &uw, H.ucon_w, s));
        CKS(upload(c, &pn, H.pcon_node, s));
        CKS(upload(c, &pw, H.pcon_w, s));
        CKS(upload(c, &ub, H.ubnd, s));
        CKS(upload(c, &lm, zmu, s));
        CKS(upload(c, &lv, lev8, s));
        CK(cudaStreamSynchronize(s));   // lev8 (pageable, local) consumed
        a.leaf_u = lu; a.leaf_p = lp; a.ucon_node = un; a.ucon_w = uw; a.pcon_node = pn; a.pcon_w = pw;
        a.ubnd = ub; a.mu = lm; a.level = lv;
        oc.leaf_mu = lm;
    }
    const size_t nu = 3 * a.nu_nodes, np = a.np;
    CKS(upload(c, &c->F, H.F, s));
    {
        std::vector<double> dinv(np);
        double wsum = 0.0;
        for (size_t n = 0; n < np; ++n) {
            dinv[n] = 1.0 / H.mp_diag[n];
            wsum += H.p_weights[n];
        }
        CKS(upload(c, &c->mp_dinv, dinv, s));
        CK(cudaStreamSynchronize(s));
        CKS(upload(c, &c->p_weights, H.p_weights, s));
        c->p_wsum = wsum;
    }
    CKS(dalloc(c, &c->sp_d, np));
    CKS(dalloc(c, &c->sp_t, np));
    CKS(dalloc(c, &c->tu, nu));
    CKS(dalloc(c, &c->partials, size_t(std::max(multidot_blocks(), gs_partials_blocks())) * (o.restart + 8)));
    CKS(dalloc(c, &c->dots, size_t(o.restart + 8)));
    CK(cudaMallocHost(&c->dots_host, size_t(3 * (o.restart + 8)) * sizeof(double)));
    CKS(dalloc(c, &c->ref_diag, 81));
    CK(launch_ref_diag(c->ref_diag, s));
    // ---- levels
    const int NL = int(H.levels.size());
    oc.lev.resize(NL);
    std::vector<std::vector<int32_t>> ca(NL), cl(NL);
    for (size_t n = 0; n < H.unodes.size(); ++n) {
        if (H.ubnd[n]) continue;
        const int li = H.copy_level[n] - H.coarsest;
        ca[li].push_back(int32_t(n));
        cl[li].push_back(H.copy_index[n]);
    }
    std::vector<std::vector<uint32_t>> inv_perm(NL);   // key-order index -> position visited
    for (int li = 0; li < NL; ++li) {
        const OctLevelHost& LH = H.levels[li];
        OctLevel& L = oc.lev[li];
        int32_t* cn;
        uint8_t* fl;
        const size_t ncl = LH.cells.size();
        // level cells keep key (row) order: it matches the row-major node numbering of the level, so
        // neighbouring threads read neighbouring nodes (Morton order measured slower here)
        std::vector<uint32_t> perm(ncl);
        for (size_t n = 0; n < ncl; ++n) perm[n] = uint32_t(n);
        inv_perm[li].resize(ncl);
        std::vector<int32_t> zcn(ncl * 27);
        std::vector<double> zmu(ncl);
        for (size_t n = 0; n < ncl; ++n) {
            inv_perm[li][perm[n]] = uint32_t(n);
            zmu[n] = LH.mu[perm[n]];
            std::copy(LH.cell_nodes.begin() + size_t(perm[n]) * 27, LH.cell_nodes.begin() + size_t(perm[n]) * 27 + 27,
                      zcn.begin() + n * 27);
        }
        CKS(upload(c, &cn, zcn, s));
        CKS(upload(c, &fl, LH.flags, s));
        L.g.n_cells = int(LH.cells.size());
        L.g.nn = LH.nodes.size();
        L.g.h = std::ldexp(1.0, -LH.l);
        L.g.cell_nodes = cn;
        L.g.flags = fl;
        L.g.dbg.status = c->dev_status;
        if (li > 0) {
            uint32_t* pa;
            uint16_t* po;
            std::vector<uint32_t> par(LH.parent.size());
            for (size_t t = 0; t < par.size(); ++t) par[t] = inv_perm[li - 1][LH.parent[t]];
            CKS(upload(c, &pa, par, s));
            CKS(upload(c, &po, LH.pos, s));
            L.g.parent = pa;
            L.g.pos = po;
        }
        const size_t n3 = 3 * L.g.nn;
        for (auto* q : {&L.v64.b, &L.v64.x, &L.v64.r, &L.v64.d, &L.v64.t, &L.v64.dinv, &L.v64.acc}) CKS(dalloc(c, q, n3));
        for (auto* q : {&L.v32.b, &L.v32.x, &L.v32.r, &L.v32.d, &L.v32.t, &L.v32.dinv, &L.v32.acc}) CKS(dalloc(c, q, n3));
        CK(cudaMemsetAsync(L.v64.acc, 0, n3 * sizeof(double), s));
        CK(cudaMemsetAsync(L.v32.acc, 0, n3 * sizeof(float), s));
        CK(cudaMemsetAsync(L.v64.d, 0, n3 * sizeof(double), s));
        CK(cudaMemsetAsync(L.v32.d, 0, n3 * sizeof(float), s));
        CKS(upload(c, &L.v64.mu, zmu, s));
        CKS(dalloc(c, &L.v32.mu, LH.mu.size()));
        CK(launch_cast_d2f(LH.mu.size(), L.v64.mu, L.v32.mu, s));
        CK(launch_oct_inv_diag(L.g, L.v64.mu, c->ref_diag, L.v64.t, L.v64.dinv, s));
        CK(launch_cast_d2f(n3, L.v64.dinv, L.v32.dinv, s));
        L.n_copy = ca[li].size();
        CKS(upload(c, &L.copy_a, ca[li], s));
        CKS(upload(c, &L.copy_l, cl[li], s));
    }
    CK(cudaStreamSynchronize(s));   // the local copy lists are consumed
    // ---- Lanczos estimates of lambda_max(D^-1 A) on the smoothed nodes, levels li >= 1
    for (int li = 1; li < NL; ++li) {
        OctLevel& L = oc.lev[li];
        const size_t n = 3 * L.g.nn;
        std::vector<double> mask(n);
        const OctLevelHost& LH = H.levels[li];
        for (int cc = 0; cc < 3; ++cc)
            for (size_t t = 0; t < L.g.nn; ++t) mask[cc * L.g.nn + t] = LH.flags[t] == 0 ? 1.0 : 0.0;
        double *sq = L.v64.r, *v = L.v64.x, *vp = L.v64.d, *w = L.v64.t, *tmp = L.v64.b;
        CK(cudaMemcpyAsync(tmp, mask.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(launch_splitmix_vector(n, uint64_t(1907000 + li), tmp, v, s));
        CK(cudaStreamSynchronize(s));   // mask (pageable) consumed
        CK(launch_sqrt_vec(n, L.v64.dinv, sq, s));
        double vv = 0.0;
        CKS(dot(c, n, v, v, s, &vv));
        CK(launch_axpby(n, 1.0 / std::sqrt(vv), v, 0.0, v, s));
        CK(cudaMemsetAsync(vp, 0, n * sizeof(double), s));
        double beta_prev = 0.0;
        std::vector<double> al, be;
        for (int it = 0; it < o.lanczos_steps; ++it) {
            CK(launch_mul(n, sq, v, tmp, s));
            CKS(oct_vmult_level<double>(c, li, tmp, w, s));
            CK(launch_mul(n, sq, w, w, s));
            double alpha = 0.0;
            CKS(dot(c, n, w, v, s, &alpha));
            CK(launch_axpby(n, -alpha, v, 1.0, w, s));
            CK(launch_axpby(n, -beta_prev, vp, 1.0, w, s));
            double b2 = 0.0;
            CKS(dot(c, n, w, w, s, &b2));
            const double beta = std::sqrt(b2);
            al.push_back(alpha);
            if (beta <= 1e-12 * std::fabs(alpha)) break;
            be.push_back(beta);
            std::swap(vp, v);
            CK(launch_axpby(n, 1.0 / beta, w, 0.0, v, s));
            beta_prev = beta;
        }
        L.lam_max = tridiag_max_eig(al, be);
        L.hi = o.eig_safety * L.lam_max;
        L.lo = L.hi / o.smoothing_range;
        CK(cudaMemsetAsync(L.v64.d, 0, n * sizeof(double), s));
    }
    // ---- dense inverse of the coarsest level on its free nodes (FP64)
    {
        OctLevel& L0 = oc.lev[0];
        const OctLevelHost& LH = H.levels[0];
        const size_t nn = L0.g.nn, n3 = 3 * nn;
        std::vector<int> idx;
        for (int cc = 0; cc < 3; ++cc)
            for (size_t t = 0; t < nn; ++t)
                if (LH.flags[t] == 0) idx.push_back(int(cc * nn + t));
        const int nf = int(idx.size());
        if (nf > 4000) return fail(STOKES_EMESH, "coarsest level too large for the dense solve");
        c->nf = nf;
        if (nf > 0) {
            CKS(dalloc(c, &c->free_idx, size_t(nf)));
            CK(cudaMemcpyAsync(c->free_idx, idx.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s));
            std::vector<double> A(size_t(nf) * nf), col(n3);
            double *e = L0.v64.b, *Ae = L0.v64.t;
            const double one = 1.0;
            for (int j = 0; j < nf; ++j) {
                CK(cudaMemsetAsync(e, 0, n3 * sizeof(double), s));
                CK(cudaMemcpyAsync(e + idx[j], &one, sizeof(double), cudaMemcpyHostToDevice, s));
                CKS(oct_vmult_level<double>(c, 0, e, Ae, s));
                CK(cudaMemcpyAsync(col.data(), Ae, n3 * sizeof(double), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                for (int i = 0; i < nf; ++i) A[size_t(i) * nf + j] = col[idx[i]];
            }
            std::vector<double> Ainv;
            CKS(spd_inverse(A, nf, Ainv));
            CKS(dalloc(c, &c->Ainv, size_t(nf) * nf));
            CK(cudaMemcpyAsync(c->Ainv, Ainv.data(), sizeof(double) * nf * nf, cudaMemcpyHostToDevice, s));
        }
    }
    CK(cudaStreamSynchronize(s));
    return debug_status(c, s, STOKES_OK);
}

}  // namespace

extern "C" {

void stokes_default_options(stokes_options* opt) {
    if (!opt) return;
    opt->cheb_degree = 4;
    opt->smoothing_range = 15.0;
    opt->eig_safety = 1.2;
    opt->lanczos_steps = 12;
    opt->schur_degree = 5;
    opt->restart = 50;
    opt->outer_arith = 1;
    opt->vmult_kernel = 0;
    opt->graphs = 1;
    opt->precond_kind = 0;
    opt->outer_solver = 0;
    opt->idr_s = 2;
    opt->gram_schmidt = 1;
    opt->wait_limit_s = 1.0;
    opt->batch_vcycle = 0;
    opt->fused_smoother = 0;
}

const char* stokes_strerror(stokes_status s) {
    switch (s) {
        case STOKES_OK: return "ok";
        case STOKES_EINVAL: return "invalid argument";
        case STOKES_ENOMEM: return "out of memory";
        case STOKES_ECUDA: return "CUDA error";
        case STOKES_NOT_CONVERGED: return "not converged";
        case STOKES_BREAKDOWN: return "breakdown";
        case STOKES_TIMEOUT: return "timeout";
        case STOKES_EMESH: return "unsupported mesh";
    }
    return "unknown status";
}

const char* stokes_last_error(void) { return g_last_error.c_str(); }

stokes_status stokes_profile(int enable) {
    if (!enable) drain();
    g_prof_on = enable != 0;
    return STOKES_OK;
}

stokes_status stokes_profile_read(int cls, double* ms, long long* launches, int reset) {
    if (cls < 0 || cls >= PROF_NCLASS) return fail(STOKES_EINVAL, "bad profile class");
    drain();
    if (ms) *ms = g_ms[cls];
    if (launches) *launches = g_cnt[cls];
    if (reset) {
        for (int i = 0; i < PROF_NCLASS; ++i) { g_ms[i] = 0.0; g_cnt[i] = 0; }
    }
    return STOKES_OK;
}

long long stokes_launch_count(void) { return g_launches; }

stokes_status stokes_setup(const stokes_mesh* mesh, const stokes_mu* mu, const stokes_bc* bc,
                           const stokes_options* opt, void* stream, stokes_ctx** out) {
    g_last_error.clear();
    if (!mesh || !mu || !bc || !out) return fail(STOKES_EINVAL, "null argument");
    *out = nullptr;
    if (mesh->kind != 0) return fail(STOKES_EMESH, "only the uniform mesh kind 0 is supported");
    if (bc->noslip_faces != 0x3Fu) return fail(STOKES_EMESH, "all six walls must be no-slip (0x3F)");
    if (mesh->n_levels < 1 || mesh->n_levels > 12 || mesh->n < 1 || mesh->n > 1024)
        return fail(STOKES_EINVAL, "n or n_levels out of range");
    const int cdiv = 1 << (mesh->n_levels - 1);
    if (mesh->n % cdiv != 0) return fail(STOKES_EMESH, "n must be c * 2^(n_levels-1)");
    const int coarse = mesh->n / cdiv;
    // the dense coarse inverse holds the 3 (2c - 1)^3 free DoFs of a c^3 coarsest mesh: at most
    // 4,000 of them (c <= 6), the same limit as on octree meshes
    if (3 * (2 * coarse - 1) * (2 * coarse - 1) * (2 * coarse - 1) > 4000)
        return fail(STOKES_EMESH, "coarsest level must have at most 6 cells per axis (dense FP64 solve)");
    CKS(validate_mu(mu, size_t(mesh->n) * mesh->n * mesh->n));
    stokes_ctx* c = new (std::nothrow) stokes_ctx();
    if (!c) return fail(STOKES_ENOMEM, "host allocation failed");
    stokes_status st = setup_impl(mesh, mu, bc, opt, static_cast<cudaStream_t>(stream), c);
    if (st != STOKES_OK) {
        const std::string msg = g_last_error;
        stokes_destroy(c);
        g_last_error = msg;
        return st;
    }
    *out = c;
    return STOKES_OK;
}

void stokes_destroy(stokes_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    for (cudaGraphExec_t& ge : c->gexec)
        if (ge) cudaGraphExecDestroy(ge);
    if (c->gev_in) cudaEventDestroy(c->gev_in);
    if (c->gev_out) cudaEventDestroy(c->gev_out);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (void* p : c->allocs) cudaFree(p);
    if (c->dots_host) cudaFreeHost(c->dots_host);
    delete c->oct;
    delete c;
}

stokes_status stokes_octree_sinker_mesh(int base_level, int n_sinkers, const double* centres, const int* max_levels,
                                        double shell_radius, double shell_half_width, uint64_t* keys, int64_t capacity,
                                        int64_t* n_leaves) {
    g_last_error.clear();
    if (!n_leaves || base_level < 0 || base_level > 15 || n_sinkers < 0 || (n_sinkers > 0 && (!centres || !max_levels)))
        return fail(STOKES_EINVAL, "bad argument");
    for (int i = 0; i < n_sinkers; ++i)
        if (max_levels[i] > 15) return fail(STOKES_EINVAL, "maximum level above 15");
    try {
        const std::vector<uint64_t> leaves =
            oct_balance(oct_refine_shells(base_level, n_sinkers, centres, max_levels, shell_radius, shell_half_width));
        *n_leaves = int64_t(leaves.size());
        if (capacity < int64_t(leaves.size())) {
            if (keys || capacity != 0) return fail(STOKES_EINVAL, "capacity below the number of leaves");
            return STOKES_OK;
        }
        if (!keys) return fail(STOKES_EINVAL, "null key buffer");
        std::copy(leaves.begin(), leaves.end(), keys);
    } catch (const std::bad_alloc&) {
        return fail(STOKES_ENOMEM, "host allocation failed");
    }
    return STOKES_OK;
}

stokes_status stokes_octree_refine_gradient(const stokes_octree* mesh, const double* u_host, double fraction,
                                            double* eta, uint64_t* keys, int64_t capacity, int64_t* n_leaves) {
    g_last_error.clear();
    if (!mesh || !u_host || !n_leaves || mesh->n_leaves < 1 || !mesh->leaf_keys || !(fraction > 0.0) ||
        fraction > 1.0)
        return fail(STOKES_EINVAL, "bad argument");
    try {
        const std::vector<uint64_t> leaves(mesh->leaf_keys, mesh->leaf_keys + mesh->n_leaves);
        OctSinkers sk;   // the tables of the active space do not depend on the viscosity
        OctHost o;
        const std::string err = oct_build(leaves, mesh->coarsest_level, sk, o, true);
        if (!err.empty()) return fail(STOKES_EMESH, err);
        for (size_t i = 0; i < 3 * o.unodes.size(); ++i)
            if (!std::isfinite(u_host[i])) return fail(STOKES_EINVAL, "non-finite velocity");
        std::vector<double> ind;
        oct_gradient_indicator(o, u_host, ind);
        if (eta) std::copy(ind.begin(), ind.end(), eta);
        const std::vector<uint64_t> out = oct_refine_by_indicator(o.leaves, ind, fraction);
        for (uint64_t c : out)
            if (oct_l(c) > 15) return fail(STOKES_EINVAL, "refinement beyond level 15");
        *n_leaves = int64_t(out.size());
        if (capacity < int64_t(out.size())) {
            if (keys || capacity != 0) return fail(STOKES_EINVAL, "capacity below the number of leaves");
            return STOKES_OK;
        }
        if (!keys) return fail(STOKES_EINVAL, "null key buffer");
        std::copy(out.begin(), out.end(), keys);
    } catch (const std::bad_alloc&) {
        return fail(STOKES_ENOMEM, "host allocation failed");
    }
    return STOKES_OK;
}

stokes_status stokes_setup_octree(const stokes_octree* mesh, const stokes_mu* mu, const stokes_bc* bc,
                                  const stokes_options* opt, void* stream, stokes_ctx** out) {
    g_last_error.clear();
    if (!mesh || !mu || !bc || !out || (mesh->n_leaves > 0 && !mesh->leaf_keys))
        return fail(STOKES_EINVAL, "null argument");
    *out = nullptr;
    if (bc->noslip_faces != 0x3Fu) return fail(STOKES_EMESH, "all six walls must be no-slip (0x3F)");
    if (mesh->n_leaves < 1) return fail(STOKES_EMESH, "no leaves");
    stokes_ctx* c = new (std::nothrow) stokes_ctx();
    if (!c) return fail(STOKES_ENOMEM, "host allocation failed");
    stokes_status st;
    try {
        st = oct_setup_impl(mesh, mu, opt, static_cast<cudaStream_t>(stream), c);
    } catch (const std::bad_alloc&) {
        st = fail(STOKES_ENOMEM, "host allocation failed");
    }
    if (st != STOKES_OK) {
        const std::string msg = g_last_error;
        stokes_destroy(c);
        g_last_error = msg;
        return st;
    }
    *out = c;
    return STOKES_OK;
}

size_t stokes_octree_table(const stokes_ctx* c, int which, int level, void* out, size_t capacity) {
    if (!c || !c->oct) return 0;
    const OctHost& H = c->oct->host;
    auto put = [&](const auto& v) -> size_t {
        using E = typename std::decay<decltype(v)>::type::value_type;
        if (out) std::memcpy(out, v.data(), std::min(capacity, v.size()) * sizeof(E));
        return v.size();
    };
    const bool lv = level >= 0 && level < int(H.levels.size());
    switch (which) {
        case 0: return put(H.leaves);
        case 1: return put(H.unodes);
        case 2: return put(H.pverts);
        case 3: return lv ? put(H.levels[level].nodes) : 0;
        case 4: return lv ? put(H.levels[level].flags) : 0;
        case 5: {
            std::vector<int32_t> li(H.copy_level.size());
            for (size_t n = 0; n < li.size(); ++n) li[n] = H.copy_level[n] - H.coarsest;
            return put(li);
        }
        case 6: return H.ucon_node.size() / kOctUCon;
        case 7: return H.pcon_node.size() / kOctPCon;
    }
    return 0;
}

size_t stokes_size(const stokes_ctx* c, int level, int what) {
    if (!c) return 0;
    if (c->oct) {
        const OctCtx& o = *c->oct;
        const int NL = int(o.lev.size());
        if (what == 4) return size_t(NL);
        if (level == -1) {
            switch (what) {
                case 0: return 3 * o.act.nu_nodes;
                case 1: return o.act.np;
                case 2: return size_t(o.act.n_leaves);
                case 3: return size_t(o.host.lmax);
            }
            return 0;
        }
        if (level < 0 || level >= NL) return 0;
        switch (what) {
            case 0: return 3 * o.lev[level].g.nn;
            case 1: return 0;
            case 2: return size_t(o.lev[level].g.n_cells);
            case 3: return size_t(o.host.levels[level].l);
        }
        return 0;
    }
    if (level == -1) level = c->L - 1;
    if (level < 0 || level >= c->L) return 0;
    const LevelGeom& g = c->lev[level].g;
    switch (what) {
        case 0: return g.n_u;
        case 1: return g.n_p;
        case 2: return g.cells;
        case 3: return size_t(g.n);
        case 4: return size_t(c->L);
    }
    return 0;
}

static stokes_status oct_vmult(stokes_ctx* c, int level, int block, int prec, const void* src, void* dst, cudaStream_t s) {
    OctCtx& o = *c->oct;
    if (level >= 0) {
        if (level >= int(o.lev.size())) return fail(STOKES_EINVAL, "level out of range");
        if (block != STOKES_BLOCK_A) return fail(STOKES_EINVAL, "multigrid levels have block A only");
        if (prec == STOKES_FP32)
            return oct_vmult_level<float>(c, level, static_cast<const float*>(src), static_cast<float*>(dst), s);
        if (prec == STOKES_FP64)
            return oct_vmult_level<double>(c, level, static_cast<const double*>(src), static_cast<double*>(dst), s);
        return fail(STOKES_EINVAL, "bad precision");
    }
    if (level != -1) return fail(STOKES_EINVAL, "level out of range");
    if (prec != STOKES_FP64) return fail(STOKES_EINVAL, "the active-space blocks are FP64 only");
    const double* sd = static_cast<const double*>(src);
    double* dd = static_cast<double*>(dst);
    switch (block) {
        case STOKES_BLOCK_A: CK(launch_oct_active(o.act, sd, nullptr, dd, nullptr, true, false, false, s)); return STOKES_OK;
        case STOKES_BLOCK_B: CK(launch_oct_active(o.act, sd, nullptr, nullptr, dd, false, false, true, s)); return STOKES_OK;
        case STOKES_BLOCK_BT: CK(launch_oct_active(o.act, nullptr, sd, dd, nullptr, false, true, false, s)); return STOKES_OK;
        case STOKES_BLOCK_MP: CK(launch_oct_mass_p(o.act, sd, dd, s)); return STOKES_OK;
        case STOKES_BLOCK_STOKES: return apply_stokes(c, sd, dd, s);
    }
    return fail(STOKES_EINVAL, "bad block");
}

stokes_status stokes_vmult(stokes_ctx* c, int level, int block, int prec, const void* src, void* dst,
                           void* stream) {
    if (c && c->oct) {
        if (!src || !dst) return fail(STOKES_EINVAL, "null vector");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        return debug_status(c, s, oct_vmult(c, level, block, prec, src, dst, s));
    }
    CKS(check_level(c, level));
    if (!src || !dst) return fail(STOKES_EINVAL, "null vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Level& Lv = c->lev[level];
    if (block == STOKES_BLOCK_A) {
        if (prec == STOKES_FP32) {
            CKS(vmult_level<float>(c, level, static_cast<const float*>(src), static_cast<float*>(dst), s));
        } else if (prec == STOKES_FP64) {
            CKS(vmult_level<double>(c, level, static_cast<const double*>(src), static_cast<double*>(dst), s));
        } else {
            return fail(STOKES_EINVAL, "bad precision");
        }
        return STOKES_OK;
    }
    if (prec != STOKES_FP64) return fail(STOKES_EINVAL, "B, B^T, M_p and Stokes blocks are FP64 only");
    if (level != c->L - 1) return fail(STOKES_EINVAL, "B, B^T, M_p and Stokes blocks are finest-level only");
    const double* sd = static_cast<const double*>(src);
    double* dd = static_cast<double*>(dst);
    switch (block) {
        case STOKES_BLOCK_B:
            CK(launch_stokes_blocks(Lv.g, Lv.v64.mu, sd, nullptr, nullptr, dd, false, false, true, c->opt.outer_arith >= 1, s));
            return STOKES_OK;
        case STOKES_BLOCK_BT:
            CK(launch_stokes_blocks(Lv.g, Lv.v64.mu, nullptr, sd, dd, nullptr, false, true, false, c->opt.outer_arith >= 1, s));
            return STOKES_OK;
        case STOKES_BLOCK_MP:
            CK(launch_mass_p(Lv.g, Lv.v64.mu, sd, dd, s));
            return STOKES_OK;
        case STOKES_BLOCK_STOKES:
            return apply_stokes(c, sd, dd, s);
    }
    return fail(STOKES_EINVAL, "bad block");
}

stokes_status gmg_vcycle(stokes_ctx* c, int prec, const void* rhs, void* x, void* stream) {
    if (!c || !rhs || !x) return fail(STOKES_EINVAL, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c->oct) {
        if (prec == STOKES_FP32)
            return debug_status(c, s, oct_vcycle<float>(c, static_cast<const double*>(rhs), static_cast<double*>(x), s));
        if (prec == STOKES_FP64)
            return debug_status(c, s, oct_vcycle<double>(c, static_cast<const double*>(rhs), static_cast<double*>(x), s));
        return fail(STOKES_EINVAL, "bad precision");
    }
    if (prec == STOKES_FP32) return vcycle<float>(c, static_cast<const float*>(rhs), static_cast<float*>(x), s);
    if (prec == STOKES_FP64) return vcycle<double>(c, static_cast<const double*>(rhs), static_cast<double*>(x), s);
    return fail(STOKES_EINVAL, "bad precision");
}

stokes_status stokes_solve(stokes_ctx* c, int vcycle_prec, const double* rhs, double* up, double rtol, int max_it,
                           stokes_solve_info* info, void* stream) {
    if (!c || !up) return fail(STOKES_EINVAL, "null argument");
    if (vcycle_prec != STOKES_FP32 && vcycle_prec != STOKES_FP64) return fail(STOKES_EINVAL, "bad precision");
    if (!(rtol > 0.0) || max_it < 1) return fail(STOKES_EINVAL, "bad rtol or max_it");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    if (c->opt.outer_solver == 1) {
        c->idr_stream = s;
        CKS(ensure_idr(c, c->opt.idr_s));
    } else if (c->opt.outer_solver == 3) {
        c->N = active_nu(c) + active_np(c);   // MINRES vectors: minres_solve
        if (!c->bvec) CKS(dalloc(c, &c->bvec, c->N));
    } else {
        CKS(ensure_krylov(c));
    }
    const size_t nu = active_nu(c), np = active_np(c);
    const double* b = rhs;
    if (!b) {
        CK(cudaMemcpyAsync(c->bvec, c->F, nu * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(c->bvec + nu, 0, np * sizeof(double), s));
        b = c->bvec;
    }
    stokes_status st = c->opt.outer_solver == 1   ? idr_solve(c, vcycle_prec, b, up, rtol, max_it, info, s)
                       : c->opt.outer_solver == 3 ? minres_solve(c, vcycle_prec, b, up, rtol, max_it, info, s)
                                                  : fgmres(c, vcycle_prec, b, up, rtol, max_it, info, s);
    const stokes_status dst = take_device_status(c, s);
    if (dst != STOKES_OK && st != STOKES_ECUDA) st = dst;
    const auto t1 = std::chrono::steady_clock::now();
    if (info) {
        info->seconds = std::chrono::duration<double>(t1 - t0).count();
        info->status = st;
    }
    return st;
}

stokes_status stokes_set_batch_vcycle(stokes_ctx* c, int mode) {
    if (!c || (mode != 0 && mode != 1)) return fail(STOKES_EINVAL, "null context or bad mode");
    c->opt.batch_vcycle = mode;
    return STOKES_OK;
}

stokes_status stokes_debug_alloc_limit(long long bytes) {
    g_alloc_left = bytes < 0 ? -1 : bytes;
    return STOKES_OK;
}

stokes_status stokes_device_status(stokes_ctx* c, void* stream) {
    if (!c) return fail(STOKES_EINVAL, "null context");
    return take_device_status(c, static_cast<cudaStream_t>(stream));
}

// Drop the captured V-cycle graphs (after a change of the smoother); they are recaptured on next use.
static stokes_status drop_graphs(stokes_ctx* c) {
    CK(cudaDeviceSynchronize());
    for (cudaGraphExec_t& ge : c->gexec)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
    return STOKES_OK;
}

int stokes_debug_build(void) { return kDebugBuild ? 1 : 0; }

stokes_status stokes_debug_index_cut(stokes_ctx* c, int table, long long cut) {
    if (!kDebugBuild) return fail(STOKES_EINVAL, "index-map checks exist in STOKES_DEBUG builds only");
    if (!c || !c->oct) return fail(STOKES_EINVAL, "an octree context is required");
    if (table < 0 || table >= OCT_NTABLES || cut < 0) return fail(STOKES_EINVAL, "bad table or cut");
    CKS(drop_graphs(c));   // captured launches hold the old bounds
    c->oct->act.dbg.cut[table] = cut;
    for (OctLevel& L : c->oct->lev) L.g.dbg.cut[table] = cut;
    return STOKES_OK;
}

stokes_status stokes_autotune(stokes_ctx* c, int what, void* stream, int* block_out, int* degree_out) {
    if (c && c->oct) return fail(STOKES_EMESH, "not available for octree meshes");
    if (!c) return fail(STOKES_EINVAL, "null context");
    if (what < 0 || what > 3) return fail(STOKES_EINVAL, "what must be a combination of 1 and 2");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Level& F = c->lev[c->L - 1];
    const size_t n = F.g.n_u;
    if (!c->tune_x) {
        CKS(dalloc(c, &c->tune_x, n));
        CKS(dalloc(c, &c->tune_r, n));
        CKS(dalloc(c, &c->tune_b, n));
    }
    // seeded right-hand side with zero constrained entries
    CK(launch_splitmix_vector(n, 4242, nullptr, c->tu, s));
    CK(launch_cast_d2f(n, c->tu, c->tune_b, s));
    CK(launch_zero_boundary<float>(F.g, c->tune_b, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    stokes_status st = STOKES_OK;
    if ((what & 1) && c->opt.vmult_kernel == 0) {   // only the cell kernel has a block size
        // threads per block of the cell kernel: the fastest FP32 level operator on the finest level
        float best = 1e30f;
        int best_bs = c->cell_block;
        for (int bs : {64, 128, 256}) {
            c->cell_block = bs;
            for (int it = 0; it < 2; ++it) st = vmult_level<float>(c, c->L - 1, c->tune_b, c->tune_r, s);
            cudaEventRecord(e0, s);
            for (int it = 0; it < 10 && st == STOKES_OK; ++it) st = vmult_level<float>(c, c->L - 1, c->tune_b, c->tune_r, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st != STOKES_OK) break;
            if (ms < best) { best = ms; best_bs = bs; }
        }
        c->cell_block = best_bs;
        if (st == STOKES_OK) st = drop_graphs(c);
    }
    if (st == STOKES_OK && (what & 2)) {
        // Chebyshev degree: wall time of a short FGMRES solve (FP32 V-cycle, relative residual 1e-3,
        // zero guess, the context's own right-hand side [F; 0]) for each candidate degree
        const int keep = c->opt.cheb_degree;
        if ((st = ensure_krylov(c)) == STOKES_OK && !c->tune_up) st = dalloc(c, &c->tune_up, c->N);
        double best_t = 1e300;
        int best_deg = keep;
        const LevelGeom& g = F.g;
        for (int deg = 3; deg <= 6 && st == STOKES_OK; ++deg) {
            c->opt.cheb_degree = deg;
            if ((st = drop_graphs(c)) != STOKES_OK) break;
            for (int rep = 0; rep < 2 && st == STOKES_OK; ++rep) {     // first run captures the graph
                cudaMemcpyAsync(c->bvec, c->F, g.n_u * sizeof(double), cudaMemcpyDeviceToDevice, s);
                cudaMemsetAsync(c->bvec + g.n_u, 0, g.n_p * sizeof(double), s);
                cudaMemsetAsync(c->tune_up, 0, c->N * sizeof(double), s);
                const auto t0 = std::chrono::steady_clock::now();
                stokes_solve_info info{};
                stokes_status sst = fgmres(c, STOKES_FP32, c->bvec, c->tune_up, 1e-3, 2000, &info, s);
                const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (sst != STOKES_OK && sst != STOKES_NOT_CONVERGED) st = sst;
                if (rep == 1 && sst == STOKES_OK && t < best_t) { best_t = t; best_deg = deg; }
            }
        }
        g_last_error.clear();
        c->opt.cheb_degree = best_deg;
        if (st == STOKES_OK) st = drop_graphs(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != STOKES_OK) return st;
    if (block_out) *block_out = c->opt.vmult_kernel != 0 ? 0 : c->cell_block;
    if (degree_out) *degree_out = c->opt.cheb_degree;
    return STOKES_OK;
}

stokes_status stokes_batch_solve(int n_problems, stokes_ctx* const* ctxs, int vcycle_prec,
                                 const double* const* rhs_devs, double* const* up_devs, double rtol, int max_it,
                                 stokes_solve_info* infos, void* const* streams) {
    if (n_problems < 1 || !ctxs || !up_devs) return fail(STOKES_EINVAL, "null argument or no problems");
    for (int i = 0; i < n_problems; ++i) {
        if (ctxs[i] && ctxs[i]->oct) return fail(STOKES_EMESH, "batched solves take uniform meshes");
        if (ctxs[i] && (ctxs[i]->opt.outer_solver == 1 || ctxs[i]->opt.outer_solver == 3))
            return fail(STOKES_EINVAL, "batched solves use (F)GMRES");
    }
    if (vcycle_prec != STOKES_FP32 && vcycle_prec != STOKES_FP64) return fail(STOKES_EINVAL, "bad precision");
    if (!(rtol > 0.0) || max_it < 1) return fail(STOKES_EINVAL, "bad rtol or max_it");
    for (int i = 0; i < n_problems; ++i) {
        if (!ctxs[i] || !up_devs[i]) return fail(STOKES_EINVAL, "null context or solution vector");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return fail(STOKES_EINVAL, "a context appears twice in the batch");
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<cudaStream_t> own;
    std::vector<FgmresRun> runs(n_problems);
    std::vector<stokes_solve_info> local(n_problems);
    stokes_status st = STOKES_OK;
    for (int i = 0; i < n_problems && st == STOKES_OK; ++i) {
        stokes_ctx* c = ctxs[i];
        cudaStream_t s = streams ? static_cast<cudaStream_t>(streams[i]) : nullptr;
        if (!streams) {
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { st = fail(STOKES_ECUDA, "stream"); break; }
            own.push_back(s);
        }
        st = ensure_krylov(c);
        if (st != STOKES_OK) break;
        const LevelGeom& g = c->lev[c->L - 1].g;
        const double* b = rhs_devs ? rhs_devs[i] : nullptr;
        if (!b) {
            if (cudaMemcpyAsync(c->bvec, c->F, g.n_u * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemsetAsync(c->bvec + g.n_u, 0, g.n_p * sizeof(double), s) != cudaSuccess) {
                st = fail(STOKES_ECUDA, "rhs copy");
                break;
            }
            b = c->bvec;
        }
        st = fgmres_init(runs[i], c, vcycle_prec, b, up_devs[i], rtol, max_it, infos ? &infos[i] : &local[i], s);
    }
    if (st == STOKES_OK) {
        if (batch_vcycle_eligible(runs)) {
            // one persistent launch per round runs the FP32 V-cycles of all problems
            BatchVcycle B;
            st = batch_vcycle_setup(B, runs);
            for (FgmresRun& r : runs) r.batched = true;
            if (st == STOKES_OK) st = fgmres_drive_batched(runs, B);
            if (st == STOKES_TIMEOUT)
                for (int i = 0; i < n_problems; ++i) (infos ? infos[i] : local[i]).status = STOKES_TIMEOUT;
        } else {
            st = fgmres_drive(runs);
        }
    }
    for (cudaStream_t s : own) cudaStreamDestroy(s);
    if (st != STOKES_OK) return st;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stokes_status worst = STOKES_OK;
    for (int i = 0; i < n_problems; ++i) {
        if (infos) infos[i].seconds = secs;
        if (runs[i].st != STOKES_OK && worst == STOKES_OK) worst = runs[i].st;
    }
    if (worst != STOKES_OK) return fail(worst, "at least one problem did not converge");
    return STOKES_OK;
}

stokes_status stokes_solve_host(stokes_ctx* c, int vcycle_prec, const double* rhs_host, double* up_host,
                                double rtol, int max_it, stokes_solve_info* info, void* stream) {
    if (!c || !up_host) return fail(STOKES_EINVAL, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t N = active_nu(c) + active_np(c);
    const auto t0 = std::chrono::steady_clock::now();
    if (!c->h_up_dev) {
        CKS(dalloc(c, &c->h_up_dev, N));
        CKS(dalloc(c, &c->h_rhs_dev, N));
    }
    const double* rhs_dev = nullptr;
    if (rhs_host) {
        CK(cudaMemcpyAsync(c->h_rhs_dev, rhs_host, N * sizeof(double), cudaMemcpyHostToDevice, s));
        rhs_dev = c->h_rhs_dev;
    }
    CK(cudaMemsetAsync(c->h_up_dev, 0, N * sizeof(double), s));
    stokes_status st = stokes_solve(c, vcycle_prec, rhs_dev, c->h_up_dev, rtol, max_it, info, stream);
    if (st != STOKES_OK && st != STOKES_NOT_CONVERGED) return st;
    CK(cudaMemcpyAsync(up_host, c->h_up_dev, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (info) info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

stokes_status stokes_get_viscosity(stokes_ctx* c, int level, double* mu_dev, void* stream) {
    if (c && c->oct) {
        if (!mu_dev) return fail(STOKES_EINVAL, "null pointer");
        OctCtx& o = *c->oct;
        const double* src = level == -1 ? o.leaf_mu : nullptr;
        size_t n = level == -1 ? size_t(o.act.n_leaves) : 0;
        if (level >= 0 && level < int(o.lev.size())) {
            src = o.lev[level].v64.mu;
            n = size_t(o.lev[level].g.n_cells);
        }
        if (!src) return fail(STOKES_EINVAL, "level out of range");
        CK(cudaMemcpyAsync(mu_dev, src, n * sizeof(double), cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
        return STOKES_OK;
    }
    CKS(check_level(c, level));
    if (!mu_dev) return fail(STOKES_EINVAL, "null pointer");
    Level& Lv = c->lev[level];
    CK(cudaMemcpyAsync(mu_dev, Lv.v64.mu, Lv.g.cells * sizeof(double), cudaMemcpyDeviceToDevice,
                       static_cast<cudaStream_t>(stream)));
    return STOKES_OK;
}

stokes_status stokes_get_inv_diagonal(stokes_ctx* c, int level, double* dinv_dev, void* stream) {
    if (c && c->oct) {
        if (!dinv_dev) return fail(STOKES_EINVAL, "null pointer");
        if (level < 0 || level >= int(c->oct->lev.size())) return fail(STOKES_EINVAL, "level out of range");
        OctLevel& L = c->oct->lev[level];
        CK(cudaMemcpyAsync(dinv_dev, L.v64.dinv, 3 * L.g.nn * sizeof(double), cudaMemcpyDeviceToDevice,
                           static_cast<cudaStream_t>(stream)));
        return STOKES_OK;
    }
    CKS(check_level(c, level));
    if (!dinv_dev) return fail(STOKES_EINVAL, "null pointer");
    Level& Lv = c->lev[level];
    CK(cudaMemcpyAsync(dinv_dev, Lv.v64.dinv, Lv.g.n_u * sizeof(double), cudaMemcpyDeviceToDevice,
                       static_cast<cudaStream_t>(stream)));
    return STOKES_OK;
}

stokes_status stokes_get_lambda_max(stokes_ctx* c, int level, double* lam_host) {
    if (c && c->oct) {
        if (!lam_host) return fail(STOKES_EINVAL, "null pointer");
        if (level < 0 || level >= int(c->oct->lev.size())) return fail(STOKES_EINVAL, "level out of range");
        *lam_host = c->oct->lev[level].lam_max;
        return STOKES_OK;
    }
    CKS(check_level(c, level));
    if (!lam_host) return fail(STOKES_EINVAL, "null pointer");
    *lam_host = c->lev[level].lam_max;
    return STOKES_OK;
}

stokes_status stokes_get_rhs(stokes_ctx* c, double* F_dev, void* stream) {
    if (!c || !F_dev) return fail(STOKES_EINVAL, "null argument");
    CK(cudaMemcpyAsync(F_dev, c->F, active_nu(c) * sizeof(double), cudaMemcpyDeviceToDevice,
                       static_cast<cudaStream_t>(stream)));
    return STOKES_OK;
}

stokes_status stokes_prolongate(stokes_ctx* c, int fine_level, int prec, const void* coarse, void* fine, int add,
                                void* stream) {
    if (c && c->oct) return fail(STOKES_EMESH, "not available for octree meshes");
    CKS(check_level(c, fine_level));
    if (fine_level < 1) return fail(STOKES_EINVAL, "fine_level must be >= 1");
    if (!coarse || !fine) return fail(STOKES_EINVAL, "null vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const LevelGeom& g = c->lev[fine_level].g;
    if (prec == STOKES_FP32)
        CK(launch_prolongate<float>(g, static_cast<const float*>(coarse), static_cast<float*>(fine), add != 0, s));
    else if (prec == STOKES_FP64)
        CK(launch_prolongate<double>(g, static_cast<const double*>(coarse), static_cast<double*>(fine), add != 0, s));
    else
        return fail(STOKES_EINVAL, "bad precision");
    return STOKES_OK;
}

stokes_status stokes_restrict(stokes_ctx* c, int fine_level, int prec, const void* fine, void* coarse,
                              void* stream) {
    if (c && c->oct) return fail(STOKES_EMESH, "not available for octree meshes");
    CKS(check_level(c, fine_level));
    if (fine_level < 1) return fail(STOKES_EINVAL, "fine_level must be >= 1");
    if (!coarse || !fine) return fail(STOKES_EINVAL, "null vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const LevelGeom& g = c->lev[fine_level].g;
    if (prec == STOKES_FP32)
        CK(launch_restrict<float>(g, static_cast<const float*>(fine), static_cast<float*>(coarse), s));
    else if (prec == STOKES_FP64)
        CK(launch_restrict<double>(g, static_cast<const double*>(fine), static_cast<double*>(coarse), s));
    else
        return fail(STOKES_EINVAL, "bad precision");
    return STOKES_OK;
}

stokes_status stokes_smooth(stokes_ctx* c, int level, int prec, const void* b, void* x, int zero_guess,
                            void* stream) {
    if (c && c->oct) return fail(STOKES_EMESH, "not available for octree meshes");
    CKS(check_level(c, level));
    if (level < 1) return fail(STOKES_EINVAL, "smoothing needs level >= 1");
    if (!b || !x) return fail(STOKES_EINVAL, "null vector");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == STOKES_FP32) {
        const float* bf = static_cast<const float*>(b);
        float* xf = static_cast<float*>(x);
        return fused_level<float>(c, level) ? smooth_fused<float>(c, level, bf, xf, zero_guess != 0, nullptr, s)
                                            : smooth<float>(c, level, bf, xf, zero_guess != 0, s);
    }
    if (prec == STOKES_FP64) {
        const double* bd = static_cast<const double*>(b);
        double* xd = static_cast<double*>(x);
        return fused_level<double>(c, level) ? smooth_fused<double>(c, level, bd, xd, zero_guess != 0, nullptr, s)
                                             : smooth<double>(c, level, bd, xd, zero_guess != 0, s);
    }
    return fail(STOKES_EINVAL, "bad precision");
}

stokes_status stokes_coarse_solve(stokes_ctx* c, int prec, const void* b, void* x, void* stream) {
    if (c && c->oct) return fail(STOKES_EMESH, "not available for octree meshes");
    if (!c || !b || !x) return fail(STOKES_EINVAL, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == STOKES_FP32) return coarse_solve<float>(c, static_cast<const float*>(b), static_cast<float*>(x), s);
    if (prec == STOKES_FP64) return coarse_solve<double>(c, static_cast<const double*>(b), static_cast<double*>(x), s);
    return fail(STOKES_EINVAL, "bad precision");
}

stokes_status stokes_schur_inverse(stokes_ctx* c, const double* rp, double* zp, void* stream) {
    if (!c || !rp || !zp) return fail(STOKES_EINVAL, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return debug_status(c, s, schur_inverse(c, rp, zp, s));
}

stokes_status stokes_precondition(stokes_ctx* c, int vcycle_prec, const double* r, double* z, void* stream) {
    if (!c || !r || !z) return fail(STOKES_EINVAL, "null argument");
    if (vcycle_prec != STOKES_FP32 && vcycle_prec != STOKES_FP64) return fail(STOKES_EINVAL, "bad precision");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return debug_status(c, s, precondition(c, vcycle_prec, r, z, s));
}

}  // extern "C"
