// batch.cu -- one persistent, cooperative launch for the FP32 V-cycle of a whole batch of
// problems (batch.cuh). The phase bodies are the ones of the single-problem kernels: the cell
// operator of q2_basis.cuh with atomic adds into the level accumulator (brick.cu's cell kernel),
// the Chebyshev and residual epilogues, the transfers of transfer.cuh, the dense coarse solve.
// Visibility between phases comes from the grid barrier (release fences before the arrival,
// an acquire fence after it, then the block barrier): loads with reuse (the cell gathers, the
// transfers) go through L1; loads without reuse (the vector epilogues, the coarse solve) read
// through L2 only (ld.global.cg).
#include "batch.cuh"
#include "brick.cuh"
#include "prof.cuh"
#include "tcgen05.cuh"
#include "transfer.cuh"

#include <algorithm>

namespace stk {

namespace {

// Grid barrier over all blocks of the cooperative launch, bounded by limit_ns of %globaltimer
// (0: gives up at once). On timeout, or when another block has given up, it records bit 1 in the
// status word and returns false: the caller leaves the kernel.
__device__ bool grid_sync(unsigned* count, unsigned* gen, unsigned nblocks, unsigned long long limit_ns,
                          unsigned* status) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (limit_ns == 0) {
            ok = 0;
        } else {
            const unsigned g0 = *reinterpret_cast<volatile unsigned*>(gen);
            __threadfence();
            if (atomicAdd(count, 1u) + 1u == nblocks) {
                atomicExch(count, 0u);
                __threadfence();
                atomicAdd(gen, 1u);
            } else {
                const unsigned long long t0 = tc::globaltimer();
                while (*reinterpret_cast<volatile unsigned*>(gen) == g0) {
                    if (*reinterpret_cast<volatile unsigned*>(status) & 2u) { ok = 0; break; }
                    if (tc::globaltimer() - t0 >= limit_ns) { ok = 0; break; }
                    __nanosleep(64);
                }
            }
            asm volatile("fence.acq_rel.gpu;" ::: "memory");   // acquire: the other blocks' writes
        }
        if (!ok) atomicOr(status, 2u);
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// acc += A_cell x for cell `cell` of the level (boundary nodes neither read nor written).
__device__ __forceinline__ void level_cell(const BatchLevel& L, size_t cell) {
    const int n = L.n, M = L.M;
    const int ci = int(cell % n), cj = int((cell / n) % n), ck = int(cell / (size_t(n) * n));
    const float* src = L.x + (size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck)));
    float u[3][27], w[3][27];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool bnd = bj || (2 * ci + i == 0) || (2 * ci + i == M - 1);
                const int off = i + M * (j + M * k);
#pragma unroll
                for (int c = 0; c < 3; ++c) u[c][i + 3 * j + 9 * k] = bnd ? 0.0f : src[c * L.nodes + off];
            }
        }
    }
    q2::cell_A(u, w);
    const float s = __ldg(L.mu + cell) * L.h;
    float* out = L.acc + (size_t(2 * ci) + size_t(M) * (size_t(2 * cj) + size_t(M) * size_t(2 * ck)));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool bk = (2 * ck + k == 0) || (2 * ck + k == M - 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const bool bj = bk || (2 * cj + j == 0) || (2 * cj + j == M - 1);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (bj || (2 * ci + i == 0) || (2 * ci + i == M - 1)) continue;
                const int off = i + M * (j + M * k);
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(out + c * L.nodes + off, s * w[c][i + 3 * j + 9 * k]);
            }
        }
    }
}

// One work item of a phase for problem p. Items beyond the phase's count for p do nothing; the
// coarse solve takes one warp per row, so a whole warp always runs it or skips it.
__device__ __forceinline__ void run_item(const BatchProblem& p, const BatchPhase& ph, size_t item) {
    const int l = p.L - 1 - ph.depth;
    switch (ph.op) {
        case BOP_ZERO: {
            const BatchLevel& C = p.lev[0];
            if (item < C.n_u) C.x[item] = 0.0f;
            return;
        }
        case BOP_COARSE: {
            const BatchLevel& C = p.lev[0];
            const int row = int(item >> 5), lane = int(item & 31);
            if (row >= p.nf) return;
            const double* a = p.Ainv + size_t(row) * p.nf;
            double sum = 0.0;
            for (int j = lane; j < p.nf; j += 32) sum += __ldg(a + j) * double(__ldcg(C.b + __ldg(p.free_idx + j)));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) C.x[__ldg(p.free_idx + row)] = float(sum);
            return;
        }
        default:
            break;
    }
    const BatchLevel& L = p.lev[l];
    switch (ph.op) {
        case BOP_CHEB0:
            if (item < L.n_u) {
                const float d = L.c2[0] * (__ldg(L.dinv + item) * __ldcg(L.b + item));
                L.d[item] = d;
                L.x[item] = d;
            }
            return;
        case BOP_LEVELOP:
            if (item < size_t(L.n) * L.n * L.n) level_cell(L, item);
            return;
        case BOP_CONSUME_CHEB:
            if (item < L.n_u) {
                const float c1 = L.c1[ph.k], c2 = L.c2[ph.k];
                const float r = __ldg(L.dinv + item) * (__ldcg(L.b + item) - __ldcg(L.acc + item));
                const float d = (c1 != 0.0f ? c1 * __ldcg(L.d + item) : 0.0f) + c2 * r;
                L.d[item] = d;
                L.x[item] = __ldcg(L.x + item) + d;
                L.acc[item] = 0.0f;
            }
            return;
        case BOP_CONSUME_RESID:
            if (item < L.n_u) {
                L.r[item] = __ldcg(L.b + item) - __ldcg(L.acc + item);
                L.acc[item] = 0.0f;
            }
            return;
        case BOP_RESTRICT: {
            const BatchLevel& C = p.lev[l - 1];
            if (item < C.nodes) restrict_node<float, false>(L.n, L.r, C.b, item);
            return;
        }
        case BOP_PROLONG: {
            const BatchLevel& C = p.lev[l - 1];
            if (item < L.nodes) prolongate_node<float, false>(L.n, C.x, L.x, true, item);
            return;
        }
    }
}

__global__ void __launch_bounds__(kBatchThreads, 1) k_batch_vcycle(BatchLaunch bl) {
    __shared__ unsigned tile_s;
    unsigned* bar_count = bl.counters + bl.n_phases;
    unsigned* bar_gen = bar_count + 1;
    for (int ph = 0; ph < bl.n_phases; ++ph) {
        const BatchPhase phase = bl.phases[ph];
        const unsigned* pre = bl.tile_prefix + size_t(ph) * (bl.n_problems + 1);
        const unsigned ntiles = pre[bl.n_problems];
        for (;;) {
            if (threadIdx.x == 0) tile_s = atomicAdd(&bl.counters[ph], 1u);   // the work queue
            __syncthreads();
            const unsigned t = tile_s;
            __syncthreads();
            if (t >= ntiles) break;
            int lo = 0, hi = bl.n_problems - 1;   // the problem whose tiles hold t: last p with pre[p] <= t
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= t) lo = mid;
                else hi = mid - 1;
            }
            if (!bl.active[lo]) continue;
            const int per = batch_items_per_thread(phase.op);
            const size_t base = size_t(t - pre[lo]) * kBatchThreads * per + threadIdx.x;
            for (int q = 0; q < per; ++q) run_item(bl.problems[lo], phase, base + size_t(q) * kBatchThreads);
        }
        if (!grid_sync(bar_count, bar_gen, gridDim.x, bl.wait_ns, bl.status)) return;
    }
}

}  // namespace

int batch_build_phases(const int* levels, int P, int degree, BatchPhase* out, int capacity) {
    int lmax = 0;
    for (int p = 0; p < P; ++p) lmax = std::max(lmax, levels[p]);
    int n = 0;
    auto push = [&](int op, int d, int k) {
        if (n < capacity) out[n] = BatchPhase{op, d, k};
        ++n;
    };
    auto any = [&](auto pred) {
        for (int p = 0; p < P; ++p)
            if (pred(levels[p])) return true;
        return false;
    };
    for (int d = 0; d < lmax; ++d) {   // down: smoothing, residual, restriction; coarse solves at their depth
        if (any([&](int L) { return L - 1 == d; })) {
            push(BOP_ZERO, d, 0);
            push(BOP_COARSE, d, 0);
        }
        if (any([&](int L) { return L - 1 - d >= 1; })) {
            push(BOP_CHEB0, d, 0);
            for (int k = 1; k < degree; ++k) {
                push(BOP_LEVELOP, d, k);
                push(BOP_CONSUME_CHEB, d, k);
            }
            push(BOP_LEVELOP, d, 0);
            push(BOP_CONSUME_RESID, d, 0);
            push(BOP_RESTRICT, d, 0);
        }
    }
    for (int d = lmax - 2; d >= 0; --d) {   // up: prolongation, smoothing
        if (!any([&](int L) { return L - 1 - d >= 1; })) continue;
        push(BOP_PROLONG, d, 0);
        for (int k = 0; k < degree; ++k) {
            push(BOP_LEVELOP, d, k);
            push(BOP_CONSUME_CHEB, d, k);
        }
    }
    return n;
}

size_t batch_items(const BatchProblem& p, const BatchPhase& ph) {
    const int l = p.L - 1 - ph.depth;
    switch (ph.op) {
        case BOP_ZERO: return l == 0 ? p.lev[0].n_u : 0;
        case BOP_COARSE: return l == 0 ? size_t(p.nf) * 32 : 0;
        default: break;
    }
    if (l < 1) return 0;
    const BatchLevel& L = p.lev[l];
    switch (ph.op) {
        case BOP_CHEB0:
        case BOP_CONSUME_CHEB:
        case BOP_CONSUME_RESID: return L.n_u;
        case BOP_LEVELOP: return size_t(L.n) * L.n * L.n;
        case BOP_RESTRICT: return p.lev[l - 1].nodes;
        case BOP_PROLONG: return L.nodes;
    }
    return 0;
}

int batch_grid_blocks() {
    int dev = 0, sms = 0, per = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_vcycle, kBatchThreads, 0) != cudaSuccess) return 0;
    return sms * per;
}

cudaError_t launch_batch_vcycle(const BatchLaunch& bl, int blocks, cudaStream_t s) {
    const int most = batch_grid_blocks();
    if (most < 1) return cudaErrorCooperativeLaunchTooLarge;
    blocks = blocks < 1 ? 1 : (blocks > most ? most : blocks);
    cudaError_t e = cudaMemsetAsync(bl.counters, 0, sizeof(unsigned) * size_t(bl.n_phases + 2), s);
    if (e != cudaSuccess) return e;
    BatchLaunch arg = bl;
    void* args[] = {&arg};
    prof_begin(PROF_VMULT_F32, s);
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_batch_vcycle), dim3(blocks), dim3(kBatchThreads), args,
                                    0, s);
    prof_end(PROF_VMULT_F32, s);
    prof_count(1);
    return e;
}

}  // namespace stk
