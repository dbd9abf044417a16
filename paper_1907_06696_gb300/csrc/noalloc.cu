// noalloc.cu -- a variant of the Schur-complement approximation S_hat^-1 that
// needs no context and allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc, so they cannot create a
// stokes_ctx (stokes_setup allocates its tables and work vectors). Examples are
// host applications whose device memory is entirely reserved up front by
// their own pool allocator, so a later cudaMalloc fails, and code that must
// not make the implicit device-wide synchronisation a cudaMalloc or cudaFree
// can cause (for example inside a time-critical step of a coupled simulation).
// They pass the cell viscosity, the input and the output; the three work
// vectors the Chebyshev iteration needs live in the fixed device array below.
//
// Limits and sharing:
// * The array holds 3 * STOKES_NOALLOC_MAX_NP doubles (~0.86 MB). Every GPU
//   that loads this library keeps it resident until the process exits.
// * All calls share it, and it keeps whatever the last call left there. The
//   work vectors are fully written before they are read (the accumulation
//   buffer of the mass matrix is cleared on the stream first), so no call
//   depends on old contents. Calls whose kernels overlap on the GPU (two
//   streams, or two host threads) race on the array and give wrong results:
//   issue them on one stream or serialise them.
// * The device address of the array is looked up with cudaGetSymbolAddress
//   on the first call made on each device (with that device current); make
//   that first call before any stream capture. Later calls on a stream that
//   is not capturing look it up again (a cheap table lookup), so a context
//   that was torn down and re-created (cudaDeviceReset), which may place the
//   array elsewhere, never gets a stale address; calls on a capturing stream
//   use the address cached for the device.
#include "../../include/stokes.h"
#include "internal.cuh"

#include <mutex>
#include <string>

namespace {

constexpr size_t kMaxNp = STOKES_NOALLOC_MAX_NP;
constexpr int kMaxDevices = 64;

// d (Chebyshev direction), t (mass-matrix product), dinv (1 / diag M_p).
static __device__ __align__(256) double g_schur_scratch[3 * kMaxNp];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_schur_scratch for the current device: looked up on the first call on the
// device and again on every call whose stream is not capturing; a capturing stream uses the
// cached address (the lookup may load the module, which capture does not allow).
cudaError_t scratch_for_current_device(cudaStream_t s, double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
        if (cap != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_schur_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" stokes_status stokes_schur_inverse_noalloc(int n, const double* mu_dev, const double* rp_dev,
                                                      double* zp_dev, int degree, void* stream) {
    using namespace stk;
    // largest n with (n + 1)^3 <= kMaxNp, checked before any size arithmetic
    constexpr int kMaxN = 32;
    static_assert(size_t(kMaxN + 1) * (kMaxN + 1) * (kMaxN + 1) <= kMaxNp, "array too small for kMaxN");
    static_assert(size_t(kMaxN + 2) * (kMaxN + 2) * (kMaxN + 2) > kMaxNp, "kMaxN not the largest size");
    if (n < 1 || n > kMaxN || degree < 0 || !mu_dev || !rp_dev || !zp_dev) return STOKES_EINVAL;
    const LevelGeom g = make_geom(n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* base = nullptr;
    if (scratch_for_current_device(s, &base) != cudaSuccess) return STOKES_ECUDA;
    double* d = base;
    double* t = base + kMaxNp;
    double* dinv = base + 2 * kMaxNp;
    // Jacobi-Chebyshev on M_p over [1/8, 27/8], zero initial guess (the same
    // recurrence and coefficients as stokes_schur_inverse); degree 0 is
    // S_hat = diag(M_p) itself (Section 3.4), a first coefficient of 1.
    const double lo = 1.0 / 8.0, hi = 27.0 / 8.0;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    const double c0 = degree == 0 ? 1.0 : 1.0 / theta;
    if (launch_mass_p_diag(g, mu_dev, t, nullptr, s) != cudaSuccess) return STOKES_ECUDA;
    if (launch_recip(g.n_p, t, dinv, s) != cudaSuccess) return STOKES_ECUDA;
    if (launch_cheb_update<double>(g.n_p, rp_dev, nullptr, dinv, d, zp_dev, 0.0, c0, false, s) != cudaSuccess)
        return STOKES_ECUDA;
    for (int it = 1; it < degree; ++it) {
        if (launch_mass_p(g, mu_dev, zp_dev, t, s) != cudaSuccess) return STOKES_ECUDA;   // clears t first
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        if (launch_cheb_update<double>(g.n_p, rp_dev, t, dinv, d, zp_dev, rho_new * rho, 2.0 * rho_new / delta,
                                       true, s) != cudaSuccess)
            return STOKES_ECUDA;
        rho = rho_new;
    }
    return STOKES_OK;
}
