"""ctypes binding of libstokes_gb300.so (include/stokes.h).

Argument marshalling only: every function forwards to the C entry point of the
same name. Device vectors are passed as torch CUDA tensors (their data_ptr())
or raw integer addresses; streams default to torch's current CUDA stream.
A missing library raises immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstokes_gb300.so")
# the same library built with STOKES_DEBUG (index-map checks on the octree path)
DEBUG_LIB_PATH = os.path.join(HERE, "libstokes_gb300_debug.so")

STOKES_OK, STOKES_EINVAL, STOKES_ENOMEM, STOKES_ECUDA = 0, 1, 2, 3
STOKES_NOT_CONVERGED, STOKES_BREAKDOWN, STOKES_TIMEOUT, STOKES_EMESH = 4, 5, 6, 7
STOKES_FP64, STOKES_FP32 = 0, 1
BLOCK_A, BLOCK_B, BLOCK_BT, BLOCK_MP, BLOCK_STOKES = 0, 1, 2, 3, 4


class StokesError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s failed: status %d (%s)" % (where, status, msg))
        self.status = status


class stokes_mesh(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("n_levels", C.c_int)]


class stokes_mu(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_sinkers", C.c_int), ("centres", C.POINTER(C.c_double)),
                ("mu_min", C.c_double), ("mu_max", C.c_double), ("delta", C.c_double),
                ("omega", C.c_double), ("beta", C.c_double), ("mu_q", C.POINTER(C.c_double))]


class stokes_bc(C.Structure):
    _fields_ = [("noslip_faces", C.c_uint32)]


class stokes_octree(C.Structure):
    _fields_ = [("coarsest_level", C.c_int), ("n_leaves", C.c_int64), ("leaf_keys", C.POINTER(C.c_uint64))]


class stokes_options(C.Structure):
    _fields_ = [("cheb_degree", C.c_int), ("smoothing_range", C.c_double), ("eig_safety", C.c_double),
                ("lanczos_steps", C.c_int), ("schur_degree", C.c_int), ("restart", C.c_int),
                ("outer_arith", C.c_int), ("vmult_kernel", C.c_int), ("graphs", C.c_int), ("precond_kind", C.c_int),
                ("outer_solver", C.c_int), ("idr_s", C.c_int), ("gram_schmidt", C.c_int),
                ("wait_limit_s", C.c_double), ("batch_vcycle", C.c_int), ("fused_smoother", C.c_int)]


class stokes_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("rel_residual_true", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# name -> (restype, argtypes); mirrors include/stokes.h
_P = C.c_void_p
_SIGS = {
    "stokes_default_options": (None, [C.POINTER(stokes_options)]),
    "stokes_setup": (C.c_int, [C.POINTER(stokes_mesh), C.POINTER(stokes_mu), C.POINTER(stokes_bc),
                               C.POINTER(stokes_options), _P, C.POINTER(_P)]),
    "stokes_destroy": (None, [_P]),
    "stokes_strerror": (C.c_char_p, [C.c_int]),
    "stokes_last_error": (C.c_char_p, []),
    "stokes_size": (C.c_size_t, [_P, C.c_int, C.c_int]),
    "stokes_vmult": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "gmg_vcycle": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "stokes_solve": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.POINTER(stokes_solve_info), _P]),
    "stokes_solve_host": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.POINTER(stokes_solve_info), _P]),
    "stokes_batch_solve": (C.c_int, [C.c_int, C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(_P), C.c_double,
                                     C.c_int, C.POINTER(stokes_solve_info), C.POINTER(_P)]),
    "stokes_get_viscosity": (C.c_int, [_P, C.c_int, _P, _P]),
    "stokes_get_inv_diagonal": (C.c_int, [_P, C.c_int, _P, _P]),
    "stokes_get_lambda_max": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double)]),
    "stokes_get_rhs": (C.c_int, [_P, _P, _P]),
    "stokes_prolongate": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int, _P]),
    "stokes_restrict": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    "stokes_smooth": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_int, _P]),
    "stokes_coarse_solve": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "stokes_schur_inverse": (C.c_int, [_P, _P, _P, _P]),
    "stokes_precondition": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "stokes_schur_inverse_noalloc": (C.c_int, [C.c_int, _P, _P, _P, C.c_int, _P]),
    "stokes_device_status": (C.c_int, [_P, _P]),
    "stokes_debug_alloc_limit": (C.c_int, [C.c_longlong]),
    "stokes_debug_build": (C.c_int, []),
    "stokes_debug_index_cut": (C.c_int, [_P, C.c_int, C.c_longlong]),
    "stokes_set_batch_vcycle": (C.c_int, [_P, C.c_int]),
    "stokes_autotune": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "stokes_profile": (C.c_int, [C.c_int]),
    "stokes_profile_read": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]),
    "stokes_launch_count": (C.c_longlong, []),
    "stokes_probe_fma": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "stokes_octree_sinker_mesh": (C.c_int, [C.c_int, C.c_int, _P, _P, C.c_double, C.c_double, _P, C.c_int64,
                                            C.POINTER(C.c_int64)]),
    "stokes_setup_octree": (C.c_int, [C.POINTER(stokes_octree), C.POINTER(stokes_mu), C.POINTER(stokes_bc),
                                      C.POINTER(stokes_options), _P, C.POINTER(_P)]),
    "stokes_octree_table": (C.c_size_t, [_P, C.c_int, C.c_int, _P, C.c_size_t]),
    "stokes_octree_refine_gradient": (C.c_int, [C.POINTER(stokes_octree), _P, C.c_double, _P, _P, C.c_int64,
                                                C.POINTER(C.c_int64)]),
}

PROF_CLASSES = ["vmult_A_fp32", "vmult_A_fp64", "stokes_fp64", "bt_fp64", "mass_p", "transfer",
                "smoother_vec", "krylov_vec", "coarse", "cast", "residual_fp64"]


def open_library(path: str):
    """Open one build of the library with the signatures set (raises if it is missing)."""
    if not os.path.exists(path):
        raise RuntimeError("%s not found; run __graft_entry__.build() first" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(path: str = LIB_PATH):
    """Load the library that every function of this module calls (once per process)."""
    global _lib
    if _lib is None:
        _lib = open_library(path)
    return _lib


class use_library:
    """Context manager: the functions of this module call `lib` (from open_library) inside the
    block, e.g. the STOKES_DEBUG build in its tests. A Context is destroyed by the build that made it."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        global _lib
        load()
        self.saved, _lib = _lib, self.lib
        return self.lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array (host buffers)
        return x.ctypes.data
    raise TypeError("expected a tensor, array or integer address, got %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status, where):
    if status != STOKES_OK:
        lib = load()
        raise StokesError(status, where, lib.stokes_last_error().decode())


class Context:
    """Owns one stokes_ctx; destroyed with the object or by close()."""

    def __init__(self, handle):
        self.handle = handle
        self.lib = load()   # the build that made the handle destroys it

    def close(self):
        if self.handle:
            self.lib.stokes_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def size(self, level=-1, what=0):
        return int(self.lib.stokes_size(self.handle, level, what))

    @property
    def n_u(self):
        return self.size(-1, 0)

    @property
    def n_p(self):
        return self.size(-1, 1)

    @property
    def n_levels(self):
        return self.size(-1, 4)


def stokes_default_options():
    o = stokes_options()
    load().stokes_default_options(C.byref(o))
    return o


def stokes_setup(n, n_levels, centres=None, mu_min=1.0, mu_max=1.0, delta=200.0, omega=0.1, beta=10.0,
                 mu_q=None, options=None, stream=None) -> Context:
    """stokes_setup for a uniform n^3 mesh. Sinker viscosity (kind 0) unless mu_q
    (host float64 array of n^3 * 27 Gauss-point values) is given (kind 1)."""
    import numpy as np
    lib = load()
    mesh = stokes_mesh(0, int(n), int(n_levels))
    mu = stokes_mu()
    keep = []
    if mu_q is not None:
        q = np.ascontiguousarray(mu_q, dtype=np.float64)
        keep.append(q)
        mu.kind = 1
        mu.mu_q = q.ctypes.data_as(C.POINTER(C.c_double))
    else:
        cen = np.ascontiguousarray(np.zeros((0, 3)) if centres is None else centres, dtype=np.float64).reshape(-1, 3)
        keep.append(cen)
        mu.kind = 0
        mu.n_sinkers = cen.shape[0]
        mu.centres = cen.ctypes.data_as(C.POINTER(C.c_double)) if cen.size else None
        mu.mu_min, mu.mu_max, mu.delta, mu.omega, mu.beta = mu_min, mu_max, delta, omega, beta
    bc = stokes_bc(0x3F)
    h = C.c_void_p()
    st = lib.stokes_setup(C.byref(mesh), C.byref(mu), C.byref(bc), C.byref(options) if options else None,
                          _stream(stream), C.byref(h))
    _check(st, "stokes_setup")
    return Context(h.value)


def stokes_setup_problem(prob, options=None, stream=None) -> Context:
    """stokes_setup from a sinker_inputs.SinkerProblem."""
    return stokes_setup(prob.n, prob.n_levels, prob.centres, prob.mu_min, prob.mu_max, prob.delta, prob.omega,
                        prob.beta, options=options, stream=stream)


def stokes_octree_sinker_mesh(base_level, centres, max_levels, shell_radius=0.05, shell_half_width=0.02):
    """Leaf keys (numpy uint64, sorted) of the refined and 2:1-balanced sinker octree."""
    import numpy as np
    lib = load()
    cen = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    lv = np.ascontiguousarray(max_levels, dtype=np.int32)
    n = C.c_int64(0)
    _check(lib.stokes_octree_sinker_mesh(int(base_level), cen.shape[0], cen.ctypes.data, lv.ctypes.data,
                                         float(shell_radius), float(shell_half_width), None, 0, C.byref(n)),
           "stokes_octree_sinker_mesh")
    keys = np.empty(n.value, dtype=np.uint64)
    _check(lib.stokes_octree_sinker_mesh(int(base_level), cen.shape[0], cen.ctypes.data, lv.ctypes.data,
                                         float(shell_radius), float(shell_half_width), keys.ctypes.data,
                                         keys.size, C.byref(n)), "stokes_octree_sinker_mesh")
    return keys


def stokes_setup_octree(leaf_keys, coarsest_level, centres, mu_min, mu_max, delta=200.0, omega=0.1, beta=10.0,
                        options=None, stream=None) -> Context:
    """stokes_setup_octree for the given leaves with the sinker viscosity."""
    import numpy as np
    lib = load()
    keys = np.ascontiguousarray(leaf_keys, dtype=np.uint64)
    mesh = stokes_octree(int(coarsest_level), keys.size, keys.ctypes.data_as(C.POINTER(C.c_uint64)))
    cen = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    mu = stokes_mu()
    mu.kind = 0
    mu.n_sinkers = cen.shape[0]
    mu.centres = cen.ctypes.data_as(C.POINTER(C.c_double)) if cen.size else None
    mu.mu_min, mu.mu_max, mu.delta, mu.omega, mu.beta = mu_min, mu_max, delta, omega, beta
    bc = stokes_bc(0x3F)
    h = C.c_void_p()
    st = lib.stokes_setup_octree(C.byref(mesh), C.byref(mu), C.byref(bc), C.byref(options) if options else None,
                                 _stream(stream), C.byref(h))
    _check(st, "stokes_setup_octree")
    return Context(h.value)


def stokes_setup_octree_problem(prob, options=None, stream=None) -> Context:
    """Mesh (stokes_octree_sinker_mesh) and set-up for a sinker_inputs.OctreeProblem."""
    keys = stokes_octree_sinker_mesh(prob.base_level, prob.centres, prob.max_levels, prob.shell_radius,
                                     prob.shell_half_width)
    return stokes_setup_octree(keys, prob.coarsest_level, prob.centres, prob.mu_min, prob.mu_max, prob.delta,
                               prob.omega, prob.beta, options=options, stream=stream)


def stokes_octree_refine_gradient(leaf_keys, coarsest_level, u_active, fraction=1.0 / 7.0):
    """Gradient-indicator refinement on the host: (new sorted leaf keys, indicators of the given
    leaves in increasing key order). u_active: host array, the active velocity of that mesh."""
    import numpy as np
    lib = load()
    keys = np.ascontiguousarray(leaf_keys, dtype=np.uint64)
    mesh = stokes_octree(int(coarsest_level), keys.size, keys.ctypes.data_as(C.POINTER(C.c_uint64)))
    u = np.ascontiguousarray(u_active, dtype=np.float64)
    eta = np.empty(keys.size, dtype=np.float64)
    n = C.c_int64(0)
    # each leaf is split at most once by the refinement and its balance (refining every leaf once
    # gives a balanced tree that contains the minimal one), so 8 n keys suffice
    out = np.empty(8 * keys.size, dtype=np.uint64)
    st = lib.stokes_octree_refine_gradient(C.byref(mesh), u.ctypes.data, float(fraction), eta.ctypes.data,
                                           out.ctypes.data, out.size, C.byref(n))
    if st == STOKES_EINVAL and n.value > out.size:
        out = np.empty(n.value, dtype=np.uint64)
        st = lib.stokes_octree_refine_gradient(C.byref(mesh), u.ctypes.data, float(fraction), eta.ctypes.data,
                                               out.ctypes.data, out.size, C.byref(n))
    _check(st, "stokes_octree_refine_gradient")
    return out[:n.value].copy(), eta


_TABLE_DTYPES = {0: "uint64", 1: "uint64", 2: "uint64", 3: "uint64", 4: "uint8", 5: "int32"}


def stokes_octree_table(ctx, which, level=0):
    """Host copy of an octree table (numpy array), or the count for which = 6, 7."""
    import numpy as np
    lib = load()
    n = int(lib.stokes_octree_table(ctx.handle, which, level, None, 0))
    if which not in _TABLE_DTYPES:
        return n
    out = np.empty(n, dtype=_TABLE_DTYPES[which])
    if n:
        lib.stokes_octree_table(ctx.handle, which, level, out.ctypes.data, n)
    return out


def stokes_vmult(ctx, level, block, prec, src, dst, stream=None):
    _check(load().stokes_vmult(ctx.handle, level, block, prec, _ptr(src), _ptr(dst), _stream(stream)), "stokes_vmult")


def gmg_vcycle(ctx, prec, rhs, x, stream=None):
    _check(load().gmg_vcycle(ctx.handle, prec, _ptr(rhs), _ptr(x), _stream(stream)), "gmg_vcycle")


def stokes_solve(ctx, vcycle_prec, rhs, up, rtol=1e-8, max_it=1000, stream=None, check=True):
    info = stokes_solve_info()
    st = load().stokes_solve(ctx.handle, vcycle_prec, _ptr(rhs), _ptr(up), rtol, max_it, C.byref(info),
                             _stream(stream))
    if check:
        _check(st, "stokes_solve")
    return info


def stokes_batch_solve(ctxs, vcycle_prec, ups, rtol=1e-8, max_it=1000, rhs=None, streams=None, check=True):
    """Solve the problems of several contexts together; ups: device solution vectors (in: guess)."""
    n = len(ctxs)
    infos = (stokes_solve_info * n)()
    P = C.c_void_p
    cptr = (P * n)(*[x.handle for x in ctxs])
    uptr = (P * n)(*[_ptr(u) for u in ups])
    rptr = (P * n)(*[_ptr(r) for r in rhs]) if rhs is not None else None
    sptr = (P * n)(*[_stream(s) for s in streams]) if streams is not None else None
    st = load().stokes_batch_solve(n, cptr, vcycle_prec, rptr, uptr, rtol, max_it, infos, sptr)
    if check:
        _check(st, "stokes_batch_solve")
    return list(infos)


def stokes_solve_host(ctx, vcycle_prec, rhs_host, up_host, rtol=1e-8, max_it=1000, stream=None, check=True):
    info = stokes_solve_info()
    st = load().stokes_solve_host(ctx.handle, vcycle_prec, _ptr(rhs_host), _ptr(up_host), rtol, max_it,
                                  C.byref(info), _stream(stream))
    if check:
        _check(st, "stokes_solve_host")
    return info


def stokes_get_viscosity(ctx, level, mu, stream=None):
    _check(load().stokes_get_viscosity(ctx.handle, level, _ptr(mu), _stream(stream)), "stokes_get_viscosity")


def stokes_get_inv_diagonal(ctx, level, dinv, stream=None):
    _check(load().stokes_get_inv_diagonal(ctx.handle, level, _ptr(dinv), _stream(stream)), "stokes_get_inv_diagonal")


def stokes_get_lambda_max(ctx, level):
    v = C.c_double()
    _check(load().stokes_get_lambda_max(ctx.handle, level, C.byref(v)), "stokes_get_lambda_max")
    return v.value


def stokes_get_rhs(ctx, F, stream=None):
    _check(load().stokes_get_rhs(ctx.handle, _ptr(F), _stream(stream)), "stokes_get_rhs")


def stokes_prolongate(ctx, fine_level, prec, coarse, fine, add=False, stream=None):
    _check(load().stokes_prolongate(ctx.handle, fine_level, prec, _ptr(coarse), _ptr(fine), int(add),
                                    _stream(stream)), "stokes_prolongate")


def stokes_restrict(ctx, fine_level, prec, fine, coarse, stream=None):
    _check(load().stokes_restrict(ctx.handle, fine_level, prec, _ptr(fine), _ptr(coarse), _stream(stream)),
           "stokes_restrict")


def stokes_smooth(ctx, level, prec, b, x, zero_guess, stream=None):
    _check(load().stokes_smooth(ctx.handle, level, prec, _ptr(b), _ptr(x), int(zero_guess), _stream(stream)),
           "stokes_smooth")


def stokes_coarse_solve(ctx, prec, b, x, stream=None):
    _check(load().stokes_coarse_solve(ctx.handle, prec, _ptr(b), _ptr(x), _stream(stream)), "stokes_coarse_solve")


def stokes_schur_inverse(ctx, rp, zp, stream=None):
    _check(load().stokes_schur_inverse(ctx.handle, _ptr(rp), _ptr(zp), _stream(stream)), "stokes_schur_inverse")


def stokes_precondition(ctx, vcycle_prec, r, z, stream=None):
    _check(load().stokes_precondition(ctx.handle, vcycle_prec, _ptr(r), _ptr(z), _stream(stream)),
           "stokes_precondition")


def stokes_set_batch_vcycle(ctx, mode):
    """How stokes_batch_solve runs the FP32 V-cycles when ctx comes first: 1 = one persistent launch
    for all problems per round, 0 = one captured graph per problem."""
    _check(load().stokes_set_batch_vcycle(ctx.handle, int(mode)), "stokes_set_batch_vcycle")


def stokes_device_status(ctx, stream=None):
    """Synchronise the stream, read and clear the context's device status word (raises
    StokesError with STOKES_TIMEOUT if a bounded wait inside a kernel gave up)."""
    _check(load().stokes_device_status(ctx.handle, _stream(stream)), "stokes_device_status")


def stokes_schur_inverse_noalloc(n, mu, rp, zp, degree=5, stream=None):
    """Context-free, allocation-free S_hat^-1 (scratch in a fixed device array)."""
    _check(load().stokes_schur_inverse_noalloc(int(n), _ptr(mu), _ptr(rp), _ptr(zp), int(degree), _stream(stream)),
           "stokes_schur_inverse_noalloc")


def stokes_autotune(ctx, what=3, stream=None):
    """Tune the level-operator block size (what & 1) and the Chebyshev degree (what & 2);
    returns (block, degree) now used by the context."""
    b, d = C.c_int(), C.c_int()
    _check(load().stokes_autotune(ctx.handle, int(what), _stream(stream), C.byref(b), C.byref(d)), "stokes_autotune")
    return b.value, d.value


def stokes_profile(enable):
    _check(load().stokes_profile(int(enable)), "stokes_profile")


def stokes_profile_read(reset=True):
    """{class name: (ms, launches)} accumulated since the last reset."""
    out = {}
    for i, name in enumerate(PROF_CLASSES):
        ms, n = C.c_double(), C.c_longlong()
        _check(load().stokes_profile_read(i, C.byref(ms), C.byref(n), 0), "stokes_profile_read")
        out[name] = (ms.value, n.value)
    if reset:
        _check(load().stokes_profile_read(0, None, None, 1), "stokes_profile_read")
    return out


def stokes_launch_count():
    return int(load().stokes_launch_count())


def stokes_probe_fma():
    """(FP32, FP64) FMA throughput of the current device in TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    _check(load().stokes_probe_fma(C.byref(a), C.byref(b)), "stokes_probe_fma")
    return a.value, b.value


def header_functions(header=None):
    """Names of the functions declared in include/stokes.h (used by the export test)."""
    import re
    header = header or os.path.join(os.path.dirname(HERE), "include", "stokes.h")
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:long\s+long|[A-Za-z_][A-Za-z0-9_]*)\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))
