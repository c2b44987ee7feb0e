"""Thin ctypes binding of the C-ABI in include/stokes.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards
device pointers taken from torch tensors; all arithmetic runs in the CUDA
library.  The library must have been built (paper_1406_6573_gb300.build or
__graft_entry__.build()); importing this module without it raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libstokes_gb300.so")

STOKES_OK = 0
STOKES_WAIT_POLLS_DEFAULT = 4194304
STOKES_F64 = 0
STOKES_F32 = 1
STOKES_PRESSURE_P = 0
STOKES_PRESSURE_Q = 1
STOKES_BASE_NOSLIP = 0
STOKES_BASE_SLIP = 1

ERRORS = {-1: "E_INVAL", -2: "E_MESH", -3: "E_NOMEM", -4: "E_CUDA", -5: "E_NONFINITE", -6: "E_NOCONV"}


class StokesError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class stokes_field(C.Structure):
    _fields_ = [("mean", C.c_double), ("n_modes", C.c_int),
                ("amp", C.POINTER(C.c_double)), ("kx", C.POINTER(C.c_double)),
                ("ky", C.POINTER(C.c_double)), ("phase", C.POINTER(C.c_double))]


class stokes_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("k", C.c_int),
                ("pressure_space", C.c_int), ("periodic_xy", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double),
                ("bed", stokes_field), ("surface", stokes_field),
                ("refine", C.POINTER(C.c_uint8)), ("basal_bc", C.c_int), ("device", C.c_int),
                ("bed_nodes", C.POINTER(C.c_double)), ("surface_nodes", C.POINTER(C.c_double))]


class stokes_params(C.Structure):
    _fields_ = [("n", C.c_double), ("A", C.c_double), ("C0", C.c_double),
                ("gamma", C.c_double), ("delta", C.c_double), ("body", C.c_double * 3),
                ("robin", C.c_int), ("logbeta", C.c_void_p), ("constraint_scale", C.c_double),
                ("linearization", C.c_int), ("sliding_m", C.c_double), ("sliding_eps", C.c_double)]


STOKES_LIN_NEWTON = 0
STOKES_LIN_PICARD = 1


class stokes_sizes(C.Structure):
    _fields_ = [("E", C.c_int64), ("Nv", C.c_int64), ("Np", C.c_int64), ("Nb", C.c_int64),
                ("k", C.c_int32), ("npr", C.c_int32), ("n_hanging_elems", C.c_int64)]


class stokes_kernel_time(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double)]


class stokes_profile(C.Structure):
    _fields_ = [(name, stokes_kernel_time) for name in
                ("clear", "element", "face", "constraint", "precond", "orthog", "vector", "setup", "transfer")]


class stokes_solver_opts(C.Structure):
    _fields_ = [("inner_prec", C.c_int), ("restart", C.c_int), ("max_krylov", C.c_int),
                ("max_newton", C.c_int), ("rtol", C.c_double), ("eta_max", C.c_double),
                ("velocity_mg", C.c_int)]


class stokes_solve_report(C.Structure):
    _fields_ = [("converged", C.c_int), ("newton_its", C.c_int), ("krylov_its", C.c_int),
                ("line_search_cuts", C.c_int), ("res0", C.c_double), ("res_final", C.c_double),
                ("seconds", C.c_double), ("constraint_scale", C.c_double), ("history", C.c_double * 64),
                ("krylov_per_newton", C.c_int * 64), ("line_search_failed", C.c_int), ("mg_levels", C.c_int)]

    def as_dict(self):
        n = min(self.newton_its + 1, 64)
        return {"converged": bool(self.converged), "newton_its": self.newton_its,
                "krylov_its": self.krylov_its, "line_search_cuts": self.line_search_cuts,
                "res0": self.res0, "res_final": self.res_final, "seconds": self.seconds,
                "constraint_scale": self.constraint_scale,
                "history": list(self.history[:n]),
                "krylov_per_newton": list(self.krylov_per_newton[:max(n - 1, 0)]),
                "line_search_failed": bool(self.line_search_failed), "mg_levels": self.mg_levels}


# every symbol declared in include/stokes.h, with its ctypes signature
_SIGS = {
    "stokes_mesh_create": (C.c_int, [C.POINTER(stokes_mesh_desc), C.POINTER(C.c_void_p)]),
    "stokes_mesh_destroy": (C.c_int, [C.c_void_p]),
    "stokes_mesh_sizes": (C.c_int, [C.c_void_p, C.POINTER(stokes_sizes)]),
    "stokes_mesh_node_coords": (C.c_int, [C.c_void_p, C.c_void_p]),
    "stokes_mesh_basal_nodes": (C.c_int, [C.c_void_p, C.c_void_p]),
    "stokes_residual": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "stokes_jacobian_apply": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_int, C.c_void_p]),
    "stokes_jacobian_apply_transpose": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p,
                                                  C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "stokes_param_grad": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "stokes_param_grad_A_fixed_order": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p,
                                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "stokes_state_apply_pressure_block": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "stokes_state_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "stokes_state_destroy": (C.c_int, [C.c_void_p]),
    "stokes_linearize": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p, C.c_void_p]),
    "stokes_state_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "stokes_state_apply_transpose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "stokes_mesh_status": (C.c_int, [C.c_void_p]),
    "stokes_solver_create": (C.c_int, [C.c_void_p, C.POINTER(stokes_solver_opts), C.POINTER(C.c_void_p)]),
    "stokes_solver_destroy": (C.c_int, [C.c_void_p]),
    "stokes_newton_solve": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p,
                                      C.POINTER(stokes_solve_report), C.c_void_p]),
    "stokes_linear_solve": (C.c_int, [C.c_void_p, C.POINTER(stokes_params), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_int, C.c_double, C.POINTER(stokes_solve_report),
                                      C.c_void_p]),
    "stokes_profile_begin": (C.c_int, [C.c_void_p]),
    "stokes_profile_end": (C.c_int, [C.c_void_p, C.POINTER(stokes_profile)]),
    "stokes_last_error": (C.c_char_p, []),
    "stokes_debug_wait_limit": (C.c_int, [C.c_void_p, C.c_uint32]),
    "stokes_debug_fail_alloc_after": (C.c_int64, [C.c_int64]),
    "stokes_debug_forest_prolongation": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64),
                                                   C.POINTER(C.c_double)]),
    "stokes_debug_mg_transfer": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                                           C.c_int64]),
}

_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != STOKES_OK:
        raise StokesError(rc, lib().stokes_last_error().decode())


def _ptr(t):
    """Device (or host) pointer of a contiguous torch tensor / numpy array; None -> NULL."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------- raw entry points
def stokes_mesh_create(desc):
    h = C.c_void_p()
    _check(lib().stokes_mesh_create(C.byref(desc), C.byref(h)))
    return h


def stokes_mesh_destroy(h):
    _check(lib().stokes_mesh_destroy(h))


def stokes_mesh_sizes(h):
    s = stokes_sizes()
    _check(lib().stokes_mesh_sizes(h, C.byref(s)))
    return s


def stokes_mesh_node_coords(h, out):
    _check(lib().stokes_mesh_node_coords(h, _ptr(out)))


def stokes_mesh_basal_nodes(h, out):
    _check(lib().stokes_mesh_basal_nodes(h, _ptr(out)))


def stokes_debug_forest_prolongation(forest, base):
    """(entries, largest |row sum - 1|) of the forest multigrid's prolongation
    from base to forest (host-only meshes); raises on a mismatch."""
    nnz = C.c_int64(0)
    err = C.c_double(0.0)
    _check(lib().stokes_debug_forest_prolongation(forest, base, C.byref(nnz), C.byref(err)))
    return nnz.value, err.value


def stokes_debug_mg_transfer(nf, k, periodic, which):
    """Dense 1-D multigrid transfer table (0 = P, 1 = R, 2 = J) as a numpy array."""
    import numpy as np
    NXf = k * nf + (0 if periodic else 1)
    NXc = k * (nf // 2) + (0 if periodic else 1)
    shape = (NXf, NXc) if which == 0 else (NXc, NXf)
    out = np.zeros(shape, dtype=np.float64)
    _check(lib().stokes_debug_mg_transfer(nf, k, int(periodic), which, out.ctypes.data, shape[0], shape[1]))
    return out


def stokes_debug_wait_limit(h, polls):
    _check(lib().stokes_debug_wait_limit(h, polls))


def stokes_debug_fail_alloc_after(n):
    return int(lib().stokes_debug_fail_alloc_after(n))


def stokes_residual(h, params, up, r, prec, stream=None):
    _check(lib().stokes_residual(h, C.byref(params), _ptr(up), _ptr(r), prec, _stream(stream)))


def stokes_jacobian_apply(h, params, up_lin, x, y, prec, stream=None):
    _check(lib().stokes_jacobian_apply(h, C.byref(params), _ptr(up_lin), _ptr(x), _ptr(y), prec,
                                       _stream(stream)))


def stokes_jacobian_apply_transpose(h, params, up_lin, x, y, prec, stream=None):
    _check(lib().stokes_jacobian_apply_transpose(h, C.byref(params), _ptr(up_lin), _ptr(x), _ptr(y),
                                                 prec, _stream(stream)))


def stokes_param_grad(h, params, up, lam, g_logbeta, g_A, stream=None):
    _check(lib().stokes_param_grad(h, C.byref(params), _ptr(up), _ptr(lam), _ptr(g_logbeta), _ptr(g_A),
                                   _stream(stream)))


def stokes_param_grad_A_fixed_order(h, params, up, lam, g_A, stream=None):
    """g_A[0] = lambda^T d r_c / d A summed in a fixed order, using the
    library's static device scratch (no allocation; calls on one device must
    not overlap)."""
    _check(lib().stokes_param_grad_A_fixed_order(h, C.byref(params), _ptr(up), _ptr(lam), _ptr(g_A),
                                                 _stream(stream)))


STOKES_GRAD_A_MAX_PARTIALS = 131072


def stokes_state_create(h, prec):
    s = C.c_void_p()
    _check(lib().stokes_state_create(h, prec, C.byref(s)))
    return s


def stokes_state_destroy(s):
    _check(lib().stokes_state_destroy(s))


def stokes_linearize(s, params, up_lin, stream=None):
    _check(lib().stokes_linearize(s, C.byref(params), _ptr(up_lin), _stream(stream)))


def stokes_state_apply(s, x, y, stream=None):
    _check(lib().stokes_state_apply(s, _ptr(x), _ptr(y), _stream(stream)))


def stokes_state_apply_transpose(s, x, y, stream=None):
    _check(lib().stokes_state_apply_transpose(s, _ptr(x), _ptr(y), _stream(stream)))


def stokes_state_apply_pressure_block(s, x, y, stream=None):
    _check(lib().stokes_state_apply_pressure_block(s, _ptr(x), _ptr(y), _stream(stream)))


def stokes_profile_begin(h):
    _check(lib().stokes_profile_begin(h))


def stokes_profile_end(h):
    p = stokes_profile()
    _check(lib().stokes_profile_end(h, C.byref(p)))
    return {name: (getattr(p, name).launches, getattr(p, name).ms) for name, _ in stokes_profile._fields_}


def stokes_mesh_status(h):
    _check(lib().stokes_mesh_status(h))


def stokes_solver_create(h, opts=None):
    s = C.c_void_p()
    _check(lib().stokes_solver_create(h, C.byref(opts) if opts is not None else None, C.byref(s)))
    return s


def stokes_solver_destroy(s):
    _check(lib().stokes_solver_destroy(s))


def stokes_newton_solve(s, params, up, stream=None, check=True):
    """Returns (status code, report dict); raises on errors other than E_NOCONV when check."""
    rep = stokes_solve_report()
    rc = lib().stokes_newton_solve(s, C.byref(params), _ptr(up), C.byref(rep), _stream(stream))
    if check and rc not in (STOKES_OK, -6):
        _check(rc)
    return rc, rep.as_dict()


def stokes_linear_solve(s, params, up_lin, b, x, transpose=False, rtol=1e-8, stream=None, check=True):
    rep = stokes_solve_report()
    rc = lib().stokes_linear_solve(s, C.byref(params), _ptr(up_lin), _ptr(b), _ptr(x), int(transpose),
                                   float(rtol), C.byref(rep), _stream(stream))
    if check and rc not in (STOKES_OK, -6):
        _check(rc)
    return rc, rep.as_dict()
