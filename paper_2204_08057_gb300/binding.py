"""ctypes binding of the C ABI in ``include/sylv.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no arithmetic of its
own: tensors are checked for device, dtype, contiguity and size, then their device pointers
and the current CUDA stream are passed through.  The library must have been built
(``paper_2204_08057_gb300.build.build()``); there is no fallback when it is missing.
"""

import collections
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_void_p

import numpy as np

from . import build as _build

# successful calls of entry points that build device state, by name (handles made so far)
calls = collections.Counter()

SYLV_OK = 0
SYLV_E_INVALID = 1
SYLV_E_CUDA = 2
SYLV_E_NOMEM = 3
SYLV_E_NOT_CONVERGED = 4
SYLV_E_BREAKDOWN = 5
SYLV_E_TIMEOUT = 6
SYLV_E_UNSUPPORTED = 7
SYLV_F32 = 0
SYLV_F64 = 1
SYLV_PREC_F64 = 0
SYLV_PREC_MIXED = 1
SYLV_PRECOND_NONE = 0
SYLV_PRECOND_BLOCK_JACOBI = 1
SYLV_PRIOR_GMRF = 0
SYLV_PRIOR_IGMRF = 1
MAX_K, MAX_M, MAX_DEGREE, MAX_RHS = 8, 16, 8, 16

EXPORTED = ["sylv_opts_default", "sylv_create", "sylv_rhs", "sylv_apply", "sylv_solve",
            "sylv_solve_host", "sylv_solve_batched", "sylv_backward", "sylv_destroy",
            "sylv_strerror", "sylv_last_error", "sylv_solve_noalloc", "sylv_solve_sylvester",
            "sylv_variance", "sylv_set_params", "sylv_residual", "sylv_variance_probing"]


class sylv_problem(ctypes.Structure):
    _fields_ = [("n", c_int64), ("k", c_int32), ("m", c_int32), ("ld", c_int64),
                ("L_rowptr", c_void_p), ("L_col", c_void_p), ("L_val", c_void_p),
                ("nnz", c_int64), ("w", c_void_p), ("D", c_void_p),
                ("tau", POINTER(c_double)), ("kappa", POINTER(c_double)),
                ("nu", POINTER(c_double)), ("beta", POINTER(c_double)),
                ("A", POINTER(c_double)), ("nu0", c_double), ("prior", c_int32),
                ("reserved", c_int32)]


class sylv_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("inner_tol", c_double), ("maxit", c_int32),
                ("max_outer", c_int32), ("precision", c_int32), ("precond", c_int32),
                ("use_graph", c_int32), ("check_every", c_int32), ("profile", c_int32),
                ("use_x0", c_int32)]


class sylv_info(ctypes.Structure):
    _fields_ = [("status", c_int32), ("iterations", c_int32), ("outer", c_int32),
                ("polls", c_int32), ("relres", c_double), ("ms_total", c_double),
                ("ms_apply", c_double), ("ms_update", c_double), ("ms_residual", c_double),
                ("n_apply", c_int32), ("n_update", c_int32), ("n_residual", c_int32),
                ("launches", c_int32), ("tile", c_int32), ("slots_mult", c_int32),
                ("apply_staged", c_int32), ("update_staged", c_int32),
                ("residual_staged", c_int32), ("reserved_info", c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SylvError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {sylv_strerror(code)} ({code}) {detail}".strip())


_LIB = None


def library_path():
    return _build.LIB


def load(path=None):
    """Loads libsylv.so (once).  Raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2204_08057_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.sylv_opts_default.argtypes = [POINTER(sylv_opts)]
    lib.sylv_create.argtypes = [POINTER(c_void_p), POINTER(sylv_problem), c_void_p]
    lib.sylv_rhs.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p]
    lib.sylv_apply.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]
    lib.sylv_residual.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]
    lib.sylv_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_int, POINTER(sylv_opts),
                               POINTER(sylv_info), c_void_p]
    lib.sylv_solve_host.argtypes = [c_void_p, c_void_p, c_void_p, c_int, POINTER(sylv_opts),
                                    POINTER(sylv_info), c_void_p]
    lib.sylv_solve_batched.argtypes = [c_int, POINTER(c_void_p), POINTER(c_void_p),
                                       POINTER(c_void_p), POINTER(c_int), POINTER(sylv_opts),
                                       POINTER(sylv_info), c_void_p]
    lib.sylv_backward.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                                  POINTER(c_double), POINTER(c_double), POINTER(c_double),
                                  POINTER(sylv_opts), POINTER(sylv_info), c_void_p]
    lib.sylv_solve_noalloc.argtypes = [c_void_p, c_void_p, c_void_p, c_int,
                                       POINTER(sylv_opts), POINTER(sylv_info), c_void_p]
    lib.sylv_solve_sylvester.argtypes = [c_void_p, c_void_p, c_void_p, c_int,
                                         POINTER(sylv_opts), POINTER(sylv_info), c_void_p]
    lib.sylv_variance.argtypes = [c_void_p, c_void_p, c_int, c_void_p, POINTER(sylv_opts),
                                  POINTER(sylv_info), c_void_p]
    lib.sylv_variance_probing.argtypes = [c_void_p, c_void_p, c_int, c_void_p,
                                          POINTER(sylv_opts), POINTER(sylv_info), c_void_p]
    lib.sylv_set_params.argtypes = [c_void_p, POINTER(c_double), POINTER(c_double),
                                    POINTER(c_double), POINTER(c_double), POINTER(c_double),
                                    c_void_p]
    lib.sylv_destroy.argtypes = [c_void_p]
    lib.sylv_destroy.restype = None
    lib.sylv_strerror.argtypes = [c_int]
    lib.sylv_strerror.restype = c_char_p
    lib.sylv_last_error.argtypes = []
    lib.sylv_last_error.restype = c_char_p
    for name in EXPORTED:
        if name not in ("sylv_destroy", "sylv_strerror", "sylv_last_error"):
            getattr(lib, name).restype = c_int
    _LIB = lib
    return lib


def sylv_strerror(code):
    return load().sylv_strerror(int(code)).decode()


def sylv_last_error():
    return load().sylv_last_error().decode()


def _check(code, where, ok=(SYLV_OK,)):
    if code not in ok:
        raise SylvError(code, where, sylv_last_error())
    return code


# ---------------------------------------------------------------------------------------------
# tensor marshalling
# ---------------------------------------------------------------------------------------------
def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, numel_min, what):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() < numel_min:
        raise ValueError(f"{what} has {t.numel()} elements, needs {numel_min}")
    return c_void_p(t.data_ptr())


def _host_doubles(x, count, what):
    if x is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    if a.size != count:
        raise ValueError(f"{what} needs {count} values, got {a.size}")
    return a, a.ctypes.data_as(POINTER(c_double))


def sylv_opts_default():
    o = sylv_opts()
    _check(load().sylv_opts_default(ctypes.byref(o)), "sylv_opts_default")
    return o


def make_opts(**kw):
    o = sylv_opts_default()
    for key, v in kw.items():
        if not hasattr(o, key):
            raise KeyError(key)
        setattr(o, key, v)
    return o


def sylv_create(*, n, k, m, ld, L_rowptr, L_col, L_val, D, tau, kappa, nu=None, beta=None,
                A=None, w=None, nu0=0.0, prior=0, stream=None):
    """Returns an opaque handle (int).  Device tensors: L_rowptr (int32, n+1), L_col (int32),
    L_val (float64), D (float64, m x ld), w (float64, n) or None.  Host: tau, kappa (k),
    nu (m), beta (k), A (m x k) or None.  prior: SYLV_PRIOR_GMRF or SYLV_PRIOR_IGMRF."""
    import torch
    nnz = int(L_col.numel())
    p = sylv_problem()
    p.n, p.k, p.m, p.ld, p.nnz, p.nu0 = int(n), int(k), int(m), int(ld), nnz, float(nu0)
    p.prior = int(prior)
    p.L_rowptr = _dev_ptr(L_rowptr, torch.int32, n + 1, "L_rowptr")
    p.L_col = _dev_ptr(L_col, torch.int32, nnz, "L_col")
    p.L_val = _dev_ptr(L_val, torch.float64, nnz, "L_val")
    p.D = _dev_ptr(D, torch.float64, (m - 1) * ld + n, "D")
    p.w = _dev_ptr(w, torch.float64, n, "w")
    keep = []
    for name, val, cnt in (("tau", tau, k), ("kappa", kappa, k), ("nu", nu, m),
                           ("beta", beta, k), ("A", A, m * k)):
        arr, ptr = _host_doubles(val, cnt, name)
        keep.append(arr)
        setattr(p, name, ptr)
    h = c_void_p()
    _check(load().sylv_create(ctypes.byref(h), ctypes.byref(p), _stream(stream)), "sylv_create")
    calls["sylv_create"] += 1
    return h.value


def sylv_destroy(h):
    if h:
        load().sylv_destroy(c_void_p(h))


def sylv_rhs(h, Yobs, B, nrhs, *, k, m, ld, n, stream=None):
    import torch
    _check(load().sylv_rhs(c_void_p(h),
                           _dev_ptr(Yobs, torch.float64, ((nrhs - 1) * m + m - 1) * ld + n,
                                    "Yobs"),
                           _dev_ptr(B, torch.float64, ((nrhs - 1) * k + k - 1) * ld + n, "B"),
                           int(nrhs), _stream(stream)), "sylv_rhs")


def sylv_apply(h, X, Y, nrhs, *, k, ld, n, stream=None):
    import torch
    if X.dtype != Y.dtype:
        raise TypeError("X and Y must have one dtype")
    dt = {torch.float32: SYLV_F32, torch.float64: SYLV_F64}.get(X.dtype)
    if dt is None:
        raise TypeError("X must be float32 or float64")
    need = ((nrhs - 1) * k + k - 1) * ld + n
    _check(load().sylv_apply(c_void_p(h), _dev_ptr(X, X.dtype, need, "X"),
                             _dev_ptr(Y, Y.dtype, need, "Y"), int(nrhs), dt, _stream(stream)),
           "sylv_apply")


def sylv_residual(h, B, X, R, nrhs, *, k, ld, n, stream=None):
    """R = B - G X (FP64 device tensors nrhs x k x ld)."""
    import torch
    need = ((nrhs - 1) * k + k - 1) * ld + n
    _check(load().sylv_residual(c_void_p(h), _dev_ptr(B, torch.float64, need, "B"),
                                _dev_ptr(X, torch.float64, need, "X"), int(nrhs),
                                _dev_ptr(R, torch.float64, need, "R"), _stream(stream)),
           "sylv_residual")


def sylv_solve(h, B, X, nrhs, opts=None, *, k, ld, n, stream=None, allow=()):
    """Returns (status, sylv_info).  Raises on statuses outside SYLV_OK and ``allow``."""
    import torch
    need = ((nrhs - 1) * k + k - 1) * ld + n
    info = sylv_info()
    code = load().sylv_solve(c_void_p(h), _dev_ptr(B, torch.float64, need, "B"),
                             _dev_ptr(X, torch.float64, need, "X"), int(nrhs),
                             ctypes.byref(opts) if opts is not None else None,
                             ctypes.byref(info), _stream(stream))
    _check(code, "sylv_solve", ok=(SYLV_OK,) + tuple(allow))
    return code, info


def _host_ptr(t, dtype, numel_min, what):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{what} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() < numel_min:
        raise ValueError(f"{what} has {t.numel()} elements, needs {numel_min}")
    return c_void_p(t.data_ptr())


def sylv_solve_host(h, Yobs, X, nrhs, opts=None, *, k, m, ld, n, stream=None, allow=()):
    """Yobs (nrhs x m x ld) and X (nrhs x k x ld): host float64 tensors (page-locked for
    overlapped copies).  Returns (status, sylv_info); X holds the solution."""
    import torch
    info = sylv_info()
    code = load().sylv_solve_host(
        c_void_p(h), _host_ptr(Yobs, torch.float64, ((nrhs - 1) * m + m - 1) * ld + n, "Yobs"),
        _host_ptr(X, torch.float64, ((nrhs - 1) * k + k - 1) * ld + n, "X"), int(nrhs),
        ctypes.byref(opts) if opts is not None else None, ctypes.byref(info), _stream(stream))
    _check(code, "sylv_solve_host", ok=(SYLV_OK,) + tuple(allow))
    return code, info


def sylv_solve_batched(handles, Bs, Xs, nrhs, opts=None, *, shapes, stream=None, allow=()):
    """handles, Bs, Xs, nrhs: lists; shapes: list of (k, ld, n).  Returns (status, infos)."""
    import torch
    ns = len(handles)
    hs = (c_void_p * ns)(*[c_void_p(h) for h in handles])
    bp = (c_void_p * ns)()
    xp = (c_void_p * ns)()
    for t in range(ns):
        k, ld, n = shapes[t]
        need = ((nrhs[t] - 1) * k + k - 1) * ld + n
        bp[t] = _dev_ptr(Bs[t], torch.float64, need, f"B[{t}]")
        xp[t] = _dev_ptr(Xs[t], torch.float64, need, f"X[{t}]")
    rr = (c_int * ns)(*[int(r) for r in nrhs])
    infos = (sylv_info * ns)()
    code = load().sylv_solve_batched(ns, hs, bp, xp, rr,
                                     ctypes.byref(opts) if opts is not None else None, infos,
                                     _stream(stream))
    _check(code, "sylv_solve_batched", ok=(SYLV_OK,) + tuple(allow))
    return code, list(infos)


def sylv_backward(h, Xhat, dLdX, Yobs, nrhs, lam=None, opts=None, *, k, m, ld, n,
                  want=("tau", "kappa", "beta"), stream=None):
    """Returns (g_tau, g_kappa, g_beta, sylv_info); entries not in ``want`` are None."""
    import torch
    need = ((nrhs - 1) * k + k - 1) * ld + n
    g = {name: (np.zeros(k) if name in want else None) for name in ("tau", "kappa", "beta")}
    ptr = {name: (v.ctypes.data_as(POINTER(c_double)) if v is not None else None)
           for name, v in g.items()}
    info = sylv_info()
    code = load().sylv_backward(
        c_void_p(h), _dev_ptr(Xhat, torch.float64, need, "Xhat"),
        _dev_ptr(dLdX, torch.float64, need, "dLdX"),
        _dev_ptr(Yobs, torch.float64, ((nrhs - 1) * m + m - 1) * ld + n, "Yobs")
        if Yobs is not None else None,
        int(nrhs), _dev_ptr(lam, torch.float64, need, "lambda") if lam is not None else None,
        ptr["tau"], ptr["kappa"], ptr["beta"],
        ctypes.byref(opts) if opts is not None else None, ctypes.byref(info), _stream(stream))
    _check(code, "sylv_backward")
    return g["tau"], g["kappa"], g["beta"], info


def sylv_solve_noalloc(h, B, X, nrhs, opts=None, *, k, ld, n, stream=None, allow=()):
    """Allocation-free solve (see sylv.h): same arguments and result as ``sylv_solve``; the
    workspace lives in the library's fixed device scratch array.  Returns (status, info)."""
    import torch
    need = ((nrhs - 1) * k + k - 1) * ld + n
    info = sylv_info()
    code = load().sylv_solve_noalloc(c_void_p(h), _dev_ptr(B, torch.float64, need, "B"),
                                     _dev_ptr(X, torch.float64, need, "X"), int(nrhs),
                                     ctypes.byref(opts) if opts is not None else None,
                                     ctypes.byref(info), _stream(stream))
    _check(code, "sylv_solve_noalloc", ok=(SYLV_OK,) + tuple(allow))
    return code, info


def sylv_solve_sylvester(h, B, X, nrhs, opts=None, *, k, ld, n, stream=None, allow=()):
    """Block-Lanczos solve of the Sylvester form (see sylv.h); same arguments and result as
    ``sylv_solve``.  Returns (status, info)."""
    import torch
    need = ((nrhs - 1) * k + k - 1) * ld + n
    info = sylv_info()
    code = load().sylv_solve_sylvester(c_void_p(h), _dev_ptr(B, torch.float64, need, "B"),
                                       _dev_ptr(X, torch.float64, need, "X"), int(nrhs),
                                       ctypes.byref(opts) if opts is not None else None,
                                       ctypes.byref(info), _stream(stream))
    _check(code, "sylv_solve_sylvester", ok=(SYLV_OK,) + tuple(allow))
    return code, info


def sylv_variance(h, Z, nprobe, var, opts=None, *, k, ld, n, stream=None, allow=()):
    """Probe estimate of the posterior variances (see sylv.h).  Returns (status, info)."""
    import torch
    need = ((nprobe - 1) * k + k - 1) * ld + n
    info = sylv_info()
    code = load().sylv_variance(c_void_p(h), _dev_ptr(Z, torch.float64, need, "Z"), int(nprobe),
                                _dev_ptr(var, torch.float64, (k - 1) * ld + n, "var"),
                                ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(info), _stream(stream))
    _check(code, "sylv_variance", ok=(SYLV_OK,) + tuple(allow))
    return code, info



def sylv_variance_probing(h, colour, ncolours, var, opts=None, *, k, ld, n, stream=None,
                          allow=()):
    """Posterior variances from the probes of a pixel colouring (see sylv.h).  colour: int32
    device tensor (n).  Returns (status, info)."""
    import torch
    info = sylv_info()
    code = load().sylv_variance_probing(c_void_p(h), _dev_ptr(colour, torch.int32, n, "colour"),
                                        int(ncolours),
                                        _dev_ptr(var, torch.float64, (k - 1) * ld + n, "var"),
                                        ctypes.byref(opts) if opts is not None else None,
                                        ctypes.byref(info), _stream(stream))
    _check(code, "sylv_variance_probing", ok=(SYLV_OK,) + tuple(allow))
    return code, info

def sylv_set_params(h, *, k, m, tau, kappa, nu=None, beta=None, A=None, stream=None):
    """New tau, kappa and mixing for an existing handle (see sylv.h)."""
    keep = []
    ptrs = []
    for name, val, cnt in (("tau", tau, k), ("kappa", kappa, k), ("nu", nu, m),
                           ("beta", beta, k), ("A", A, m * k)):
        arr, ptr = _host_doubles(val, cnt, name)
        keep.append(arr)
        ptrs.append(ptr)
    _check(load().sylv_set_params(c_void_p(h), *ptrs, _stream(stream)), "sylv_set_params")
