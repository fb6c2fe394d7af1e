"""Python binding of the GB300 FEAST library (libfeast_gb300.so).

Argument marshalling only: every step of the eigensolver runs in the CUDA
kernels behind the C-ABI declared in include/feast.h.  Functions keep the C
names.  Buffers may be torch tensors (CUDA or CPU) or numpy arrays; CUDA
tensors are passed as device pointers, everything else as host pointers (the
library copies host data through its own device workspace).

Importing this package loads the shared library and raises ImportError when it
has not been built (``python -m paper_0901_2665_gb300.build``); there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfeast_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_0901_2665_gb300.build`")

_lib = ctypes.CDLL(LIB_PATH)

FEAST_OK = 0
FEAST_ERR_ARG = 1
FEAST_ERR_BQ_NOT_SPD = 2
FEAST_ERR_NO_CONVERGENCE = 3
FEAST_ERR_M0_TOO_SMALL = 4
FEAST_ERR_PIVOT = 5
FEAST_ERR_OOM = 6
FEAST_ERR_CUDA = 7
FEAST_ERR_TIMEOUT = 8
FEAST_ERR_JACOBI = 9
FEAST_ERR_NONFINITE = 10
STATUS_NAMES = {v: k for k, v in globals().items() if k.startswith("FEAST_ERR_") or k == "FEAST_OK"}

FEAST_PREC_FP64 = 0
FEAST_PREC_MIXED = 1
FEAST_INNER_DIRECT = 0
FEAST_INNER_COCG = 1

EXPORTED = [
    "feast_default_options", "feast_init", "feast_destroy", "feast_last_error", "feast_get_info",
    "feast_solve", "feast_solve_hermitian", "feast_contour", "feast_stencil_apply", "feast_node_solve", "feast_quadrature",
    "feast_reduced_eig", "feast_rayleigh_ritz", "feast_residuals", "feast_reduced_eig_noalloc",
    "feast_selftest_wait_timeout",
    "feast_solve_batched", "feast_mlp_create", "feast_mlp_destroy", "feast_mlp_set_layer", "feast_mlp_get_layer",
    "feast_mlp_forward", "feast_mlp_train_step", "feast_sine_expand", "feast_sine_project", "feast_predict_Y",
]


class feast_operator(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("A27", ctypes.c_void_p), ("B27", ctypes.c_void_p)]


class feast_options(ctypes.Structure):
    _fields_ = [("max_loops", ctypes.c_int), ("precision", ctypes.c_int), ("ir_tol", ctypes.c_double),
                ("ir_max", ctypes.c_int), ("seed", ctypes.c_uint64), ("profile", ctypes.c_int),
                ("ir_early", ctypes.c_int), ("inner_solver", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("inner_max_iter", ctypes.c_int)]


KERNEL_CLASS_SLOTS = 12   # FEAST_KERNEL_CLASSES


class feast_info(ctypes.Structure):
    _fields_ = [("loops", ctypes.c_int), ("m_found", ctypes.c_int),
                ("trace", ctypes.c_double * 64), ("rel_change", ctypes.c_double * 64),
                ("resid_max", ctypes.c_double), ("resid_paper_max", ctypes.c_double),
                ("t_factor_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("t_rr_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double),
                ("ir_steps_max", ctypes.c_int), ("ir_resid_max", ctypes.c_double),
                ("factor_flops", ctypes.c_longlong), ("gpu_launches", ctypes.c_longlong),
                ("kernel_ms", ctypes.c_double * KERNEL_CLASS_SLOTS),
                ("kernel_launches", ctypes.c_longlong * KERNEL_CLASS_SLOTS),
                ("kernel_flops", ctypes.c_double * KERNEL_CLASS_SLOTS),
                ("sweep_graphs", ctypes.c_longlong), ("inner_iters_max", ctypes.c_int),
                ("inner_rel_max", ctypes.c_double), ("loop_graphs", ctypes.c_int)]


KERNEL_CLASSES = ["sweep_gemm", "solve_gemm", "panel_inverse", "panel_product", "schur", "solve_coupling",
                  "fp64_residual", "fp64_path", "ff_residual", "sweep_narrow"]


_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_lib.feast_default_options.argtypes = [ctypes.POINTER(feast_options)]
_lib.feast_default_options.restype = None
_lib.feast_init.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(feast_options), _vp]
_lib.feast_destroy.argtypes = [_vp]
_lib.feast_last_error.argtypes = [_vp]
_lib.feast_last_error.restype = ctypes.c_char_p
_lib.feast_get_info.argtypes = [_vp, ctypes.POINTER(feast_info)]
_lib.feast_solve.argtypes = [_vp, ctypes.POINTER(feast_operator), _d, _d, _i, _i, _d, _vp, _vp, _vp, _vp,
                             ctypes.POINTER(_i), ctypes.POINTER(_i)]
_lib.feast_solve_hermitian.argtypes = [_vp, ctypes.POINTER(feast_operator), _d, _d, _i, _i, _d, _vp, _vp, _vp, _vp,
                                       ctypes.POINTER(_i), ctypes.POINTER(_i)]
_lib.feast_contour.argtypes = [_d, _d, _i, _vp, _vp, _vp, _vp, _vp]
_lib.feast_stencil_apply.argtypes = [_vp, _i, _i, _i, _vp, _vp, _vp, _i]
_lib.feast_selftest_wait_timeout.argtypes = [_vp, ctypes.c_longlong]
_lib.feast_node_solve.argtypes = [_vp, ctypes.POINTER(feast_operator), _d, _d, _vp, _vp, _i, _i]
_lib.feast_quadrature.argtypes = [_vp, ctypes.POINTER(feast_operator), _d, _d, _i, _vp, _vp, _i, _i]
_lib.feast_reduced_eig.argtypes = [_vp, _vp, _vp, _i, _vp, _vp]
_lib.feast_rayleigh_ritz.argtypes = [_vp, ctypes.POINTER(feast_operator), _vp, _i, _vp, _vp, _vp, _vp]
_lib.feast_residuals.argtypes = [_vp, ctypes.POINTER(feast_operator), _vp, _vp, _i, _vp, _vp]
_lib.feast_reduced_eig_noalloc.argtypes = [_vp, _vp, _i, _vp, _vp, _vp]
_lib.feast_mlp_create.argtypes = [ctypes.POINTER(_vp), _i, _i, _i, _i, _vp]
_lib.feast_mlp_destroy.argtypes = [_vp]
_lib.feast_mlp_set_layer.argtypes = [_vp, _i, _vp, _vp]
_lib.feast_mlp_get_layer.argtypes = [_vp, _i, _vp, _vp, _vp, _vp]
_lib.feast_mlp_forward.argtypes = [_vp, _vp, _i, _vp]
_lib.feast_mlp_train_step.argtypes = [_vp, _vp, _vp, _vp, _i, ctypes.c_float, ctypes.POINTER(_d)]
_lib.feast_sine_expand.argtypes = [_vp, _i, _i, _i, _i, _i, _i, _vp, _vp]
_lib.feast_sine_project.argtypes = [_vp, _i, _i, _i, _i, _i, _i, _vp, _vp]
_lib.feast_predict_Y.argtypes = [_vp, _vp, _i, _i, _i, _i, _i, _i, _vp]
_lib.feast_solve_batched.argtypes = [_vp, _i, ctypes.POINTER(feast_operator), _vp, _vp, _vp, _i, _d, _vp, _vp, _vp,
                                     _vp, _vp, _vp, _vp, _i]
for _f in EXPORTED:
    if _f not in ("feast_default_options", "feast_last_error"):
        getattr(_lib, _f).restype = ctypes.c_int


class FeastError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(buf):
    """Address of a torch tensor / numpy array (None -> NULL)."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not (buf.flags["C_CONTIGUOUS"] or buf.flags["F_CONTIGUOUS"]):
            raise ValueError("array must be contiguous")
        return buf.ctypes.data
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch is optional for the binding
        pass
    return None


def default_options() -> feast_options:
    o = feast_options()
    _lib.feast_default_options(ctypes.byref(o))
    return o


def make_operator(nx, ny, nz, A27, B27):
    """feast_operator over two [27][N] float64 buffers (kept alive by the caller)."""
    return feast_operator(nx, ny, nz, _ptr(A27), _ptr(B27))


def feast_contour(lmin: float, lmax: float, Ne: int):
    arrs = [np.zeros(Ne) for _ in range(5)]
    st = _lib.feast_contour(lmin, lmax, Ne, *[a.ctypes.data for a in arrs])
    if st != FEAST_OK:
        raise FeastError(st, "feast_contour")
    x, w, theta, zr, zi = arrs
    return x, w, theta, zr + 1j * zi


@dataclasses.dataclass
class SolveResult:
    status: int
    m_found: int
    loops: int
    info: feast_info


class Handle:
    """Owns one feast_handle (feast_init / feast_destroy)."""

    def __init__(self, precision: int = FEAST_PREC_FP64, max_loops: int = 20, ir_tol: float = 1e-12,
                 ir_max: int = 30, seed: int = 1000, stream=None, profile: bool = False, ir_early: bool = True,
                 inner_solver: int = FEAST_INNER_DIRECT, inner_tol: float = 1e-3, inner_max_iter: int = 5000):
        opt = default_options()
        opt.precision, opt.max_loops, opt.ir_tol, opt.ir_max, opt.seed = precision, max_loops, ir_tol, ir_max, seed
        opt.profile = 1 if profile else 0
        opt.ir_early = 1 if ir_early else 0
        opt.inner_solver, opt.inner_tol, opt.inner_max_iter = inner_solver, inner_tol, inner_max_iter
        self._h = _vp()
        st = _lib.feast_init(ctypes.byref(self._h), ctypes.byref(opt), stream if stream is not None else _current_stream())
        if st != FEAST_OK:
            raise FeastError(st, "feast_init failed")

    def close(self):
        if self._h:
            _lib.feast_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return _lib.feast_last_error(self._h).decode()

    def _check(self, st, what, allow=()):
        if st != FEAST_OK and st not in allow:
            raise FeastError(st, f"{what}: {self.last_error()}")
        return st

    def info(self) -> feast_info:
        inf = feast_info()
        self._check(_lib.feast_get_info(self._h, ctypes.byref(inf)), "feast_get_info")
        return inf

    def feast_solve(self, op: feast_operator, lmin, lmax, M0, Ne, tol, Y0, lam, X, resid=None,
                    allow=(FEAST_ERR_NO_CONVERGENCE, FEAST_ERR_M0_TOO_SMALL)) -> SolveResult:
        m, loops = ctypes.c_int(0), ctypes.c_int(0)
        st = _lib.feast_solve(self._h, ctypes.byref(op), float(lmin), float(lmax), int(M0), int(Ne), float(tol),
                              _ptr(Y0), _ptr(lam), _ptr(X), _ptr(resid), ctypes.byref(m), ctypes.byref(loops))
        self._check(st, "feast_solve", allow)
        return SolveResult(st, m.value, loops.value, self.info())

    def feast_solve_hermitian(self, op: feast_operator, lmin, lmax, M0, Ne, tol, Y0, lam, X, resid=None,
                              allow=(FEAST_ERR_NO_CONVERGENCE, FEAST_ERR_M0_TOO_SMALL)) -> SolveResult:
        """op: feast_operator over complex [27][N] A27 and B27 (device);
        Y0 (or None) and X: complex N x M0 device buffers."""
        m, loops = ctypes.c_int(0), ctypes.c_int(0)
        st = _lib.feast_solve_hermitian(self._h, ctypes.byref(op), float(lmin), float(lmax), int(M0), int(Ne),
                                        float(tol), _ptr(Y0), _ptr(lam), _ptr(X), _ptr(resid), ctypes.byref(m),
                                        ctypes.byref(loops))
        self._check(st, "feast_solve_hermitian", allow)
        return SolveResult(st, m.value, loops.value, self.info())

    def feast_solve_batched(self, ops, lmin, lmax, M0, Ne, tol, Y0, lam, X, resid=None, workers=0, raise_on_error=True):
        """ops: list of feast_operator; lmin/lmax/M0: per-instance sequences;
        Y0, lam, X, resid: per-instance buffers (Y0 / resid may be None).
        Returns (status, m_found, loops, statuses) as numpy arrays."""
        cnt = len(ops)
        op_arr = (feast_operator * cnt)(*ops)
        lo = np.ascontiguousarray(lmin, dtype=np.float64)
        hi = np.ascontiguousarray(lmax, dtype=np.float64)
        m0 = np.ascontiguousarray(M0, dtype=np.int32)
        P = ctypes.c_void_p * cnt
        y_arr = P(*[_ptr(y) for y in Y0]) if Y0 is not None else None
        r_arr = P(*[_ptr(r) for r in resid]) if resid is not None else None
        mf = np.zeros(cnt, dtype=np.int32)
        lp = np.zeros(cnt, dtype=np.int32)
        sts = np.zeros(cnt, dtype=np.int32)
        st = _lib.feast_solve_batched(self._h, cnt, op_arr, lo.ctypes.data, hi.ctypes.data, m0.ctypes.data, int(Ne),
                                      float(tol), y_arr, P(*[_ptr(x) for x in lam]), P(*[_ptr(x) for x in X]), r_arr,
                                      mf.ctypes.data, lp.ctypes.data, sts.ctypes.data, int(workers))
        if raise_on_error:
            self._check(st, "feast_solve_batched")
        return st, mf, lp, sts

    def feast_selftest_wait_timeout(self, polls: int):
        """Runs the give-up path of the bounded device waits (a wait on an
        mbarrier nothing completes, limited to `polls` polls); raises
        FeastError(FEAST_ERR_TIMEOUT) as designed."""
        self._check(_lib.feast_selftest_wait_timeout(self._h, int(polls)), "feast_selftest_wait_timeout")

    def feast_stencil_apply(self, nx, ny, nz, C27, X, Y, k):
        self._check(_lib.feast_stencil_apply(self._h, nx, ny, nz, _ptr(C27), _ptr(X), _ptr(Y), int(k)),
                    "feast_stencil_apply")

    def feast_node_solve(self, op, Z: complex, RHS, Qe, k, precision=FEAST_PREC_FP64):
        self._check(_lib.feast_node_solve(self._h, ctypes.byref(op), Z.real, Z.imag, _ptr(RHS), _ptr(Qe), int(k),
                                          int(precision)), "feast_node_solve")
        return self.info()

    def feast_quadrature(self, op, lmin, lmax, Ne, RHS, Q, k, precision=FEAST_PREC_FP64):
        self._check(_lib.feast_quadrature(self._h, ctypes.byref(op), float(lmin), float(lmax), int(Ne), _ptr(RHS),
                                          _ptr(Q), int(k), int(precision)), "feast_quadrature")
        return self.info()

    def feast_reduced_eig(self, AQ, BQ, M0, eps, Phi, allow=()):
        return self._check(_lib.feast_reduced_eig(self._h, _ptr(AQ), _ptr(BQ), int(M0), _ptr(eps), _ptr(Phi)),
                           "feast_reduced_eig", allow)

    def feast_rayleigh_ritz(self, op, Q, M0, eps, X, AQ=None, BQ=None):
        self._check(_lib.feast_rayleigh_ritz(self._h, ctypes.byref(op), _ptr(Q), int(M0), _ptr(eps), _ptr(X),
                                             _ptr(AQ), _ptr(BQ)), "feast_rayleigh_ritz")

    def feast_residuals(self, op, lam, X, k, resid, resid_paper=None):
        self._check(_lib.feast_residuals(self._h, ctypes.byref(op), _ptr(lam), _ptr(X), int(k), _ptr(resid),
                                         _ptr(resid_paper)), "feast_residuals")


def feast_reduced_eig_noalloc(AQ, BQ, M0, eps, Phi, stream=None) -> int:
    """Allocation-free reduced eigensolve (no handle; device buffers).  Returns
    the feast_status code (FEAST_OK, FEAST_ERR_ARG, FEAST_ERR_BQ_NOT_SPD, ...)."""
    return _lib.feast_reduced_eig_noalloc(_ptr(AQ), _ptr(BQ), int(M0), _ptr(eps), _ptr(Phi),
                                          stream if stream is not None else _current_stream())


class Mlp:
    """Owns one feast_mlp (the learned-start network)."""

    def __init__(self, in_dim, width, out_dim, max_batch, stream=None):
        self._n = _vp()
        st = _lib.feast_mlp_create(ctypes.byref(self._n), int(in_dim), int(width), int(out_dim), int(max_batch),
                                   stream if stream is not None else _current_stream())
        if st != FEAST_OK:
            raise FeastError(st, "feast_mlp_create")
        self.in_dim, self.width, self.out_dim, self.max_batch = in_dim, width, out_dim, max_batch

    def close(self):
        if self._n:
            _lib.feast_mlp_destroy(self._n)
            self._n = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ok(st, what):
        if st != FEAST_OK:
            raise FeastError(st, what)

    def feast_mlp_set_layer(self, k, W, b):
        self._ok(_lib.feast_mlp_set_layer(self._n, int(k), _ptr(W), _ptr(b)), "feast_mlp_set_layer")

    def feast_mlp_get_layer(self, k, W=None, b=None, gW=None, gb=None):
        self._ok(_lib.feast_mlp_get_layer(self._n, int(k), _ptr(W), _ptr(b), _ptr(gW), _ptr(gb)), "feast_mlp_get_layer")

    def feast_mlp_forward(self, X, B, out):
        self._ok(_lib.feast_mlp_forward(self._n, _ptr(X), int(B), _ptr(out)), "feast_mlp_forward")

    def feast_mlp_train_step(self, X, target, weights, B, lr):
        loss = ctypes.c_double(0.0)
        self._ok(_lib.feast_mlp_train_step(self._n, _ptr(X), _ptr(target), _ptr(weights), int(B), float(lr),
                                           ctypes.byref(loss)), "feast_mlp_train_step")
        return loss.value

    def feast_predict_Y(self, features, nx, ny, nz, M0, px, py, Y):
        self._ok(_lib.feast_predict_Y(self._n, _ptr(features), nx, ny, nz, M0, px, py, _ptr(Y)), "feast_predict_Y")


def feast_sine_expand(coef, nx, ny, nz, M0, px, py, Y, stream=None):
    st = _lib.feast_sine_expand(_ptr(coef), nx, ny, nz, M0, px, py, _ptr(Y),
                                stream if stream is not None else _current_stream())
    if st != FEAST_OK:
        raise FeastError(st, "feast_sine_expand")


def feast_sine_project(X, nx, ny, nz, M0, px, py, coef, stream=None):
    st = _lib.feast_sine_project(_ptr(X), nx, ny, nz, M0, px, py, _ptr(coef),
                                 stream if stream is not None else _current_stream())
    if st != FEAST_OK:
        raise FeastError(st, "feast_sine_project")


def library_path() -> str:
    return LIB_PATH
