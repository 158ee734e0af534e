"""Thin ctypes binding of libcggm.so (include/cggm.h), argument marshalling only.

Every function here forwards to the C entry point of the same name; all arithmetic of
the solver runs in the CUDA kernels of the library.  Arrays may be numpy arrays (host)
or torch tensors (host or CUDA device); outputs are numpy arrays unless ``out=``
tensors are given.  There is no CPU fallback: without the compiled library the import
of this module fails.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcggm.so")

CGGM_OK, CGGM_EINVAL, CGGM_ENOTPD, CGGM_ENOMEM, CGGM_EMAXITER = 0, -1, -2, -3, -4
CGGM_ELINESEARCH, CGGM_ECUDA, CGGM_ETIMEDOUT, CGGM_ENONFINITE, CGGM_ECANCELLED = -5, -6, -7, -8, -9
CGGM_FP64, CGGM_MIXED = 0, 1
CGGM_F32, CGGM_F64, CGGM_BF16, CGGM_I8_GENO = 0, 1, 2, 3
CGGM_SWEEP_BATCH_AUTO = -1
CGGM_ORDER_NATURAL, CGGM_ORDER_RCM, CGGM_ORDER_GIVEN, CGGM_ORDER_MINDEG, CGGM_ORDER_AMD = \
    0, 1, 2, 3, 4

EXPORTED = [
    "cggm_create", "cggm_destroy", "cggm_opts_default", "cggm_status_string", "cggm_solve",
    "cggm_solve_dense", "cggm_free_coo", "cggm_server_stats", "cggm_predict",
    "cggm_objective", "cggm_grad", "cggm_cholesky", "cggm_lambda_sweep", "cggm_theta_sweep",
    "cggm_active_sets", "cggm_lambda_sweep_noalloc", "cggm_contract", "cggm_server_create",
    "cggm_server_submit", "cggm_server_poll", "cggm_server_destroy", "cggm_footprint",
    "cggm_spd_solve", "cggm_grad_lambda_block", "cggm_tuned_batch", "cggm_partition_columns",
    "cggm_partition_theta_columns", "cggm_chol_symbolic", "cggm_chol_supernodes",
    "cggm_block_order", "cggm_permute_csr", "cggm_chol_structure", "cggm_tuner_save",
    "cggm_tuner_load", "cggm_block_count", "cggm_spchol_create", "cggm_spchol_factor",
    "cggm_spchol_solve", "cggm_spchol_export", "cggm_spchol_destroy",
]


class cggm_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("ls_sigma", ctypes.c_double), ("ls_beta", ctypes.c_double),
                ("ls_max_trials", ctypes.c_int), ("penalize_diag", ctypes.c_int),
                ("sweep_batch", ctypes.c_int), ("target_f", ctypes.c_double),
                ("verbose", ctypes.c_int), ("sxx_rows", ctypes.c_int64)]


class cggm_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("f", ctypes.c_double),
                ("subgrad", ctypes.c_double), ("l1norm", ctypes.c_double),
                ("m_lambda", ctypes.c_int64), ("m_theta", ctypes.c_int64),
                ("ls_trials", ctypes.c_int), ("seconds", ctypes.c_double),
                ("sec_products", ctypes.c_double), ("sec_factor", ctypes.c_double),
                ("sec_active", ctypes.c_double), ("sec_sweep_lambda", ctypes.c_double),
                ("sec_linesearch", ctypes.c_double), ("sec_sweep_theta", ctypes.c_double),
                ("launches", ctypes.c_int64), ("coords_lambda", ctypes.c_int64),
                ("coords_theta", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cggm_coo(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("row", ctypes.POINTER(ctypes.c_int32)),
                ("col", ctypes.POINTER(ctypes.c_int32)), ("val", ctypes.POINTER(ctypes.c_double))]


class cggm_request(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("xdtype", ctypes.c_int), ("Y", ctypes.c_void_p),
                ("ydtype", ctypes.c_int), ("n", ctypes.c_int64), ("p", ctypes.c_int64),
                ("q", ctypes.c_int64), ("n_lambda", ctypes.c_int),
                ("lambdas", ctypes.POINTER(ctypes.c_double)), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("Lambda_out", ctypes.c_void_p), ("Theta_out", ctypes.c_void_p)]


class cggm_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("arrival_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double),
                ("iterations", ctypes.c_int), ("f_last", ctypes.c_double),
                ("footprint", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CGGMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_lib().cggm_status_string(status).decode()} ({status})")


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i64, dbl, ip = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.cggm_create.argtypes = [ctypes.POINTER(vp), ip, vp]
        lib.cggm_destroy.argtypes = [vp]
        lib.cggm_destroy.restype = None
        lib.cggm_opts_default.argtypes = [ctypes.POINTER(cggm_opts)]
        lib.cggm_opts_default.restype = None
        lib.cggm_status_string.argtypes = [ip]
        lib.cggm_status_string.restype = ctypes.c_char_p
        coo_p = ctypes.POINTER(cggm_coo)
        lib.cggm_solve.argtypes = [vp, vp, ip, vp, ip, i64, i64, i64, dbl, dbl, dbl, coo_p,
                                   coo_p, ctypes.POINTER(cggm_opts), coo_p, coo_p,
                                   ctypes.POINTER(cggm_info)]
        lib.cggm_solve_dense.argtypes = [vp, vp, ip, vp, ip, i64, i64, i64, dbl, dbl, dbl, vp,
                                         vp, ctypes.POINTER(cggm_opts), vp, vp,
                                         ctypes.POINTER(cggm_info)]
        lib.cggm_free_coo.argtypes = [coo_p]
        lib.cggm_free_coo.restype = None
        lib.cggm_predict.argtypes = [vp, vp, ip, i64, i64, i64, coo_p, coo_p, vp, vp]
        lib.cggm_objective.argtypes = [vp, vp, ip, vp, ip, i64, i64, i64, vp, vp, dbl, dbl, ip,
                                       ctypes.POINTER(dbl)]
        lib.cggm_grad.argtypes = [vp, vp, ip, vp, ip, i64, i64, i64, vp, vp, vp, vp]
        lib.cggm_cholesky.argtypes = [vp, i64, vp, vp, ctypes.POINTER(dbl), vp, ip]
        lib.cggm_lambda_sweep.argtypes = [vp, i64, vp, vp, vp, vp, i64, vp, vp, dbl, ip, ip, vp]
        lib.cggm_theta_sweep.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, i64, vp, vp, dbl, ip, vp]
        lib.cggm_active_sets.argtypes = [vp, i64, i64, vp, vp, vp, vp, dbl, dbl, ip, vp, vp,
                                         ctypes.POINTER(i64), vp, vp, ctypes.POINTER(i64)]
        lib.cggm_contract.argtypes = [vp, i64, i64, i64, ctypes.c_float, vp, i64, vp, i64,
                                      ctypes.c_float, vp, i64, ip]
        lib.cggm_server_create.argtypes = [ctypes.POINTER(vp), ip, ip, i64]
        lib.cggm_server_submit.argtypes = [vp, ctypes.POINTER(cggm_request),
                                           ctypes.POINTER(ctypes.c_uint64)]
        lib.cggm_server_poll.argtypes = [vp, ctypes.c_uint64, ip, ctypes.POINTER(cggm_result)]
        lib.cggm_server_destroy.argtypes = [vp]
        lib.cggm_server_destroy.restype = None
        lib.cggm_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                          ctypes.POINTER(i64)]
        lib.cggm_footprint.argtypes = [i64, i64, i64, ip]
        lib.cggm_footprint.restype = i64
        lib.cggm_tuned_batch.argtypes = [i64, i64, ip]
        lib.cggm_tuned_batch.restype = ip
        lib.cggm_lambda_sweep_noalloc.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, dbl, ip, vp,
                                                  vp]
        lib.cggm_spd_solve.argtypes = [vp, i64, vp, vp, vp, i64, vp, i64, dbl, ip, vp,
                                       ctypes.POINTER(ip), ctypes.POINTER(dbl)]
        lib.cggm_grad_lambda_block.argtypes = [vp, vp, ip, vp, ip, i64, i64, i64, vp, vp, vp, vp,
                                               i64, i64, dbl, ip, vp, ctypes.POINTER(ip)]
        lib.cggm_partition_columns.argtypes = [i64, i64, vp, vp, vp, i64, vp,
                                               ctypes.POINTER(i64), ctypes.POINTER(dbl)]
        lib.cggm_partition_theta_columns.argtypes = [i64, i64, i64, vp, vp, i64, vp,
                                                     ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.cggm_chol_symbolic.argtypes = [i64, vp, vp, ip, vp, vp, vp, vp, ctypes.POINTER(i64)]
        lib.cggm_chol_supernodes.argtypes = [i64, vp, vp, vp, ctypes.POINTER(i64)]
        lib.cggm_block_order.argtypes = [ip, i64, i64, vp, vp, vp, vp, ctypes.POINTER(i64),
                                         ctypes.POINTER(i64)]
        lib.cggm_permute_csr.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
        lib.cggm_chol_structure.argtypes = [i64, vp, vp, vp, vp, vp, i64, vp, vp, vp]
        lib.cggm_tuner_save.argtypes = [ctypes.c_char_p, ctypes.POINTER(i64)]
        lib.cggm_tuner_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(i64)]
        lib.cggm_block_count.argtypes = [ip, i64, i64, i64, ctypes.POINTER(i64),
                                         ctypes.POINTER(i64)]
        lib.cggm_spchol_create.argtypes = [vp, i64, vp, vp, ip, vp, ctypes.POINTER(vp)]
        lib.cggm_spchol_factor.argtypes = [vp, vp, ctypes.POINTER(dbl)]
        lib.cggm_spchol_solve.argtypes = [vp, i64, vp, i64, vp]
        lib.cggm_spchol_export.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                           ctypes.POINTER(i64), vp, vp, vp, vp, vp, vp]
        lib.cggm_spchol_destroy.argtypes = [vp]
        for name in EXPORTED:
            f = getattr(lib, name)
            if f.restype is ctypes.c_int or name in ("cggm_create", "cggm_solve",
                                                     "cggm_solve_dense", "cggm_objective",
                                                     "cggm_grad", "cggm_cholesky",
                                                     "cggm_lambda_sweep", "cggm_theta_sweep",
                                                     "cggm_active_sets",
                                                     "cggm_lambda_sweep_noalloc",
                                                     "cggm_contract", "cggm_server_create",
                                                     "cggm_spd_solve", "cggm_grad_lambda_block",
                                                     "cggm_partition_columns",
                                                     "cggm_partition_theta_columns",
                                                     "cggm_chol_symbolic",
                                                     "cggm_chol_supernodes",
                                                     "cggm_block_order",
                                                     "cggm_permute_csr",
                                                     "cggm_chol_structure",
                                                     "cggm_tuner_save", "cggm_tuner_load",
                                                     "cggm_block_count",
                                                     "cggm_server_submit", "cggm_server_poll",
                                                     "cggm_server_stats", "cggm_predict"):
                f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _check(status: int, where: str, allow=(CGGM_OK,)):
    if status not in allow:
        raise CGGMError(status, where)
    return status


class _Arr:
    """Keeps a contiguous array alive and exposes its address (host numpy or torch)."""

    def __init__(self, a, dtype):
        self.obj = None
        try:
            import torch
            if isinstance(a, torch.Tensor):
                tdt = torch.bfloat16 if dtype == "bf16" else {
                    np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
                    np.int8: torch.int8}[np.dtype(dtype).type]
                t = a.to(dtype=tdt).contiguous()
                self.obj = t
                self.ptr = t.data_ptr()
                return
        except ImportError:
            pass
        arr = np.ascontiguousarray(a, dtype=dtype)
        self.obj = arr
        self.ptr = arr.ctypes.data


def _x_dtype(a):
    """(element type, cggm_dtype) of an input matrix: float32, float64, bfloat16 (torch
    tensors) and int8 (genotype counts, standardised by the library) pass through as they
    are; anything else is converted to float64."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return {torch.float32: (np.float32, CGGM_F32), torch.bfloat16: ("bf16", CGGM_BF16),
                    torch.int8: (np.int8, CGGM_I8_GENO)}.get(a.dtype, (np.float64, CGGM_F64))
    except ImportError:
        pass
    return {np.dtype(np.float32): (np.float32, CGGM_F32), np.dtype(np.int8): (np.int8, CGGM_I8_GENO)}.get(
        np.asarray(a).dtype, (np.float64, CGGM_F64))


def opts_default() -> cggm_opts:
    o = cggm_opts()
    _lib().cggm_opts_default(ctypes.byref(o))
    return o


@dataclasses.dataclass
class SolveResult:
    Lambda: object
    Theta: object
    info: dict
    status: int
    Lambda_coo: object = None  # (row, col, val) of cggm_solve: upper triangle of Lambda
    Theta_coo: object = None   # (row, col, val): the nonzero entries of Theta


class _CooIn:
    """A caller's sparse parameter as a cggm_coo over arrays kept alive here.  Accepts a
    (row, col, val) triple or a dense matrix (host numpy or torch), whose nonzero entries
    (only row <= col when `upper`) are listed."""

    def __init__(self, a, upper):
        if isinstance(a, tuple) and len(a) == 3:
            r, c, v = a
        else:
            try:
                import torch
                if isinstance(a, torch.Tensor):
                    a = a.detach().cpu().numpy()
            except ImportError:
                pass
            d = np.asarray(a, dtype=np.float64)
            if upper:
                d = np.triu(d)
            r, c = np.nonzero(d)
            v = d[r, c]
        self.r = np.ascontiguousarray(r, dtype=np.int32)
        self.c = np.ascontiguousarray(c, dtype=np.int32)
        self.v = np.ascontiguousarray(v, dtype=np.float64)
        if not (self.r.shape == self.c.shape == self.v.shape) or self.r.ndim != 1:
            raise ValueError("row, col and val must be 1-D arrays of one length")
        self.coo = cggm_coo(nnz=self.r.size,
                            row=self.r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            col=self.c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            val=self.v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def _coo_take(coo: cggm_coo):
    """Copy a library-allocated coordinate list into numpy arrays and release it."""
    k = int(coo.nnz)
    try:
        r = np.ctypeslib.as_array(coo.row, shape=(k,)).copy() if k else np.zeros(0, np.int32)
        c = np.ctypeslib.as_array(coo.col, shape=(k,)).copy() if k else np.zeros(0, np.int32)
        v = np.ctypeslib.as_array(coo.val, shape=(k,)).copy() if k else np.zeros(0)
    finally:
        _lib().cggm_free_coo(ctypes.byref(coo))
    return r, c, v


def coo_to_dense(coo, shape, symmetric=False):
    """A dense numpy matrix holding the listed entries (both triangles when `symmetric`)."""
    r, c, v = coo
    A = np.zeros(shape)
    A[r, c] = v
    if symmetric:
        A[c, r] = v
    return A


class Context:
    """Owns a cggm_ctx (device workspace + stream)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        h = ctypes.c_void_p()
        _check(_lib().cggm_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream or 0)),
               "cggm_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib().cggm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- cggm_solve --------------------------------------------------------------------
    def cggm_solve(self, X, Y, lam_L, lam_T, tol=0.0, warm_Lambda=None, warm_Theta=None,
                   opts: Optional[cggm_opts] = None, allow_maxiter=True) -> SolveResult:
        """cggm_solve: sparse exchange of the parameters.  warm_Lambda / warm_Theta: a
        (row, col, val) triple (Lambda: its upper triangle) or a dense host matrix whose
        nonzero entries are passed.  The result carries the returned coordinate lists
        (Lambda_coo, Theta_coo) and, for convenience, dense numpy copies of them."""
        n, p = X.shape
        q = Y.shape[1]
        xd, xt = _x_dtype(X)
        yd, yt = _x_dtype(Y)
        Xa, Ya = _Arr(X, xd), _Arr(Y, yd)
        wl = _CooIn(warm_Lambda, True) if warm_Lambda is not None else None
        wt = _CooIn(warm_Theta, False) if warm_Theta is not None else None
        outL, outT = cggm_coo(), cggm_coo()
        info = cggm_info()
        o = opts if opts is not None else opts_default()
        st = _lib().cggm_solve(self._h, Xa.ptr, xt, Ya.ptr, yt, n, p, q, float(lam_L),
                               float(lam_T), float(tol),
                               ctypes.byref(wl.coo) if wl else None,
                               ctypes.byref(wt.coo) if wt else None, ctypes.byref(o),
                               ctypes.byref(outL), ctypes.byref(outT), ctypes.byref(info))
        Lc, Tc = _coo_take(outL), _coo_take(outT)
        _check(st, "cggm_solve", (CGGM_OK, CGGM_EMAXITER) if allow_maxiter else (CGGM_OK,))
        return SolveResult(Lambda=coo_to_dense(Lc, (q, q), symmetric=True),
                           Theta=coo_to_dense(Tc, (p, q)), info=info.as_dict(), status=st,
                           Lambda_coo=Lc, Theta_coo=Tc)

    def cggm_solve_dense(self, X, Y, lam_L, lam_T, tol=0.0, warm_Lambda=None, warm_Theta=None,
                         opts: Optional[cggm_opts] = None, Lambda_out=None, Theta_out=None,
                         allow_maxiter=True) -> SolveResult:
        """cggm_solve_dense: dense parameters, host or device (torch CUDA tensors)."""
        n, p = X.shape
        q = Y.shape[1]
        xd, xt = _x_dtype(X)
        yd, yt = _x_dtype(Y)
        Xa, Ya = _Arr(X, xd), _Arr(Y, yd)
        wl = _Arr(warm_Lambda, np.float64) if warm_Lambda is not None else None
        wt = _Arr(warm_Theta, np.float64) if warm_Theta is not None else None
        Lo = Lambda_out if Lambda_out is not None else np.empty((q, q))
        To = Theta_out if Theta_out is not None else np.empty((p, q))
        La, Ta = _Arr(Lo, np.float64), _Arr(To, np.float64)
        info = cggm_info()
        o = opts if opts is not None else opts_default()
        st = _lib().cggm_solve_dense(self._h, Xa.ptr, xt, Ya.ptr, yt, n, p, q, float(lam_L),
                                     float(lam_T), float(tol), wl.ptr if wl else None,
                                     wt.ptr if wt else None, ctypes.byref(o), La.ptr, Ta.ptr,
                                     ctypes.byref(info))
        _check(st, "cggm_solve_dense",
               (CGGM_OK, CGGM_EMAXITER) if allow_maxiter else (CGGM_OK,))
        return SolveResult(Lambda=La.obj if Lambda_out is None else Lambda_out,
                           Theta=Ta.obj if Theta_out is None else Theta_out,
                           info=info.as_dict(), status=st)

    def cggm_predict(self, X, Lam, Th, q=None, want_B=True):
        """cggm_predict: Yhat = X B with B = -Theta Lambda^-1.  Lam (upper triangle used) and
        Th: (row, col, val) triples (then q is required) or dense host matrices.  Returns
        (Yhat, B or None)."""
        n, p = X.shape
        xd, xt = _x_dtype(X)
        Xa = _Arr(X, xd)
        if q is None:
            q = Lam.shape[0]
        L = _CooIn(Lam, True)
        T = _CooIn(Th, False)
        Yh = np.empty((n, q))
        B = np.empty((p, q)) if want_B else None
        _check(_lib().cggm_predict(self._h, Xa.ptr, xt, n, p, q, ctypes.byref(L.coo),
                                   ctypes.byref(T.coo), Yh.ctypes.data,
                                   B.ctypes.data if B is not None else None), "cggm_predict")
        return Yh, B

    def cggm_objective(self, X, Y, Lam, Th, lam_L, lam_T, penalize_diag=True) -> float:
        n, p = X.shape
        q = Y.shape[1]
        xd, xt = _x_dtype(X)
        yd, yt = _x_dtype(Y)
        Xa, Ya = _Arr(X, xd), _Arr(Y, yd)
        La, Ta = _Arr(Lam, np.float64), _Arr(Th, np.float64)
        f = ctypes.c_double()
        _check(_lib().cggm_objective(self._h, Xa.ptr, xt, Ya.ptr, yt, n, p, q, La.ptr, Ta.ptr,
                                     float(lam_L), float(lam_T), int(bool(penalize_diag)),
                                     ctypes.byref(f)), "cggm_objective")
        return f.value

    def cggm_grad(self, X, Y, Lam, Th):
        n, p = X.shape
        q = Y.shape[1]
        xd, xt = _x_dtype(X)
        yd, yt = _x_dtype(Y)
        Xa, Ya = _Arr(X, xd), _Arr(Y, yd)
        La, Ta = _Arr(Lam, np.float64), _Arr(Th, np.float64)
        GL, GT = np.empty((q, q)), np.empty((p, q))
        _check(_lib().cggm_grad(self._h, Xa.ptr, xt, Ya.ptr, yt, n, p, q, La.ptr, Ta.ptr,
                                GL.ctypes.data, GT.ctypes.data), "cggm_grad")
        return GL, GT

    def cggm_cholesky(self, Lam, want_sigma=True):
        q = Lam.shape[0]
        La = _Arr(Lam, np.float64)
        L = np.empty((q, q))
        S = np.empty((q, q)) if want_sigma else None
        ld = ctypes.c_double()
        _check(_lib().cggm_cholesky(self._h, q, La.ptr, L.ctypes.data, ctypes.byref(ld),
                                    S.ctypes.data if S is not None else None, CGGM_FP64),
               "cggm_cholesky")
        return L, ld.value, S

    def cggm_lambda_sweep(self, Sigma, Psi, Syy, Lam, ai, aj, lam_L, penalize_diag=True,
                          precision=CGGM_FP64):
        q = Lam.shape[0]
        args = [_Arr(a, np.float64) for a in (Sigma, Psi, Syy, Lam)]
        ia, ja = _Arr(ai, np.int32), _Arr(aj, np.int32)
        m = len(ai)
        D = np.empty((q, q))
        _check(_lib().cggm_lambda_sweep(self._h, q, *[a.ptr for a in args], m,
                                        ia.ptr if m else None, ja.ptr if m else None,
                                        float(lam_L), int(bool(penalize_diag)), int(precision),
                                        D.ctypes.data), "cggm_lambda_sweep")
        return D

    def cggm_theta_sweep(self, X, Sxy, Sigma, Theta, ti, tj, lam_T, precision=CGGM_FP64):
        n, p = X.shape
        q = Sigma.shape[0]
        Xa, Sa, Sg, Ta = (_Arr(a, np.float64) for a in (X, Sxy, Sigma, Theta))
        ia, ja = _Arr(ti, np.int32), _Arr(tj, np.int32)
        m = len(ti)
        out = np.empty((p, q))
        _check(_lib().cggm_theta_sweep(self._h, n, p, q, Xa.ptr, Sa.ptr, Sg.ptr, Ta.ptr, m,
                                       ia.ptr if m else None, ja.ptr if m else None,
                                       float(lam_T), int(precision), out.ctypes.data),
               "cggm_theta_sweep")
        return out

    def cggm_contract(self, A, B, C=None, alpha=1.0, beta=0.0, mode=1):
        """C = alpha A B^T + beta C on the tensor cores; A, B, C float32 CUDA tensors."""
        import torch
        M, K = A.shape
        N = B.shape[0]
        if C is None:
            C = torch.zeros((M, N), device=A.device, dtype=torch.float32)
        _check(_lib().cggm_contract(self._h, M, N, K, float(alpha), A.data_ptr(), A.stride(0),
                                    B.data_ptr(), B.stride(0), float(beta), C.data_ptr(),
                                    C.stride(0), int(mode)), "cggm_contract")
        return C

    def cggm_spd_solve(self, indptr, indices, data, B=None, c0=0, k=None, tol=1e-10,
                       max_iter=1000, allow_maxiter=False):
        """Solve Lambda X = B by conjugate gradient, Lambda q x q in CSR (indptr, indices,
        data); B q x k, or None for the identity columns c0 .. c0 + k - 1 (columns of
        Sigma = Lambda^-1).  Returns (X, iterations, largest residual ratio)."""
        q = len(indptr) - 1
        rp = _Arr(indptr, np.int64)
        ci = _Arr(indices, np.int32)
        va = _Arr(data, np.float64)
        if B is not None:
            b = _Arr(B, np.float64)
            k = b.obj.shape[1]
        X = np.empty((q, int(k)))
        it, res = ctypes.c_int(), ctypes.c_double()
        st = _lib().cggm_spd_solve(self._h, q, rp.ptr, ci.ptr, va.ptr, int(k),
                                   b.ptr if B is not None else None, int(c0), float(tol),
                                   int(max_iter), X.ctypes.data, ctypes.byref(it),
                                   ctypes.byref(res))
        _check(st, "cggm_spd_solve", (CGGM_OK, CGGM_EMAXITER) if allow_maxiter else (CGGM_OK,))
        return X, it.value, res.value

    def cggm_spchol(self, indptr, indices, ordering=CGGM_ORDER_AMD, perm=None):
        """Sparse Cholesky plan (cggm_spchol_create) for the q x q pattern in CSR; see
        SparseCholesky."""
        return SparseCholesky(self, indptr, indices, ordering, perm)

    def cggm_grad_lambda_block(self, X, Y, indptr, indices, data, Th, c0, k, tol=1e-10,
                               max_iter=1000):
        """Columns c0 .. c0 + k - 1 of the Lambda gradient from the sparse Lambda (CSR) by
        conjugate gradient, without forming Sigma.  Returns (G block q x k, iterations)."""
        n, p = X.shape
        q = Y.shape[1]
        xd, xt = _x_dtype(X)
        yd, yt = _x_dtype(Y)
        Xa, Ya = _Arr(X, xd), _Arr(Y, yd)
        rp, ci, va = _Arr(indptr, np.int64), _Arr(indices, np.int32), _Arr(data, np.float64)
        Ta = _Arr(Th, np.float64)
        G = np.empty((q, int(k)))
        it = ctypes.c_int()
        _check(_lib().cggm_grad_lambda_block(self._h, Xa.ptr, xt, Ya.ptr, yt, n, p, q, rp.ptr,
                                             ci.ptr, va.ptr, Ta.ptr, int(c0), int(k), float(tol),
                                             int(max_iter), G.ctypes.data, ctypes.byref(it)),
               "cggm_grad_lambda_block")
        return G, it.value

    def cggm_active_sets(self, G_L, G_T, Lam, Th, lam_L, lam_T, penalize_diag=True):
        q = Lam.shape[0]
        p = Th.shape[0]
        a = [_Arr(x, np.float64) for x in (G_L, G_T, Lam, Th)]
        li = np.empty(q * (q + 1) // 2, dtype=np.int32)
        lj = np.empty_like(li)
        ti = np.empty(p * q, dtype=np.int32)
        tj = np.empty_like(ti)
        mL, mT = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib().cggm_active_sets(self._h, p, q, *[x.ptr for x in a], float(lam_L),
                                       float(lam_T), int(bool(penalize_diag)), li.ctypes.data,
                                       lj.ctypes.data, ctypes.byref(mL), ti.ctypes.data,
                                       tj.ctypes.data, ctypes.byref(mT)), "cggm_active_sets")
        return li[:mL.value], lj[:mL.value], ti[:mT.value], tj[:mT.value]


def tuned_batch(q: int, m: int, precision: int) -> int:
    """Batch size the tuner chose for the size class of (q, m, precision); 0 if not tuned yet."""
    return _lib().cggm_tuned_batch(int(q), int(m), int(precision))


def _host_i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


class SparseCholesky:
    """Numeric sparse Cholesky in double precision on the context's GPU (cggm_spchol_*):
    P A P^T = L L^T for a q x q symmetric matrix in CSR whose lower triangle (with the
    diagonal) carries the values.  factor(values) returns log det A; solve() gives A^-1 B
    or columns of A^-1; export() the supernodal structure and blocks; dense_factor() L as a
    dense q x q array in pivot order (small cases)."""

    def __init__(self, ctx, indptr, indices, ordering=CGGM_ORDER_AMD, perm=None):
        rp = np.ascontiguousarray(indptr, dtype=np.int64)
        self.q = q = rp.size - 1
        self.nnz = int(rp[-1]) if q >= 0 else 0
        ci, pci = _host_i32(indices)
        ppi = None
        if perm is not None:
            perm, ppi = _host_i32(perm)
        self._ctx = ctx
        self._h = ctypes.c_void_p()
        _check(_lib().cggm_spchol_create(ctx._h, q, rp.ctypes.data_as(ctypes.c_void_p), pci,
                                         int(ordering), ppi, ctypes.byref(self._h)),
               "cggm_spchol_create")

    def factor(self, values) -> float:
        v = _Arr(values, np.float64)
        ld = ctypes.c_double()
        _check(_lib().cggm_spchol_factor(self._h, v.ptr, ctypes.byref(ld)), "cggm_spchol_factor")
        return ld.value

    def solve(self, B=None, c0=0, k=None):
        if B is not None:
            b = _Arr(B, np.float64)
            k = b.obj.shape[1] if b.obj.ndim == 2 else 1
        X = np.empty((self.q, int(k)))
        _check(_lib().cggm_spchol_solve(self._h, int(k), b.ptr if B is not None else None,
                                        int(c0), X.ctypes.data), "cggm_spchol_solve")
        return X

    def export(self, blocks=True) -> dict:
        ns, nb, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lib = _lib()
        _check(lib.cggm_spchol_export(self._h, ctypes.byref(ns), ctypes.byref(nb),
                                      ctypes.byref(nl), None, None, None, None, None, None),
               "cggm_spchol_export")
        out = {"nsuper": ns.value, "nblock": nb.value, "nnz_L": nl.value,
               "perm": np.empty(self.q, np.int32), "super_start": np.empty(ns.value + 1, np.int64),
               "rows_ptr": np.empty(ns.value + 1, np.int64),
               "block_ptr": np.empty(ns.value + 1, np.int64)}
        _check(lib.cggm_spchol_export(self._h, None, None, None, out["perm"].ctypes.data,
                                      out["super_start"].ctypes.data, out["rows_ptr"].ctypes.data,
                                      None, out["block_ptr"].ctypes.data, None),
               "cggm_spchol_export")
        out["rows"] = np.empty(int(out["rows_ptr"][-1]), np.int32)
        blk = np.empty(nb.value) if blocks else None
        _check(lib.cggm_spchol_export(self._h, None, None, None, None, None, None,
                                      out["rows"].ctypes.data, None,
                                      blk.ctypes.data if blocks else None),
               "cggm_spchol_export")
        out["blocks"] = blk
        return out

    def dense_factor(self):
        """L (pivot order) as a dense q x q array from the exported blocks."""
        e = self.export()
        L = np.zeros((self.q, self.q))
        for s in range(e["nsuper"]):
            f, l = int(e["super_start"][s]), int(e["super_start"][s + 1])
            rows = e["rows"][e["rows_ptr"][s]:e["rows_ptr"][s + 1]]
            nc = l - f
            blk = e["blocks"][e["block_ptr"][s]:e["block_ptr"][s + 1]].reshape(rows.size, nc)
            L[np.ix_(rows, np.arange(f, l))] = blk
        return np.tril(L)

    def close(self):
        if self._h:
            _lib().cggm_spchol_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def partition_columns(q: int, ei, ej, max_block: int, w=None):
    """Column blocks for the block coordinate descent of Algorithm 2
    (cggm_partition_columns): the graph on q columns with edges (ei[t], ej[t]) of weight
    w[t] (default 1) cut into blocks of at most max_block columns.  Host memory only.
    Returns (block, nblocks, cut): the block id of every column, the number of blocks and
    the weight of the edges between blocks."""
    ei, pi = _host_i32(ei)
    ej, pj = _host_i32(ej)
    if ei.shape != ej.shape:
        raise ValueError("ei and ej differ in length")
    pw = None
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != ei.shape:
            raise ValueError("w and ei differ in length")
        pw = w.ctypes.data_as(ctypes.c_void_p)
    block = np.empty(max(int(q), 0), dtype=np.int32)
    k = ctypes.c_int64()
    cut = ctypes.c_double()
    _check(_lib().cggm_partition_columns(int(q), int(ei.size), pi, pj, pw, int(max_block),
                                         block.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k),
                                         ctypes.byref(cut)), "cggm_partition_columns")
    return block, int(k.value), float(cut.value)


def partition_theta_columns(p: int, q: int, ti, tj, max_block: int):
    """Column blocks for the blocked Theta pass of Algorithm 2
    (cggm_partition_theta_columns) from the active coordinates (ti, tj).  Host memory only.
    Returns (block, nblocks, row_blocks): row_blocks is the number of (row, block) pairs
    holding an active entry, the cost Section 4.2 minimises."""
    ti, pi = _host_i32(ti)
    tj, pj = _host_i32(tj)
    if ti.shape != tj.shape:
        raise ValueError("ti and tj differ in length")
    block = np.empty(max(int(q), 0), dtype=np.int32)
    k = ctypes.c_int64()
    rb = ctypes.c_int64()
    _check(_lib().cggm_partition_theta_columns(int(p), int(q), int(ti.size), pi, pj,
                                               int(max_block),
                                               block.ctypes.data_as(ctypes.c_void_p),
                                               ctypes.byref(k), ctypes.byref(rb)),
           "cggm_partition_theta_columns")
    return block, int(k.value), int(rb.value)


def chol_symbolic(q: int, row_ptr, col, ordering: int = CGGM_ORDER_AMD, perm=None):
    """Symbolic analysis of the sparse Cholesky factor of a q x q pattern in CSR
    (cggm_chol_symbolic).  Host memory only.  Returns (perm, parent, colcount, nnz_L):
    the pivot order (new -> old), the elimination tree of the permuted pattern, the
    entries of each column of L (diagonal included) and their sum."""
    q = int(q)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci, pci = _host_i32(col)
    if rp.shape != (q + 1,) and q > 0:
        raise ValueError("row_ptr must hold q + 1 entries")
    ppi = None
    if perm is not None:
        perm, ppi = _host_i32(perm)
        if perm.shape != (q,):
            raise ValueError("perm must hold q entries")
    n = max(q, 0)
    perm_out = np.empty(n, dtype=np.int32)
    parent = np.empty(n, dtype=np.int32)
    count = np.empty(n, dtype=np.int64)
    nnz = ctypes.c_int64()
    _check(_lib().cggm_chol_symbolic(q, rp.ctypes.data_as(ctypes.c_void_p), pci, int(ordering),
                                     ppi, perm_out.ctypes.data_as(ctypes.c_void_p),
                                     parent.ctypes.data_as(ctypes.c_void_p),
                                     count.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nnz)),
           "cggm_chol_symbolic")
    return perm_out, parent, count, int(nnz.value)


def chol_supernodes(parent, colcount):
    """Fundamental supernodes (cggm_chol_supernodes) from the elimination tree and column
    counts of chol_symbolic: the start pivot of each supernode, then q."""
    parent, pp = _host_i32(parent)
    cc = np.ascontiguousarray(colcount, dtype=np.int64)
    q = parent.size
    if cc.shape != (q,):
        raise ValueError("parent and colcount differ in length")
    start = np.empty(q + 1, dtype=np.int64)
    ns = ctypes.c_int64()
    _check(_lib().cggm_chol_supernodes(q, pp, cc.ctypes.data_as(ctypes.c_void_p),
                                       start.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ns)),
           "cggm_chol_supernodes")
    return start[:ns.value + 1].copy()


def block_count(kind: str, q: int, bytes_per_value: int, budget_bytes: int):
    """Blocks of Algorithm 2 for a memory budget by Section 4's rule (cggm_block_count);
    kind "lambda" or "theta".  Returns (k, max_block)."""
    k = ctypes.c_int64()
    mb = ctypes.c_int64()
    _check(_lib().cggm_block_count({"lambda": 0, "theta": 1}[kind], int(q), int(bytes_per_value),
                                   int(budget_bytes), ctypes.byref(k), ctypes.byref(mb)),
           "cggm_block_count")
    return int(k.value), int(mb.value)


def block_order(kind: str, q: int, ci, cj, block):
    """Visiting order of a blocked pass of Algorithm 2 (cggm_block_order); kind "lambda"
    or "theta".  Host memory only.  Returns (order, columns, misses): positions into the
    coordinate list in visiting order, the Sigma columns the pass forms, and its misses
    (off-diagonal block pairs loaded for Lambda, rows of S_xx formed for Theta)."""
    k = {"lambda": 0, "theta": 1}[kind]
    ci, pi = _host_i32(ci)
    cj, pj = _host_i32(cj)
    block, pb = _host_i32(block)
    if ci.shape != cj.shape:
        raise ValueError("ci and cj differ in length")
    if block.shape != (int(q),):
        raise ValueError("block must hold q entries")
    order = np.empty(ci.size, dtype=np.int32)
    cols = ctypes.c_int64()
    miss = ctypes.c_int64()
    _check(_lib().cggm_block_order(k, int(q), int(ci.size), pi, pj, pb,
                                   order.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cols),
                                   ctypes.byref(miss)), "cggm_block_order")
    return order, int(cols.value), int(miss.value)


def permute_csr(q: int, row_ptr, col, val, perm):
    """B = P A P^T of a q x q CSR matrix (cggm_permute_csr), B[k][l] = A[perm[k]][perm[l]].
    Host memory only; val may be None for a pattern.  Returns (row_ptr, col, val)."""
    q = int(q)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci, pci = _host_i32(col)
    perm, pp = _host_i32(perm)
    if rp.shape != (q + 1,) or perm.shape != (q,):
        raise ValueError("row_ptr must hold q + 1 entries and perm q")
    nnz = int(rp[-1]) if q > 0 else 0
    if ci.size != nnz:
        raise ValueError("col must hold row_ptr[q] entries")
    pv = None
    out_val = None
    if val is not None:
        val = np.ascontiguousarray(val, dtype=np.float64)
        if val.shape != (nnz,):
            raise ValueError("val must hold row_ptr[q] entries")
        pv = val.ctypes.data_as(ctypes.c_void_p)
        out_val = np.empty(nnz, dtype=np.float64)
    out_rp = np.empty(q + 1, dtype=np.int64)
    out_ci = np.empty(nnz, dtype=np.int32)
    _check(_lib().cggm_permute_csr(q, rp.ctypes.data_as(ctypes.c_void_p), pci, pv, pp,
                                   out_rp.ctypes.data_as(ctypes.c_void_p),
                                   out_ci.ctypes.data_as(ctypes.c_void_p),
                                   out_val.ctypes.data_as(ctypes.c_void_p)
                                   if out_val is not None else None), "cggm_permute_csr")
    return out_rp, out_ci, out_val


def chol_structure(q: int, row_ptr, col, perm, parent, colcount, super_start):
    """Row structure of each supernode of the factor (cggm_chol_structure) from the outputs
    of chol_symbolic and chol_supernodes.  Host memory only.  Returns (rows_ptr, rows)."""
    q = int(q)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci, pci = _host_i32(col)
    perm, pp = _host_i32(perm)
    parent, ppar = _host_i32(parent)
    cc = np.ascontiguousarray(colcount, dtype=np.int64)
    ss = np.ascontiguousarray(super_start, dtype=np.int64)
    ns = ss.size - 1
    vp = ctypes.c_void_p
    rows_ptr = np.empty(ns + 1, dtype=np.int64)
    args = [q, rp.ctypes.data_as(vp), pci, pp, ppar, cc.ctypes.data_as(vp), ns,
            ss.ctypes.data_as(vp), rows_ptr.ctypes.data_as(vp)]
    _check(_lib().cggm_chol_structure(*args, None), "cggm_chol_structure")
    rows = np.empty(int(rows_ptr[-1]), dtype=np.int32)
    _check(_lib().cggm_chol_structure(*args, rows.ctypes.data_as(vp)), "cggm_chol_structure")
    return rows_ptr, rows


def tuner_save(path) -> int:
    """Write the batch-size tuner's table to `path` (cggm_tuner_save); returns the classes."""
    n = ctypes.c_int64()
    _check(_lib().cggm_tuner_save(os.fsencode(path), ctypes.byref(n)), "cggm_tuner_save")
    return int(n.value)


def tuner_load(path) -> int:
    """Merge a saved tuner table into this process's (cggm_tuner_load); returns the classes."""
    n = ctypes.c_int64()
    _check(_lib().cggm_tuner_load(os.fsencode(path), ctypes.byref(n)), "cggm_tuner_load")
    return int(n.value)


def make_opts(**kw) -> cggm_opts:
    o = opts_default()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": CGGM_FP64, "mixed": CGGM_MIXED}[v]
        if v is None and k == "target_f":
            v = -math.inf
        setattr(o, k, v)
    return o


class Server:
    """Regularisation-path server (cggm_server_*): submit requests as they arrive, poll
    for results.  Keeps every submitted request's arrays alive until it is done."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(_lib().cggm_server_create(ctypes.byref(h), int(device), int(slots),
                                         int(hbm_budget_bytes)), "cggm_server_create")
        self._h = h
        self._keep = {}

    def submit(self, X, Y, lambdas, tol=0.01, max_iter=0, precision=CGGM_MIXED,
               want_outputs=True):
        n, p = X.shape
        q = Y.shape[1]
        xd, xt = _x_dtype(X)
        yd, yt = _x_dtype(Y)
        Xa, Ya = _Arr(X, xd), _Arr(Y, yd)
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        Lo = np.empty((len(lam), q, q)) if want_outputs else None
        To = np.empty((len(lam), p, q)) if want_outputs else None
        r = cggm_request(X=Xa.ptr, xdtype=xt, Y=Ya.ptr, ydtype=yt, n=n, p=p, q=q,
                         n_lambda=len(lam), lambdas=lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         tol=float(tol), max_iter=int(max_iter), precision=int(precision),
                         Lambda_out=Lo.ctypes.data if Lo is not None else None,
                         Theta_out=To.ctypes.data if To is not None else None)
        rid = ctypes.c_uint64()
        _check(_lib().cggm_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)),
               "cggm_server_submit")
        self._keep[rid.value] = (Xa, Ya, lam, Lo, To)
        return rid.value

    def poll(self, rid, wait=False):
        out = cggm_result()
        _check(_lib().cggm_server_poll(self._h, ctypes.c_uint64(rid), int(bool(wait)),
                                       ctypes.byref(out)), "cggm_server_poll")
        d = out.as_dict()
        if d["done"]:
            _, _, _, Lo, To = self._keep[rid]
            d["Lambda"], d["Theta"] = Lo, To
        return d

    def stats(self):
        """cggm_server_stats: pass launches, passes launched, launches holding several."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib().cggm_server_stats(self._h, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c)), "cggm_server_stats")
        return {"pass_launches": a.value, "passes": b.value, "shared_launches": c.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib().cggm_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(n, p, q, precision=CGGM_MIXED) -> int:
    return int(_lib().cggm_footprint(n, p, q, precision))

