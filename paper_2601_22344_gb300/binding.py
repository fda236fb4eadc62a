"""ctypes binding of librplu (include/rplu.h).

Argument marshalling only: every step of the factorization runs in the CUDA
kernels behind the C-ABI.  There is no CPU fallback: if the compiled library
is missing, importing this module raises.

Inputs may be torch tensors (CUDA or CPU) or numpy arrays.  Outputs live where
the input lives: CUDA tensors for a CUDA input (written in place by the
kernels, on the current torch stream), numpy arrays otherwise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Any, Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "librplu.so")

RPLU_OK, RPLU_ERR_INVALID, RPLU_ERR_NOMEM, RPLU_ERR_CUDA, RPLU_ERR_TIMEOUT, RPLU_NOT_CONVERGED, RPLU_CANCELLED = range(7)
DTYPES = {"f32": 0, "f64": 1, "c64": 2, "c128": 3}
PIVOTS = {"random": 0, "c2": 1, "complete": 2, "given": 3}
_NP = {0: np.float32, 1: np.float64, 2: np.complex64, 3: np.complex128}


class Opts(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int32),
        ("pivot", ctypes.c_int32),
        ("rel_tol", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("given_I", ctypes.c_void_p),
        ("given_J", ctypes.c_void_p),
        ("T_hist", ctypes.c_void_p),
        ("d_out", ctypes.c_void_p),
        ("lda", ctypes.c_int64),
        ("overwrite_input", ctypes.c_int32),
        ("pass_block", ctypes.c_int32),
        ("prof", ctypes.c_void_p),
        ("bound_nu", ctypes.c_double),
        ("bound_leaf", ctypes.c_int32),
        ("bound_stop", ctypes.c_int32),
        ("attempts", ctypes.c_void_p),
    ]


class Job(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("k_max", ctypes.c_int64),
        ("lda", ctypes.c_int64),
        ("rel_tol", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("A", ctypes.c_void_p),
        ("x", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("I", ctypes.c_void_p),
        ("J", ctypes.c_void_p),
        ("L", ctypes.c_void_p),
        ("U", ctypes.c_void_p),
        ("k_done", ctypes.c_int64),
        ("status", ctypes.c_int32),
        ("memory", ctypes.c_int32),
        ("rel_res", ctypes.c_double),
    ]


class SessionOpts(ctypes.Structure):
    _fields_ = [
        ("hbm_budget", ctypes.c_int64),
        ("max_jobs", ctypes.c_int32),
        ("max_dim", ctypes.c_int32),
        ("idle_us", ctypes.c_double),
        ("pivot", ctypes.c_int32),
        ("large_streams", ctypes.c_int32),
        ("dense_kernel_cells", ctypes.c_int64),
        ("cauchy_max_dim", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("bound_nu", ctypes.c_double),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("k_max", ctypes.c_int64),
        ("lda", ctypes.c_int64),
        ("rel_tol", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("A", ctypes.c_void_p),
        ("x", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
    ]


class TicketInfo(ctypes.Structure):
    _fields_ = [
        ("state", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("k_done", ctypes.c_int64),
        ("rel_res", ctypes.c_double),
        ("latency_ms", ctypes.c_double),
        ("queue_ms", ctypes.c_double),
    ]


class RPLUError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rplu status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librplu.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_2601_22344_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.rplu_dense.restype = ctypes.c_int
    lib.rplu_dense.argtypes = [P, i64, i64, i64, ctypes.c_uint64, ctypes.POINTER(Opts), P, P, P, P,
                               ctypes.POINTER(i64)]
    lib.rplu_cauchy.restype = ctypes.c_int
    lib.rplu_cauchy.argtypes = [P, P, i64, i64, i64, ctypes.c_uint64, ctypes.POINTER(Opts), P, P, P, P,
                                ctypes.POINTER(i64)]
    lib.rplu_cauchy_like.restype = ctypes.c_int
    lib.rplu_cauchy_like.argtypes = [P, P, P, P, i64, i64, i64, i64, ctypes.c_uint64, ctypes.POINTER(Opts), P, P, P,
                                     P, ctypes.POINTER(i64)]
    lib.rplu_bh_bounds.restype = ctypes.c_int
    lib.rplu_bh_bounds.argtypes = [P, P, P, P, i64, i64, i64, ctypes.c_double, i64, ctypes.POINTER(Opts),
                                   P]
    lib.rplu_bh_plan_stats.restype = ctypes.c_int
    lib.rplu_bh_plan_stats.argtypes = [P, P, i64, i64, ctypes.c_double, i64, ctypes.POINTER(Opts), P]
    lib.rplu_cur_aaa.restype = ctypes.c_int
    lib.rplu_cur_aaa.argtypes = [P, P, i64, ctypes.c_double, i64, ctypes.c_uint64, ctypes.POINTER(Opts), P, P,
                                 ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32), P]
    lib.rplu_barycentric.restype = ctypes.c_int
    lib.rplu_barycentric.argtypes = [P, P, P, i64, P, i64, ctypes.POINTER(Opts), P]
    lib.rplu_cauchy_cur.restype = ctypes.c_int
    lib.rplu_cauchy_cur.argtypes = [P, P, i64, i64, i64, ctypes.c_uint64, ctypes.POINTER(Opts), P, P, P,
                                    ctypes.POINTER(i64)]
    lib.rplu_toeplitz3_cur.restype = ctypes.c_int
    lib.rplu_toeplitz3_cur.argtypes = [i64, ctypes.c_double, ctypes.c_double, ctypes.c_double, i64, ctypes.c_uint64,
                                       ctypes.POINTER(Opts), P, P, P, ctypes.POINTER(i64)]
    lib.rplu_sparse_cur.restype = ctypes.c_int
    lib.rplu_sparse_cur.argtypes = [i64, i64, P, P, P, i64, ctypes.c_uint64, ctypes.POINTER(Opts), P, P, P,
                                    ctypes.POINTER(i64)]
    lib.rplu_batch.restype = ctypes.c_int
    lib.rplu_batch.argtypes = [ctypes.POINTER(Job), ctypes.c_int32, ctypes.POINTER(Opts)]
    lib.rplu_batch_plan_create.restype = ctypes.c_int
    lib.rplu_batch_plan_create.argtypes = [ctypes.POINTER(Job), ctypes.c_int32, ctypes.POINTER(Opts), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_void_p)]
    lib.rplu_batch_plan_run.restype = ctypes.c_int
    lib.rplu_batch_plan_run.argtypes = [P, P]
    lib.rplu_batch_plan_wait.restype = ctypes.c_int
    lib.rplu_batch_plan_wait.argtypes = [P]
    lib.rplu_batch_plan_shape.restype = ctypes.c_int
    lib.rplu_batch_plan_shape.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    lib.rplu_batch_plan_destroy.restype = None
    lib.rplu_batch_plan_destroy.argtypes = [P]
    lib.rplu_session_opts_init.restype = None
    lib.rplu_session_opts_init.argtypes = [ctypes.POINTER(SessionOpts)]
    lib.rplu_session_create.restype = ctypes.c_int
    lib.rplu_session_create.argtypes = [ctypes.POINTER(SessionOpts), ctypes.POINTER(ctypes.c_void_p)]
    lib.rplu_session_submit.restype = ctypes.c_int
    lib.rplu_session_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(i64)]
    lib.rplu_session_poll.restype = ctypes.c_int
    lib.rplu_session_poll.argtypes = [P, i64, ctypes.POINTER(TicketInfo)]
    lib.rplu_session_wait.restype = ctypes.c_int
    lib.rplu_session_wait.argtypes = [P, i64, ctypes.c_double, ctypes.POINTER(TicketInfo)]
    lib.rplu_session_fetch.restype = ctypes.c_int
    lib.rplu_session_fetch.argtypes = [P, i64, P, P, P, P]
    lib.rplu_session_cancel.restype = ctypes.c_int
    lib.rplu_session_cancel.argtypes = [P, i64]
    lib.rplu_session_completed.restype = ctypes.c_int
    lib.rplu_session_completed.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(TicketInfo), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32)]
    lib.rplu_session_stats.restype = ctypes.c_int
    lib.rplu_session_stats.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.rplu_session_destroy.restype = None
    lib.rplu_session_destroy.argtypes = [P]
    lib.rplu_status_string.restype = ctypes.c_char_p
    lib.rplu_status_string.argtypes = [ctypes.c_int]
    lib.rplu_last_error.restype = ctypes.c_char_p
    lib.rplu_last_error.argtypes = []
    lib.rplu_version.restype = ctypes.c_int32
    lib.rplu_opts_init.restype = None
    lib.rplu_opts_init.argtypes = [ctypes.POINTER(Opts)]
    return lib


lib = _load()

EXPORTED = ["rplu_opts_init", "rplu_dense", "rplu_cauchy", "rplu_cauchy_cur", "rplu_toeplitz3_cur", "rplu_sparse_cur", "rplu_cauchy_like", "rplu_bh_bounds", "rplu_bh_plan_stats",
            "rplu_cur_aaa", "rplu_barycentric", "rplu_batch", "rplu_batch_plan_create",
            "rplu_batch_plan_run", "rplu_batch_plan_wait", "rplu_batch_plan_shape", "rplu_batch_plan_destroy",
            "rplu_session_opts_init", "rplu_session_create", "rplu_session_submit", "rplu_session_poll",
            "rplu_session_wait", "rplu_session_fetch", "rplu_session_cancel", "rplu_session_completed",
            "rplu_session_stats",
            "rplu_session_destroy",
            "rplu_status_string", "rplu_last_error", "rplu_version"]


@dataclass
class Result:
    I: Any
    J: Any
    L: Any          # n x k_done
    U: Any          # k_done x m
    k_done: int
    T: np.ndarray   # ||S^(t)||_F^2, t = 0..k_done
    d: Optional[Any]
    status: int


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _dtype_code(a) -> int:
    if _is_torch(a):
        import torch
        m = {torch.float32: 0, torch.float64: 1, torch.complex64: 2, torch.complex128: 3}
        if a.dtype not in m:
            raise TypeError(f"unsupported dtype {a.dtype}")
        return m[a.dtype]
    m = {np.dtype(np.float32): 0, np.dtype(np.float64): 1, np.dtype(np.complex64): 2,
         np.dtype(np.complex128): 3}
    if a.dtype not in m:
        raise TypeError(f"unsupported dtype {a.dtype}")
    return m[a.dtype]


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


class _Alloc:
    """Output allocation on the input's side: torch CUDA tensors for a CUDA
    input, pinned torch CPU tensors for a pinned CPU tensor, numpy otherwise."""

    def __init__(self, like):
        self.torch = _is_torch(like) and like.is_cuda
        self.pinned = _is_torch(like) and not like.is_cuda and like.is_pinned()
        self.device = like.device if self.torch else None

    def empty(self, shape, code):
        if self.torch or self.pinned:
            import torch
            tdt = {0: torch.float32, 1: torch.float64, 2: torch.complex64, 3: torch.complex128,
                   "i64": torch.int64}[code]
            if self.pinned:
                return torch.empty(shape, dtype=tdt, pin_memory=True)
            return torch.empty(shape, dtype=tdt, device=self.device)
        npdt = np.int64 if code == "i64" else _NP[code]
        return np.empty(shape, dtype=npdt)

    def stream(self):
        if self.torch:
            import torch
            return torch.cuda.current_stream(self.device).cuda_stream
        return None


def _host_array(a, dtype=None):
    if _is_torch(a):
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _check(status: int, allow_not_converged=True):
    if status == RPLU_OK or (allow_not_converged and status == RPLU_NOT_CONVERGED):
        return
    raise RPLUError(status, lib.rplu_last_error().decode())


def _opts(code, pivot, rel_tol, stream, given, k, T, d, lda=0, overwrite=False, prof=None, pass_block=0):
    o = Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.dtype = code
    o.pivot = PIVOTS[pivot]
    o.rel_tol = float(rel_tol)
    o.stream = stream
    keep = []
    if pivot == "given":
        gI = np.ascontiguousarray(np.asarray(given[0], dtype=np.int64))
        gJ = np.ascontiguousarray(np.asarray(given[1], dtype=np.int64))
        if len(gI) < k or len(gJ) < k:
            raise ValueError("given pivots shorter than k")
        o.given_I = gI.ctypes.data
        o.given_J = gJ.ctypes.data
        keep += [gI, gJ]
    o.T_hist = T.ctypes.data
    o.d_out = _ptr(d)
    o.lda = lda
    o.overwrite_input = int(overwrite)
    o.pass_block = int(pass_block)
    if prof is not None:
        if not (isinstance(prof, np.ndarray) and prof.dtype == np.float64 and prof.size >= 4):
            raise TypeError("prof must be a float64 numpy array of 4 entries")
        o.prof = prof.ctypes.data
    return o, keep


def _finish(al, I, J, L, U, kd, T, d, status):
    k = kd
    if al.torch or al.pinned:
        return Result(I[:k], J[:k], L[:k].T, U[:k], k, T[:k + 1].copy(), d, status)
    return Result(I[:k].copy(), J[:k].copy(), np.ascontiguousarray(L[:k].T), U[:k].copy(), k,
                  T[:k + 1].copy(), d, status)


def rplu_dense(A, k: int, seed: int = 0, *, pivot: str = "random", rel_tol: float = 0.0, given=None,
               overwrite_input: bool = False, return_d: bool = False, prof=None, pass_block: int = 0) -> Result:
    """Dense-form RPLU (rplu_dense in include/rplu.h) of a 2-D array A.
    prof: optional float64[4] accumulator (see rplu_opts.prof); pass_block:
    steps between write-backs of the residual (0 = library default)."""
    if _is_torch(A):
        if A.dim() != 2 or (A.shape[1] > 1 and A.stride(1) != 1):
            raise ValueError("A must be 2-D with unit column stride")
        lda = A.stride(0) if A.shape[0] > 1 else A.shape[1]
        if not A.is_cuda and not A.is_pinned():
            A = A.detach().contiguous().numpy()
            lda = A.shape[1]
    else:
        A = np.ascontiguousarray(A)
        lda = A.shape[1]
    n, m = A.shape
    code = _dtype_code(A)
    al = _Alloc(A)
    kk = max(k, 1)
    I = al.empty((kk,), "i64")
    J = al.empty((kk,), "i64")
    L = al.empty((kk, n), code)   # column-major n x k
    U = al.empty((kk, m), code)
    T = np.zeros(k + 1)
    d = al.empty((max(n, 1),), 1) if return_d else None
    o, keep = _opts(code, pivot, rel_tol, al.stream(), given, k, T, d, lda, overwrite_input, prof, pass_block)
    kd = ctypes.c_int64(0)
    st = lib.rplu_dense(_ptr(A), n, m, k, ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(o), _ptr(I), _ptr(J),
                        _ptr(L), _ptr(U), ctypes.byref(kd))
    _check(st)
    return _finish(al, I, J, L, U, kd.value, T, d[:n] if d is not None else None, st)


def rplu_cauchy(x, y, k: int, seed: int = 0, *, pivot: str = "random", rel_tol: float = 0.0, given=None,
                return_d: bool = False, prof=None) -> Result:
    """Matrix-free RPLU of A_ij = 1/(x_i - y_j) (rplu_cauchy in include/rplu.h).
    x and y must have the same dtype: float32/float64 (real points) or
    complex64/complex128."""
    if _is_torch(x) and not x.is_cuda and x.is_pinned():
        if x.dtype != y.dtype or not y.is_pinned():
            raise TypeError("x and y must share dtype and pinning")
    elif not _is_torch(x) or not x.is_cuda:
        x = _host_array(x)
        y = _host_array(y, dtype=x.dtype)
    elif x.dtype != y.dtype or not y.is_cuda:
        raise TypeError("x and y must share dtype and device")
    else:
        x = x.contiguous()
        y = y.contiguous()
    n, m = x.shape[0], y.shape[0]
    code = _dtype_code(x)
    al = _Alloc(x)
    kk = max(k, 1)
    I = al.empty((kk,), "i64")
    J = al.empty((kk,), "i64")
    L = al.empty((kk, n), code)
    U = al.empty((kk, m), code)
    T = np.zeros(k + 1)
    d = al.empty((max(n, 1),), 1) if return_d else None
    o, keep = _opts(code, pivot, rel_tol, al.stream(), given, k, T, d, prof=prof)
    kd = ctypes.c_int64(0)
    st = lib.rplu_cauchy(_ptr(x), _ptr(y), n, m, k, ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(o), _ptr(I),
                         _ptr(J), _ptr(L), _ptr(U), ctypes.byref(kd))
    _check(st)
    return _finish(al, I, J, L, U, kd.value, T, d[:n] if d is not None else None, st)


@dataclass
class CurResult:
    I: Any
    J: Any
    core: Any         # k_done x k_done, FP64: A ~ A(:,J) core A(I,:)
    k_done: int
    T: np.ndarray
    status: int


def rplu_cauchy_cur(x, y, k: int, seed: int = 0, *, pivot: str = "random", rel_tol: float = 0.0,
                    given=None, prof=None) -> CurResult:
    """Matrix-free RPLU of the Cauchy matrix 1/(x_i - y_j) in CUR form
    (rplu_cauchy_cur in include/rplu.h): pivots and the core inverse, no L, U."""
    if _is_torch(x) and x.is_cuda:
        if not (_is_torch(y) and y.is_cuda and y.dtype == x.dtype):
            raise TypeError("x and y must share dtype and device")
        x, y = x.contiguous(), y.contiguous()
    else:
        x = _host_array(x)
        y = _host_array(y, dtype=x.dtype)
    n, m = x.shape[0], y.shape[0]
    code = _dtype_code(x)
    al = _Alloc(x)
    kk = max(k, 1)
    I = al.empty((kk,), "i64")
    J = al.empty((kk,), "i64")
    C = al.empty((kk, kk), 3 if code in (2, 3) else 1)  # the core is FP64
    T = np.zeros(k + 1)
    o, keep = _opts(code, pivot, rel_tol, al.stream(), given, k, T, None, prof=prof)
    kd = ctypes.c_int64(0)
    st = lib.rplu_cauchy_cur(_ptr(x), _ptr(y), n, m, k, ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(o),
                             _ptr(I), _ptr(J), _ptr(C), ctypes.byref(kd))
    _check(st)
    kdone = kd.value
    return CurResult(I[:kdone], J[:kdone], C[:kdone, :kdone], kdone, T[:kdone + 1].copy(), st)


def rplu_toeplitz3_cur(N: int, k: int, seed: int = 0, *, length: float = 320.0, delta: float = 50.0,
                       sigma: float = 80.0, pivot: str = "random", rel_tol: float = 0.0, given=None, prof=None,
                       device: str = "cuda") -> CurResult:
    """RPLU in CUR form of the multi-level Toeplitz matrix of the drifted
    Gaussian kernel on an N^3 grid (rplu_toeplitz3_cur in include/rplu.h):
    pivots and the FP64 core inverse.  Outputs are torch CUDA tensors
    (device="cuda") or numpy arrays (device="host")."""
    if device == "cuda":
        import torch
        like = torch.empty(0, dtype=torch.float64, device="cuda")
    elif device == "host":
        like = np.empty(0)
    else:
        raise ValueError("device must be 'cuda' or 'host'")
    al = _Alloc(like)
    kk = max(k, 1)
    I = al.empty((kk,), "i64")
    J = al.empty((kk,), "i64")
    C = al.empty((kk, kk), 1)
    T = np.zeros(k + 1)
    o, keep = _opts(1, pivot, rel_tol, al.stream(), given, k, T, None, prof=prof)
    kd = ctypes.c_int64(0)
    st = lib.rplu_toeplitz3_cur(int(N), float(length), float(delta), float(sigma), int(k),
                                ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(o), _ptr(I), _ptr(J), _ptr(C),
                                ctypes.byref(kd))
    _check(st)
    kdone = kd.value
    return CurResult(I[:kdone], J[:kdone], C[:kdone, :kdone], kdone, T[:kdone + 1].copy(), st)


def rplu_sparse_cur(A, k: int, seed: int = 0, *, pivot: str = "random", rel_tol: float = 0.0, given=None,
                    prof=None, device: str = "cuda") -> CurResult:
    """RPLU in CUR form of a sparse real matrix (rplu_sparse_cur in
    include/rplu.h).  A: a scipy.sparse matrix, taken in canonical CSR form
    (duplicates summed, indices sorted) in FP64.  Outputs are torch CUDA
    tensors (device="cuda") or numpy arrays (device="host")."""
    import scipy.sparse as sp

    S = sp.csr_matrix(A, dtype=np.float64, copy=True)
    S.sum_duplicates()
    S.sort_indices()
    indptr = np.ascontiguousarray(S.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(S.indices, dtype=np.int32)
    data = np.ascontiguousarray(S.data, dtype=np.float64)
    n, m = S.shape
    if device == "cuda":
        import torch
        like = torch.empty(0, dtype=torch.float64, device="cuda")
    elif device == "host":
        like = np.empty(0)
    else:
        raise ValueError("device must be 'cuda' or 'host'")
    al = _Alloc(like)
    kk = max(k, 1)
    I = al.empty((kk,), "i64")
    J = al.empty((kk,), "i64")
    C = al.empty((kk, kk), 1)
    T = np.zeros(k + 1)
    o, keep = _opts(1, pivot, rel_tol, al.stream(), given, k, T, None, prof=prof)
    kd = ctypes.c_int64(0)
    st = lib.rplu_sparse_cur(n, m, _ptr(indptr), _ptr(indices), _ptr(data), int(k),
                             ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(o), _ptr(I), _ptr(J), _ptr(C),
                             ctypes.byref(kd))
    _check(st)
    kdone = kd.value
    return CurResult(I[:kdone], J[:kdone], C[:kdone, :kdone], kdone, T[:kdone + 1].copy(), st)


def _generators(x, y, G, B):
    on_dev = _is_torch(x) and x.is_cuda
    if on_dev:
        if not all(_is_torch(v) and v.is_cuda and v.dtype == x.dtype for v in (y, G, B)):
            raise TypeError("x, y, G and B must share dtype and device")
        x, y, G, B = x.contiguous(), y.contiguous(), G.contiguous(), B.contiguous()
    else:
        x = _host_array(x)
        y = _host_array(y, dtype=x.dtype)
        G = _host_array(G, dtype=x.dtype)
        B = _host_array(B, dtype=x.dtype)
    n, m = x.shape[0], y.shape[0]
    p = G.shape[1] if len(G.shape) == 2 else 1
    if tuple(G.shape[:1]) != (n,) or (len(B.shape) == 2 and tuple(B.shape) != (p, m)):
        raise ValueError("G must be n x p and B p x m")
    return x, y, G, B, n, m, p


def rplu_bh_bounds(x, y, G, B, nu: float = 5.0, leaf: int = 32):
    """Row-norm upper bounds of App. C for the Cauchy-like matrix of (x, y, G,
    B) (rplu_bh_bounds in include/rplu.h): float64 array (or CUDA tensor) of n."""
    x, y, G, B, n, m, p = _generators(x, y, G, B)
    al = _Alloc(x)
    u = al.empty((max(n, 1),), 1)
    o = Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.dtype = _dtype_code(x)
    o.stream = al.stream()
    st = lib.rplu_bh_bounds(_ptr(x), _ptr(y), _ptr(G), _ptr(B), n, m, p, float(nu), int(leaf), ctypes.byref(o),
                            _ptr(u))
    _check(st)
    return u[:n]


def rplu_bh_plan_stats(x, y, nu: float = 5.0, leaf: int = 32) -> dict:
    """Size of the App. C plan for the points x, y (rplu_bh_plan_stats in include/rplu.h)."""
    if _is_torch(x) and x.is_cuda:
        x, y = x.contiguous(), y.contiguous()
    else:
        x = _host_array(x)
        y = _host_array(y, dtype=x.dtype)
    o = Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.dtype = _dtype_code(x)
    st = np.zeros(6, dtype=np.int64)
    _check(lib.rplu_bh_plan_stats(_ptr(x), _ptr(y), x.shape[0], y.shape[0], float(nu), int(leaf), ctypes.byref(o),
                                  st.ctypes.data))
    keys = ("target_leaves", "source_nodes", "source_leaves", "aggregated_entries", "exact_pairs",
            "max_target_leaf")
    return {k_: int(v) for k_, v in zip(keys, st)}


@dataclass
class CurAaa:
    support: Any      # indices into z of the support points
    weights: Any      # barycentric weights (2-norm 1)
    k: int
    which: str        # "I" (row pivots, X half) or "J" (column pivots, Y half)
    err_I: float      # max |f - r| over the samples for each candidate
    err_J: float
    status: int

    def __call__(self, zq, z, f):
        """r(zq) (rplu_barycentric): zq on the device of z, from the samples z, f
        this fit was made on."""
        return rplu_barycentric(z, f, self.support, self.weights, zq)


def rplu_barycentric(z, f, support, weights, zq):
    """r(zq) of Eq. aaa-barycentric for the support points z[support] with values
    f[support] and the given weights (rplu_barycentric in include/rplu.h)."""
    if _is_torch(z) and z.is_cuda:
        import torch
        sup = torch.as_tensor(support, device=z.device, dtype=torch.int64)
        t, ft = z[sup].to(torch.complex128).contiguous(), f[sup].to(torch.complex128).contiguous()
        w = torch.as_tensor(weights, device=z.device).to(torch.complex128).contiguous()
        zq = torch.as_tensor(zq, device=z.device).to(torch.complex128).contiguous()
    else:
        sup = np.asarray(support.cpu() if _is_torch(support) else support, dtype=np.int64)
        t = np.ascontiguousarray(np.asarray(z, dtype=np.complex128)[sup])
        ft = np.ascontiguousarray(np.asarray(f, dtype=np.complex128)[sup])
        w = np.ascontiguousarray(np.asarray(weights.cpu() if _is_torch(weights) else weights, dtype=np.complex128))
        zq = np.ascontiguousarray(np.asarray(zq, dtype=np.complex128))
    al = _Alloc(zq)
    rq = al.empty((max(zq.shape[0], 1),), 3)
    o = Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.dtype = 3
    o.stream = al.stream()
    _check(lib.rplu_barycentric(_ptr(t), _ptr(ft), _ptr(w), t.shape[0], _ptr(zq), zq.shape[0], ctypes.byref(o),
                                _ptr(rq)))
    return rq[:zq.shape[0]]


def rplu_cur_aaa(z, f, eps: float, k_max: int = 1000, seed: int = 0, *, pivot: str = "random",
                 nu: float = 5.0, leaf: int = 0) -> CurAaa:
    """CUR-AAA rational approximation (rplu_cur_aaa in include/rplu.h): z, f
    complex128 samples and values (numpy arrays or CUDA tensors)."""
    on_dev = _is_torch(z) and z.is_cuda
    if on_dev:
        import torch
        z = z.to(torch.complex128).contiguous()
        f = f.to(device=z.device, dtype=torch.complex128).contiguous()
    else:
        z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
        f = np.ascontiguousarray(np.asarray(f, dtype=np.complex128))
    m = z.shape[0]
    al = _Alloc(z)
    kk = max(1, min(k_max, m // 2))
    sup = al.empty((kk,), "i64")
    w = al.empty((kk,), 3)
    o = Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.dtype = 3
    o.pivot = PIVOTS[pivot]
    o.stream = al.stream()
    o.bound_nu = float(nu)
    o.bound_leaf = int(leaf)
    kd = ctypes.c_int64(0)
    which = ctypes.c_int32(0)
    err = np.zeros(2)
    st = lib.rplu_cur_aaa(_ptr(z), _ptr(f), m, float(eps), int(k_max), ctypes.c_uint64(seed & (2**64 - 1)),
                          ctypes.byref(o), _ptr(sup), _ptr(w), ctypes.byref(kd), ctypes.byref(which),
                          err.ctypes.data)
    _check(st)
    k = kd.value
    return CurAaa(sup[:k], w[:k], k, "IJ"[which.value], float(err[0]), float(err[1]), st)


def rplu_cauchy_like(x, y, G, B, k: int, seed: int = 0, *, pivot: str = "random", rel_tol: float = 0.0,
                     given=None, return_d: bool = False, prof=None, bound_nu: float = 0.0,
                     bound_leaf: int = 0, bound_stop: str = "sum") -> Result:
    """RPLU of the Cauchy-like matrix A_ij = sum_l G[i,l] B[l,j] / (x_i - y_j)
    through its generators (rplu_cauchy_like in include/rplu.h).  x, y, G
    (n x p) and B (p x m) share one dtype and device.  bound_nu >= 1 selects
    Algorithm 3's rejection-sampled row draw against the bounds of App. C
    (quadtree leaves of at most bound_leaf points, 0 = library default); the
    result then carries `attempts` (proposals per step, 65 = exact fallback);
    with pivot="c2" the approximate C2PLU with the same bounds; bound_stop="max"
    stops on max(u) <= rel_tol^2 max(u at step 0) (the CUR-AAA rule)."""
    on_dev = _is_torch(x) and x.is_cuda
    if on_dev:
        if not all(_is_torch(v) and v.is_cuda and v.dtype == x.dtype for v in (y, G, B)):
            raise TypeError("x, y, G and B must share dtype and device")
        x, y, G, B = x.contiguous(), y.contiguous(), G.contiguous(), B.contiguous()
    else:
        x = _host_array(x)
        y = _host_array(y, dtype=x.dtype)
        G = _host_array(G, dtype=x.dtype)
        B = _host_array(B, dtype=x.dtype)
    n, m = x.shape[0], y.shape[0]
    p = G.shape[1] if len(G.shape) == 2 else 1
    if tuple(G.shape[:1]) != (n,) or (len(B.shape) == 2 and tuple(B.shape) != (p, m)):
        raise ValueError("G must be n x p and B p x m")
    code = _dtype_code(x)
    al = _Alloc(x)
    kk = max(k, 1)
    I = al.empty((kk,), "i64")
    J = al.empty((kk,), "i64")
    L = al.empty((kk, n), code)
    U = al.empty((kk, m), code)
    T = np.zeros(k + 1)
    d = al.empty((max(n, 1),), 1) if return_d else None
    o, keep = _opts(code, pivot, rel_tol, al.stream(), given, k, T, d, prof=prof)
    o.bound_nu = float(bound_nu)
    o.bound_leaf = int(bound_leaf)
    o.bound_stop = {"sum": 0, "max": 1}[bound_stop]
    att = np.zeros(max(k, 1), dtype=np.int32)
    if bound_nu:
        o.attempts = att.ctypes.data
    kd = ctypes.c_int64(0)
    st = lib.rplu_cauchy_like(_ptr(x), _ptr(y), _ptr(G), _ptr(B), n, m, p, k, ctypes.c_uint64(seed & (2**64 - 1)),
                              ctypes.byref(o), _ptr(I), _ptr(J), _ptr(L), _ptr(U), ctypes.byref(kd))
    _check(st)
    res = _finish(al, I, J, L, U, kd.value, T, d[:n] if d is not None else None, st)
    res.attempts = att[:kd.value].copy() if bound_nu else None
    return res


def status_string(status: int) -> str:
    return lib.rplu_status_string(status).decode()


def version() -> int:
    return int(lib.rplu_version())
