"""CPU oracle for Randomly Pivoted LU -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
bench.py may import this package.  The product library (the CUDA path behind
include/rplu.h) never calls it and shares no code with it.

The arithmetic lives in rplu_oracle.c (plain sequential C, FP64/complex128,
compiled without FMA contraction); this module only compiles it with gcc and
marshals numpy arrays through ctypes.

Functions and the paper passages they follow:
  rplu_dense   Algorithm 1 (Sec. 1) with the two-stage pivot draw of Sec. 4.1;
               modes: random (RPLU), c2 (complete 2-norm pivoting, Sec. 2),
               complete (complete pivoting, Sec. 1), given (fixed pivots).
  rplu_cauchy  matrix-free LU-form RPLU for A_ij = 1/(x_i - y_j) (Sec. 5.1
               with p = 1), residual rows/columns as in Algorithm 2 (Sec. 4.1)
               and the row-norm update formula of Sec. 4.1.
  rplu_cauchy_like
               RPLU of a Cauchy-like matrix (Eq. cauchy-like) through its
               generators: Algorithm 3 (Sec. 5.1) with the generator updates
               of Eqs. generator_update_g/b and exact row norms recomputed
               from the generators every step.
  bh_bounds, rplu_cauchy_like_bh
               the row-norm upper bounds of App. C (quadtrees, Algorithms
               C.1/C.2) and the factorization with Algorithm 3's rejection-
               sampled row draw.
  u01          the counter-based uniform draw both sides implement.

Modules in numpy over the C oracle's draws:
  cur_form     Algorithm 2 (RPLU in CUR form, Sec. 4.1) over a general operator:
               dense, Cauchy, sparse, and the multi-level Toeplitz matrix of the
               drifted Gaussian kernel (Sec. 4.2, Eq. kernel).
  cur_aaa      CUR-AAA (Sec. 5.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rplu_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES = {"random": 0, "c2": 1, "complete": 2, "given": 3}


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle (default: oracle/_build/liboracle.so) with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _given(given, k):
    if given is None:
        return None, None
    gI = np.ascontiguousarray(np.asarray(given[0], dtype=np.int64))
    gJ = np.ascontiguousarray(np.asarray(given[1], dtype=np.int64))
    if len(gI) < k or len(gJ) < k:
        raise ValueError("given pivots shorter than k")
    return gI, gJ


class Oracle:
    """ctypes binding of one compiled copy of rplu_oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_u01.restype = ctypes.c_double
        lib.oracle_u01.argtypes = [ctypes.c_uint64, i64, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_inverse_cdf.restype = i64
        lib.oracle_inverse_cdf.argtypes = [P, i64, ctypes.c_double, ctypes.c_double, P]
        dense_args = [P, i64, i64, i64, ctypes.c_uint64, ctypes.c_int32, P, P, ctypes.c_double,
                      P, P, P, P, P, P, P, P]
        for name in ("oracle_rplu_dense_f64", "oracle_rplu_dense_c128"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = dense_args
        lib.oracle_rplu_cauchy.restype = ctypes.c_int
        lib.oracle_rplu_cauchy.argtypes = [P, P, i64, i64, i64, ctypes.c_uint64, ctypes.c_int32, P, P,
                                           ctypes.c_double, P, P, P, P, P, P, P, P, P]
        lib.oracle_rplu_cauchy_like.restype = ctypes.c_int
        lib.oracle_rplu_cauchy_like.argtypes = [P, P, P, P, i64, i64, i64, i64, ctypes.c_uint64, ctypes.c_int32,
                                                P, P, ctypes.c_double, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_bh_bounds.restype = ctypes.c_int
        lib.oracle_bh_bounds.argtypes = [P, P, P, P, i64, i64, i64, ctypes.c_double, i64, P, P]
        lib.oracle_rplu_cauchy_like_bh.restype = ctypes.c_int
        lib.oracle_rplu_cauchy_like_bh.argtypes = [P, P, P, P, i64, i64, i64, i64, ctypes.c_uint64, ctypes.c_double,
                                                   i64, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P,
                                                   P, P, P, P]
        self.lib = lib
        self.path = path

    def u01(self, seed: int, t: int, s: int, a: int = 0) -> float:
        """U01(seed, t, s, a): the uniform draw for step t, stage s (0 row,
        1 column), redraw attempt a."""
        return self.lib.oracle_u01(ctypes.c_uint64(seed & (2**64 - 1)), t, s, a)

    def inverse_cdf(self, w, target: float, total: float):
        w = np.ascontiguousarray(w, dtype=np.float64)
        margin = np.zeros(1)
        i = self.lib.oracle_inverse_cdf(_ptr(w), len(w), target, total, _ptr(margin))
        return int(i), float(margin[0])

    def rplu_dense(self, A, k: int, seed: int = 0, mode: str = "random", tol: float = 0.0, given=None) -> dict:
        """Dense-form RPLU of A (n x m, real or complex) to rank k.

        Returns a dict with I, J (int64[k_done]), L (n x k_done), U (k_done x m),
        T (||S^(t)||_F^2 for t = 0..k_done), row_margin, col_margin (distance of
        each draw to the nearest CDF boundary, relative to the total) and k_done."""
        A = np.asarray(A)
        cplx = np.iscomplexobj(A)
        A = np.ascontiguousarray(A, dtype=np.complex128 if cplx else np.float64)
        n, m = A.shape
        dt = A.dtype
        I = np.zeros(max(k, 1), np.int64)
        J = np.zeros(max(k, 1), np.int64)
        L = np.zeros((max(k, 1), n), dt)  # column-major n x k == row-major k x n
        U = np.zeros((max(k, 1), m), dt)
        T = np.zeros(k + 1)
        rm = np.zeros(max(k, 1))
        cm = np.zeros(max(k, 1))
        kd = np.zeros(1, np.int64)
        gI, gJ = _given(given, k)
        f = self.lib.oracle_rplu_dense_c128 if cplx else self.lib.oracle_rplu_dense_f64
        rc = f(_ptr(A), n, m, k, ctypes.c_uint64(seed & (2**64 - 1)), MODES[mode], _ptr(gI), _ptr(gJ), tol,
               _ptr(I), _ptr(J), _ptr(L), _ptr(U), _ptr(T), _ptr(rm), _ptr(cm), _ptr(kd))
        if rc != 0:
            raise ValueError("oracle_rplu_dense: invalid arguments")
        kd = int(kd[0])
        return dict(I=I[:kd].copy(), J=J[:kd].copy(), L=np.ascontiguousarray(L[:kd].T), U=U[:kd].copy(),
                    T=T[:kd + 1].copy(), row_margin=rm[:kd].copy(), col_margin=cm[:kd].copy(), k_done=kd)

    def rplu_cauchy(self, x, y, k: int, seed: int = 0, mode: str = "random", tol: float = 0.0,
                    given=None) -> dict:
        """Matrix-free RPLU of the Cauchy matrix A_ij = 1/(x_i - y_j),
        complex128.  Same outputs as rplu_dense plus d, the row-norm estimates
        after the last step."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.complex128))
        n, m = len(x), len(y)
        I = np.zeros(max(k, 1), np.int64)
        J = np.zeros(max(k, 1), np.int64)
        L = np.zeros((max(k, 1), n), np.complex128)
        U = np.zeros((max(k, 1), m), np.complex128)
        d = np.zeros(max(n, 1))
        T = np.zeros(k + 1)
        rm = np.zeros(max(k, 1))
        cm = np.zeros(max(k, 1))
        kd = np.zeros(1, np.int64)
        gI, gJ = _given(given, k)
        rc = self.lib.oracle_rplu_cauchy(_ptr(x), _ptr(y), n, m, k, ctypes.c_uint64(seed & (2**64 - 1)),
                                         MODES[mode], _ptr(gI), _ptr(gJ), tol, _ptr(I), _ptr(J), _ptr(L),
                                         _ptr(U), _ptr(d), _ptr(T), _ptr(rm), _ptr(cm), _ptr(kd))
        if rc != 0:
            raise ValueError("oracle_rplu_cauchy: invalid arguments")
        kd = int(kd[0])
        return dict(I=I[:kd].copy(), J=J[:kd].copy(), L=np.ascontiguousarray(L[:kd].T), U=U[:kd].copy(),
                    d=d[:n].copy(), T=T[:kd + 1].copy(), row_margin=rm[:kd].copy(), col_margin=cm[:kd].copy(),
                    k_done=kd)


    def rplu_cauchy_like(self, x, y, G, B, k: int, seed: int = 0, mode: str = "random", tol: float = 0.0,
                         given=None) -> dict:
        """RPLU of the Cauchy-like matrix A_pq = sum_l G[p,l] B[l,q] / (x_p - y_q)
        (G n x P, B P x m) through its generators, complex128.  Same outputs as
        rplu_dense plus G, B: the generators after the last step."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.complex128))
        G = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(len(x), -1))
        P_ = G.shape[1]
        B = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).reshape(P_, len(y)))
        n, m = len(x), len(y)
        I = np.zeros(max(k, 1), np.int64)
        J = np.zeros(max(k, 1), np.int64)
        L = np.zeros((max(k, 1), n), np.complex128)
        U = np.zeros((max(k, 1), m), np.complex128)
        T = np.zeros(k + 1)
        rm = np.zeros(max(k, 1))
        cm = np.zeros(max(k, 1))
        Go = np.zeros_like(G)
        Bo = np.zeros_like(B)
        kd = np.zeros(1, np.int64)
        gI, gJ = _given(given, k)
        rc = self.lib.oracle_rplu_cauchy_like(_ptr(x), _ptr(y), _ptr(G), _ptr(B), n, m, P_, k,
                                              ctypes.c_uint64(seed & (2**64 - 1)), MODES[mode], _ptr(gI), _ptr(gJ),
                                              tol, _ptr(I), _ptr(J), _ptr(L), _ptr(U), _ptr(T), _ptr(rm), _ptr(cm),
                                              _ptr(Go), _ptr(Bo), _ptr(kd))
        if rc != 0:
            raise ValueError("oracle_rplu_cauchy_like: invalid arguments")
        kd = int(kd[0])
        return dict(I=I[:kd].copy(), J=J[:kd].copy(), L=np.ascontiguousarray(L[:kd].T), U=U[:kd].copy(),
                    T=T[:kd + 1].copy(), row_margin=rm[:kd].copy(), col_margin=cm[:kd].copy(), G=Go, B=Bo,
                    k_done=kd)


    def bh_bounds(self, x, y, G, B, nu: float = 5.0, leaf: int = 64):
        """Row-norm upper bounds u (App. C) for the Cauchy-like matrix of (x, y, G, B)."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.complex128))
        G = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(len(x), -1))
        B = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).reshape(G.shape[1], len(y)))
        u = np.zeros(len(x))
        rc = self.lib.oracle_bh_bounds(_ptr(x), _ptr(y), _ptr(G), _ptr(B), len(x), len(y), G.shape[1], nu, leaf, None,
                                       _ptr(u))
        if rc != 0:
            raise ValueError("oracle_bh_bounds: invalid arguments")
        return u

    def rplu_cauchy_like_bh(self, x, y, G, B, k: int, seed: int = 0, nu: float = 5.0, leaf: int = 64,
                            tol: float = 0.0, mode: str = "random", stop: str = "sum") -> dict:
        """RPLU of the Cauchy-like matrix through its generators with Algorithm 3's
        row draw (rejection sampling against the App. C upper bounds); mode "c2":
        the approximate C2PLU with the same bounds (Sec. 5.1); stop "max": the
        CUR-AAA stopping rule max(u) <= tol^2 max(u at step 0) (Sec. 5.3)."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.complex128))
        G = np.ascontiguousarray(np.asarray(G, dtype=np.complex128).reshape(len(x), -1))
        P_ = G.shape[1]
        B = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).reshape(P_, len(y)))
        n, m = len(x), len(y)
        kk = max(k, 1)
        I = np.zeros(kk, np.int64)
        J = np.zeros(kk, np.int64)
        L = np.zeros((kk, n), np.complex128)
        U = np.zeros((kk, m), np.complex128)
        T = np.zeros(k + 1)
        rm, cm, am = np.zeros(kk), np.zeros(kk), np.zeros(kk)
        att = np.zeros(kk, np.int32)
        kd = np.zeros(1, np.int64)
        rc = self.lib.oracle_rplu_cauchy_like_bh(_ptr(x), _ptr(y), _ptr(G), _ptr(B), n, m, P_, k,
                                                 ctypes.c_uint64(seed & (2**64 - 1)), nu, leaf, tol,
                                                 {"random": 0, "c2": 1}[mode], {"sum": 0, "max": 1}[stop], _ptr(I), _ptr(J),
                                                 _ptr(L), _ptr(U), _ptr(T), _ptr(rm), _ptr(cm), _ptr(am), _ptr(att),
                                                 _ptr(kd))
        if rc != 0:
            raise ValueError("oracle_rplu_cauchy_like_bh: invalid arguments")
        kd = int(kd[0])
        return dict(I=I[:kd].copy(), J=J[:kd].copy(), L=np.ascontiguousarray(L[:kd].T), U=U[:kd].copy(),
                    T=T[:kd + 1].copy(), row_margin=rm[:kd].copy(), col_margin=cm[:kd].copy(),
                    acc_margin=am[:kd].copy(), attempts=att[:kd].copy(), k_done=kd)


def _default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def u01(seed: int, t: int, s: int, a: int = 0) -> float:
    return _default().u01(seed, t, s, a)


def inverse_cdf(w, target: float, total: float):
    return _default().inverse_cdf(w, target, total)


def rplu_dense(A, k: int, seed: int = 0, mode: str = "random", tol: float = 0.0, given=None) -> dict:
    return _default().rplu_dense(A, k, seed, mode, tol, given)


def rplu_cauchy_like(x, y, G, B, k: int, seed: int = 0, mode: str = "random", tol: float = 0.0,
                     given=None) -> dict:
    return _default().rplu_cauchy_like(x, y, G, B, k, seed, mode, tol, given)


def rplu_cauchy(x, y, k: int, seed: int = 0, mode: str = "random", tol: float = 0.0, given=None) -> dict:
    return _default().rplu_cauchy(x, y, k, seed, mode, tol, given)


def bh_bounds(x, y, G, B, nu: float = 5.0, leaf: int = 64):
    return _default().bh_bounds(x, y, G, B, nu, leaf)


def rplu_cauchy_like_bh(x, y, G, B, k: int, seed: int = 0, nu: float = 5.0, leaf: int = 64, tol: float = 0.0,
                        mode: str = "random", stop: str = "sum") -> dict:
    return _default().rplu_cauchy_like_bh(x, y, G, B, k, seed, nu, leaf, tol, mode, stop)
