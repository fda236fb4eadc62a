"""Python marshalling for rplu_batch and the batch plans (include/rplu.h):
many independent problems per call.  Jobs are dicts:
    {"kind": "dense", "A": 2-D array, "dtype": "f32"|"f64"}
    {"kind": "cauchy", "x": 1-D real array, "y": 1-D real array, "dtype": ...}
Arrays may be numpy (host; the library stages them) or CUDA torch tensors.
Outputs are allocated like the inputs (numpy or CUDA tensors).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Any

import numpy as np

from .binding import DTYPES, PIVOTS, Job, Opts, RPLUError, lib

_NP = {"f32": np.float32, "f64": np.float64}


def job_seed(base: int, b: int) -> int:
    """Seed of job b in a batch drawn from one base seed."""
    return (int(base) + 0x9E3779B97F4A7C15 * (b + 1)) & (2**64 - 1)


@dataclass
class JobResult:
    I: Any
    J: Any
    L: Any          # n x k_done
    U: Any          # k_done x m
    k_done: int
    status: int
    rel_res: float


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _fill(arr, specs, rel_tol, seed, k_max):
    """Fill the Job array; returns (keep-alive list, per-job output buffers)."""
    keep, outs = [], []
    for b, sp in enumerate(specs):
        dt = sp.get("dtype", "f64")
        j = arr[b]
        src = sp["A"] if sp["kind"] == "dense" else sp["x"]
        dev = _is_torch(src) and src.is_cuda
        if dev:
            import torch
            tdt = torch.float32 if dt == "f32" else torch.float64
            if sp["kind"] == "dense":
                A = sp["A"].to(tdt).contiguous()
                n, m = A.shape
                j.kind, j.A, j.lda = 0, A.data_ptr(), m
                keep.append(A)
            else:
                x = sp["x"].to(tdt).contiguous()
                y = sp["y"].to(tdt).contiguous()
                n, m = x.numel(), y.numel()
                j.kind, j.x, j.y = 1, x.data_ptr(), y.data_ptr()
                keep += [x, y]
            k = min(n, m) if k_max is None else min(k_max, n, m)
            kk = max(k, 1)
            I = torch.full((kk,), -1, dtype=torch.int64, device=src.device)
            J = torch.full((kk,), -1, dtype=torch.int64, device=src.device)
            L = torch.zeros((kk, n), dtype=tdt, device=src.device)
            U = torch.zeros((kk, m), dtype=tdt, device=src.device)
            j.I, j.J, j.L, j.U = I.data_ptr(), J.data_ptr(), L.data_ptr(), U.data_ptr()
        else:
            npdt = _NP[dt]
            if sp["kind"] == "dense":
                A = np.ascontiguousarray(sp["A"], dtype=npdt)
                n, m = A.shape
                j.kind, j.A, j.lda = 0, A.ctypes.data, m
                keep.append(A)
            else:
                x = np.ascontiguousarray(sp["x"], dtype=npdt)
                y = np.ascontiguousarray(sp["y"], dtype=npdt)
                n, m = len(x), len(y)
                j.kind, j.x, j.y = 1, x.ctypes.data, y.ctypes.data
                keep += [x, y]
            k = min(n, m) if k_max is None else min(k_max, n, m)
            kk = max(k, 1)
            I = np.full(kk, -1, np.int64)
            J = np.full(kk, -1, np.int64)
            L = np.zeros((kk, n), npdt)
            U = np.zeros((kk, m), npdt)
            j.I, j.J, j.L, j.U = I.ctypes.data, J.ctypes.data, L.ctypes.data, U.ctypes.data
        j.dtype = DTYPES[dt]
        j.n, j.m, j.k_max = n, m, k
        j.rel_tol = sp.get("rel_tol", rel_tol)
        j.seed = sp.get("seed", job_seed(seed, b))
        outs.append((I, J, L, U))
    return keep, outs


def _results(arr, outs):
    res = []
    for b, (I, J, L, U) in enumerate(outs):
        kd = int(arr[b].k_done)
        if _is_torch(L):
            r = JobResult(I[:kd].clone(), J[:kd].clone(), L[:kd].t().contiguous(), U[:kd].clone(), kd,
                          int(arr[b].status), float(arr[b].rel_res))
        else:
            r = JobResult(I[:kd].copy(), J[:kd].copy(), np.ascontiguousarray(L[:kd].T), U[:kd].copy(), kd,
                          int(arr[b].status), float(arr[b].rel_res))
        res.append(r)
    return res


def _opts(pivot, stream):
    o = Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.pivot = PIVOTS[pivot]
    o.stream = stream
    return o


def rplu_batch(specs, rel_tol: float = 1e-6, seed: int = 0, pivot: str = "random", k_max=None, stream=None):
    """One call of rplu_batch over all jobs; returns one JobResult per job."""
    n_jobs = len(specs)
    arr = (Job * max(n_jobs, 1))()
    keep, outs = _fill(arr, specs, rel_tol, seed, k_max)
    o = _opts(pivot, stream)
    lib.rplu_batch(arr, n_jobs, ctypes.byref(o))
    return _results(arr, outs)


class BatchPlan:
    """A captured, replayable batch (rplu_batch_plan_*).  All job arrays must be
    CUDA tensors.  run() enqueues one replay on `stream` (a cudaStream_t
    handle, e.g. torch.cuda.current_stream().cuda_stream); wait() blocks and
    returns the worst status; results() returns the per-job factors."""

    def __init__(self, specs, rel_tol: float = 1e-6, seed: int = 0, pivot: str = "random", k_max=None,
                 tune: bool = False):
        self.n_jobs = len(specs)
        self.arr = (Job * max(self.n_jobs, 1))()
        self._keep, self.outs = _fill(self.arr, specs, rel_tol, seed, k_max)
        o = _opts(pivot, None)
        h = ctypes.c_void_p()
        st = lib.rplu_batch_plan_create(self.arr, self.n_jobs, ctypes.byref(o), int(bool(tune)), ctypes.byref(h))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        self.h = h

    def run(self, stream=None):
        st = lib.rplu_batch_plan_run(self.h, stream)
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())

    def wait(self) -> int:
        return int(lib.rplu_batch_plan_wait(self.h))

    def results(self):
        return _results(self.arr, self.outs)

    def shape(self):
        s = (ctypes.c_int32 * 4)()
        ms = ctypes.c_double()
        st = lib.rplu_batch_plan_shape(self.h, s, ctypes.byref(ms))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        return {"threads": s[0], "tile_rows": s[1], "write_back": s[2], "ctas_per_sm": s[3],
                "tuned_ms": ms.value}

    def close(self):
        if getattr(self, "h", None):
            lib.rplu_batch_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
