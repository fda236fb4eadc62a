"""Python marshalling for rplu_batch (include/rplu.h): many independent
problems in one call.  Jobs are dicts:
    {"kind": "dense", "A": 2-D array, "dtype": "f32"|"f64"}
    {"kind": "cauchy", "x": 1-D real array, "y": 1-D real array, "dtype": ...}
Inputs and outputs are host (numpy) buffers; the library stages them.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from .binding import DTYPES, PIVOTS, Job, Opts, lib

_NP = {"f32": np.float32, "f64": np.float64}


def job_seed(base: int, b: int) -> int:
    """Seed of job b in a batch drawn from one base seed."""
    return (int(base) + 0x9E3779B97F4A7C15 * (b + 1)) & (2**64 - 1)


@dataclass
class JobResult:
    I: np.ndarray
    J: np.ndarray
    L: np.ndarray
    U: np.ndarray
    k_done: int
    status: int
    rel_res: float


def rplu_batch(specs, rel_tol: float = 1e-6, seed: int = 0, pivot: str = "random", k_max=None, stream=None):
    n_jobs = len(specs)
    arr = (Job * max(n_jobs, 1))()
    keep = []
    outs = []
    for b, sp in enumerate(specs):
        dt = sp.get("dtype", "f64")
        npdt = _NP[dt]
        j = arr[b]
        if sp["kind"] == "dense":
            A = np.ascontiguousarray(sp["A"], dtype=npdt)
            n, m = A.shape
            j.kind = 0
            j.A = A.ctypes.data
            j.lda = m
            keep.append(A)
        else:
            x = np.ascontiguousarray(sp["x"], dtype=npdt)
            y = np.ascontiguousarray(sp["y"], dtype=npdt)
            n, m = len(x), len(y)
            j.kind = 1
            j.x = x.ctypes.data
            j.y = y.ctypes.data
            keep += [x, y]
        k = min(n, m) if k_max is None else min(k_max, n, m)
        j.dtype = DTYPES[dt]
        j.n, j.m, j.k_max = n, m, k
        j.rel_tol = rel_tol
        j.seed = job_seed(seed, b)
        I = np.full(max(k, 1), -1, np.int64)
        J = np.full(max(k, 1), -1, np.int64)
        L = np.zeros((max(k, 1), n), npdt)
        U = np.zeros((max(k, 1), m), npdt)
        j.I, j.J, j.L, j.U = I.ctypes.data, J.ctypes.data, L.ctypes.data, U.ctypes.data
        outs.append((I, J, L, U))
    o = Opts()
    lib.rplu_opts_init(ctypes.byref(o))
    o.pivot = PIVOTS[pivot]
    o.stream = stream
    lib.rplu_batch(arr, n_jobs, ctypes.byref(o))
    res = []
    for b in range(n_jobs):
        I, J, L, U = outs[b]
        kd = int(arr[b].k_done)
        res.append(JobResult(I[:kd].copy(), J[:kd].copy(), np.ascontiguousarray(L[:kd].T), U[:kd].copy(), kd,
                             int(arr[b].status), float(arr[b].rel_res)))
    return res
