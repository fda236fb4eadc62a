"""Python marshalling for rplu_batch and the batch plans (include/rplu.h):
many independent problems per call.  Jobs are dicts:
    {"kind": "dense", "A": 2-D array, "dtype": "f32"|"f64"|"c64"}
    {"kind": "cauchy", "x": 1-D array, "y": 1-D array, "dtype": ...}  (real points, or complex for "c64")
Arrays may be numpy (host; the library stages them) or CUDA torch tensors.
Outputs are allocated like the inputs (numpy or CUDA tensors).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Any

import numpy as np

from .binding import DTYPES, PIVOTS, Job, Opts, RPLUError, lib

_NP = {"f32": np.float32, "f64": np.float64, "c64": np.complex64}


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
            tdt = {"f32": torch.float32, "f64": torch.float64, "c64": torch.complex64}[dt]
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
        j.memory = 2 if dev else 1  # inputs and outputs on the same side
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


def _job_dtype():
    """The numpy structured dtype of a ctypes Job (pointer fields as uint64), built once."""
    global _JOB_DTYPE
    if _JOB_DTYPE is None:
        names, formats, offsets = [], [], []
        for name, ct in Job._fields_:
            names.append(name)
            formats.append(np.uint64 if ct is ctypes.c_void_p else np.dtype(ct))
            offsets.append(getattr(Job, name).offset)
        _JOB_DTYPE = np.dtype({"names": names, "formats": formats, "offsets": offsets,
                               "itemsize": ctypes.sizeof(Job)})
    return _JOB_DTYPE


_JOB_DTYPE = None


def _job_view(arr, n_jobs):
    """A numpy structured view of a ctypes Job array (pointer fields as uint64)."""
    raw = (ctypes.c_char * (ctypes.sizeof(Job) * n_jobs)).from_buffer(arr)
    return np.frombuffer(raw, dtype=_job_dtype(), count=n_jobs)


def _host_cauchy_uniform(specs):
    """The dtype when every job is a Cauchy job with host (numpy) points of
    one dtype and default per-job options, else None."""
    if not specs:
        return None
    dt = specs[0].get("dtype", "f64")
    for sp in specs:
        if sp["kind"] != "cauchy" or sp.get("dtype", "f64") != dt or "seed" in sp or "rel_tol" in sp:
            return None
        if _is_torch(sp["x"]) or _is_torch(sp["y"]):
            return None
    return dt


def _fill_host_cauchy(arr, specs, dt, rel_tol, seed, k_max):
    """_fill for host Cauchy jobs of one dtype, vectorized: the points are
    packed into one array per side, the outputs are slices of one packed array
    per factor, and the job table is written through a structured view."""
    npdt = _NP[dt]
    xs = [sp["x"] for sp in specs]
    ys = [sp["y"] for sp in specs]
    if not all(type(v) is np.ndarray and v.ndim == 1 for v in xs + ys):
        xs = [np.asarray(v, dtype=npdt).ravel() for v in xs]
        ys = [np.asarray(v, dtype=npdt).ravel() for v in ys]
    n = np.fromiter(map(len, xs), np.int64, len(xs))
    m = np.fromiter(map(len, ys), np.int64, len(ys))
    X = np.concatenate(xs).astype(npdt, copy=False)
    Y = np.concatenate(ys).astype(npdt, copy=False)
    return _fill_packed(arr, X, Y, n, m, dt, rel_tol, seed, k_max)


def _fill_packed(arr, X, Y, n, m, dt, rel_tol, seed, k_max, out=None):
    """The job table of Cauchy jobs whose points are consecutive ranges of X
    and Y (job b: n[b] points of X, m[b] of Y), outputs in packed arrays:
    new ones, or those of `out` (a PackedResults of the same n, m, k_max and
    dtype), which the call then overwrites."""
    npdt = _NP[dt]
    n_jobs = len(n)
    k = np.minimum(n, m) if k_max is None else np.minimum(np.minimum(n, m), int(k_max))
    kk = np.maximum(k, 1)
    w = np.dtype(npdt).itemsize
    ox = np.concatenate(([0], np.cumsum(n)[:-1]))
    oy = np.concatenate(([0], np.cumsum(m)[:-1]))
    if out is not None:
        I, J, L, U, n0, m0, oi, oL, oU, k0 = out._packed
        if L.dtype != npdt or not (np.array_equal(n0, n) and np.array_equal(m0, m) and np.array_equal(k0, k)):
            raise ValueError("out holds the outputs of jobs of other sizes, k_max or dtype")
    else:
        oi = np.concatenate(([0], np.cumsum(kk)[:-1]))
        oL = np.concatenate(([0], np.cumsum(kk * n)[:-1]))
        oU = np.concatenate(([0], np.cumsum(kk * m)[:-1]))
        I = np.empty(int(kk.sum()), np.int64)
        J = np.empty(int(kk.sum()), np.int64)
        L = np.empty(int((kk * n).sum()), npdt)
        U = np.empty(int((kk * m).sum()), npdt)
    v = _job_view(arr, n_jobs)
    v["kind"] = 1
    # every buffer is host memory; reused outputs (pages already resident) are written in place by the
    # device where it reaches pageable host memory, fresh ones come through the pinned staging (the
    # device's first touch of a page is an operating-system fault)
    v["memory"] = 3 if out is not None else 1
    v["dtype"] = DTYPES[dt]
    v["n"], v["m"], v["k_max"] = n, m, k
    v["rel_tol"] = rel_tol
    b = np.arange(n_jobs, dtype=np.uint64)
    v["seed"] = (np.uint64(int(seed) & (2**64 - 1)) + np.uint64(0x9E3779B97F4A7C15) * (b + np.uint64(1)))
    v["x"] = np.uint64(X.ctypes.data) + (ox * w).astype(np.uint64)
    v["y"] = np.uint64(Y.ctypes.data) + (oy * w).astype(np.uint64)
    v["I"] = np.uint64(I.ctypes.data) + (oi * 8).astype(np.uint64)
    v["J"] = np.uint64(J.ctypes.data) + (oi * 8).astype(np.uint64)
    v["L"] = np.uint64(L.ctypes.data) + (oL * w).astype(np.uint64)
    v["U"] = np.uint64(U.ctypes.data) + (oU * w).astype(np.uint64)
    return [X, Y], (I, J, L, U, n, m, oi, oL, oU, k)


def rplu_batch_cauchy_packed(x, y, n, m, dtype: str = "f32", rel_tol: float = 1e-6, seed: int = 0,
                             pivot: str = "random", k_max=None, stream=None, out=None):
    """Cauchy jobs given as consecutive ranges of two host point arrays, as a
    hierarchical matrix stores its blocks: job b factors 1/(x_p - y_q) over
    the next n[b] points of x and the next m[b] points of y.  One call of
    rplu_batch; job b's seed is job_seed(seed, b).  Returns PackedResults.

    out: the PackedResults of an earlier call with the same n, m, k_max and
    dtype; this call writes its factors into that call's arrays (whose views
    then show the new factors) instead of allocating new ones.  In a loop
    this saves the first touch of fresh capacity-sized arrays (each job's L
    and U regions are sized for min(n, m) columns) and their release, and on
    a device that accesses pageable host memory in place the points are
    gathered and the factors written by the device itself (job memory hint
    3), without the pinned staging copies."""
    npdt = _NP[dtype]
    X = np.ascontiguousarray(x, dtype=npdt).ravel()
    Y = np.ascontiguousarray(y, dtype=npdt).ravel()
    n = np.asarray(n, dtype=np.int64)
    m = np.asarray(m, dtype=np.int64)
    if n.shape != m.shape or n.ndim != 1 or int(n.sum()) != X.size or int(m.sum()) != Y.size:
        raise ValueError("n and m must be 1-D, of one length, summing to the sizes of x and y")
    n_jobs = len(n)
    arr = (Job * max(n_jobs, 1))()
    o = _opts(pivot, stream)
    if out is not None and not isinstance(out, PackedResults):
        raise TypeError("out must be the PackedResults of an earlier call")
    keep, packed = _fill_packed(arr, X, Y, n, m, dtype, rel_tol, seed, k_max, out)
    lib.rplu_batch(arr, n_jobs, ctypes.byref(o))
    return PackedResults(arr, packed, n_jobs)


class PackedResults:
    """The per-job results of a vectorized host call: a sequence of JobResult
    whose entries are views into the packed output arrays, made when indexed
    (a batch of thousands of jobs returns without building them all)."""

    def __init__(self, arr, packed, n_jobs):
        self._packed = packed
        v = _job_view(arr, n_jobs)
        self.k_done = v["k_done"].copy()
        self.status = v["status"].copy()
        self.rel_res = v["rel_res"].copy()
        self._n = n_jobs

    def __len__(self):
        return self._n

    def __getitem__(self, b):
        if isinstance(b, slice):
            return [self[q] for q in range(*b.indices(self._n))]
        if b < 0:
            b += self._n
        if not 0 <= b < self._n:
            raise IndexError(b)
        I, J, L, U, n, m, oi, oL, oU, _ = self._packed
        k, nb, mb, i0, l0, u0 = int(self.k_done[b]), int(n[b]), int(m[b]), int(oi[b]), int(oL[b]), int(oU[b])
        return JobResult(I[i0:i0 + k], J[i0:i0 + k], L[l0:l0 + k * nb].reshape(k, nb).T,
                         U[u0:u0 + k * mb].reshape(k, mb), k, int(self.status[b]), float(self.rel_res[b]))

    def __iter__(self):
        return (self[b] for b in range(self._n))


def rplu_batch(specs, rel_tol: float = 1e-6, seed: int = 0, pivot: str = "random", k_max=None, stream=None):
    """One call of rplu_batch over all jobs; returns one JobResult per job.
    Host Cauchy jobs of one dtype take a vectorized path whose results
    (a PackedResults sequence) are views into packed arrays (L as an
    n x k_done view, U k_done x m)."""
    n_jobs = len(specs)
    arr = (Job * max(n_jobs, 1))()
    o = _opts(pivot, stream)
    dt = _host_cauchy_uniform(specs)
    if dt is not None:
        keep, packed = _fill_host_cauchy(arr, specs, dt, rel_tol, seed, k_max)
        lib.rplu_batch(arr, n_jobs, ctypes.byref(o))
        return PackedResults(arr, packed, n_jobs)
    keep, outs = _fill(arr, specs, rel_tol, seed, k_max)
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
