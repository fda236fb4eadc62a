"""Python marshalling for serving sessions (rplu_session_*, include/rplu.h).

Requests are dicts like the batch jobs, served in FP32 or (complex inputs) complex64:
    {"kind": "dense", "A": 2-D array}  or  {"kind": "cauchy", "x": 1-D, "y": 1-D}
with optional "rel_tol", "k_max" and "seed".  Arrays may be CUDA torch tensors
or numpy arrays; the session keeps a reference until the request is fetched,
so the buffers stay valid while it is queued.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from .binding import Request, RPLUError, SessionOpts, TicketInfo, lib

QUEUED, RUNNING, DONE, CANCELLED = range(4)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    return a.data_ptr() if _is_torch(a) else a.ctypes.data


def _is_complex(a):
    return a.is_complex() if _is_torch(a) else np.iscomplexobj(a)


def _as(a, complex_):
    """The request's array in its served type: complex64 or float32."""
    if _is_torch(a):
        import torch
        return a.to(torch.complex64 if complex_ else torch.float32).contiguous()
    return np.ascontiguousarray(a, dtype=np.complex64 if complex_ else np.float32)


@dataclass
class Info:
    state: int
    status: int
    k_done: int
    rel_res: float
    latency_ms: float
    queue_ms: float


class Session:
    """A serving session (rplu_session_opts in include/rplu.h): hbm_budget
    device bytes (0: 80% of free memory); the persistent kernel takes dense
    requests up to max_dim (and dense_kernel_cells entries) and Cauchy ones up
    to cauchy_max_dim (0: 4096); larger ones run on large_streams streams,
    their Cauchy rows drawn by Algorithm 3 against Barnes-Hut bounds when
    bound_nu >= 1 (else exact norms); idle kernel CTAs exit after idle_us."""

    def __init__(self, hbm_budget: int = 0, max_jobs: int = 4096, max_dim: int = 2048, idle_us: float = 1000.0,
                 pivot: str = "random", large_streams: int = 8, dense_kernel_cells: int = 0,
                 cauchy_max_dim: int = 0, bound_nu: float = 0.0):
        o = SessionOpts()
        lib.rplu_session_opts_init(ctypes.byref(o))
        o.hbm_budget, o.max_jobs, o.max_dim, o.idle_us = int(hbm_budget), int(max_jobs), int(max_dim), float(idle_us)
        o.large_streams = int(large_streams)
        o.dense_kernel_cells = int(dense_kernel_cells)
        o.cauchy_max_dim = int(cauchy_max_dim)
        o.bound_nu = float(bound_nu)
        o.pivot = {"random": 0, "c2": 1}[pivot]
        h = ctypes.c_void_p()
        st = lib.rplu_session_create(ctypes.byref(o), ctypes.byref(h))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        self.h = h
        self._keep = {}
        self._shape = {}

    def submit(self, spec, rel_tol: float = 1e-6, seed: int = 0, k_max=None) -> int:
        r = Request()
        keep = []
        if spec["kind"] == "dense":
            cplx = _is_complex(spec["A"])
            A = _as(spec["A"], cplx)
            n, m = A.shape
            r.kind, r.A, r.lda = 0, _ptr(A), m
            keep.append(A)
        else:
            cplx = _is_complex(spec["x"]) or _is_complex(spec["y"])
            x, y = _as(spec["x"], cplx), _as(spec["y"], cplx)
            n, m = int(x.shape[0]), int(y.shape[0])
            r.kind, r.x, r.y = 1, _ptr(x), _ptr(y)
            keep += [x, y]
        k = spec.get("k_max", k_max)
        r.dtype = 2 if cplx else 0
        r.n, r.m = n, m
        r.k_max = min(n, m) if k is None else min(int(k), n, m)
        r.rel_tol = float(spec.get("rel_tol", rel_tol))
        r.seed = int(spec.get("seed", seed)) & (2**64 - 1)
        t = ctypes.c_int64()
        st = lib.rplu_session_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        self._keep[t.value] = keep
        self._shape[t.value] = (n, m, int(r.k_max), bool(keep and _is_torch(keep[0])), cplx)
        return t.value

    def poll(self, ticket: int) -> Info:
        i = TicketInfo()
        st = lib.rplu_session_poll(self.h, ticket, ctypes.byref(i))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        return Info(i.state, i.status, i.k_done, i.rel_res, i.latency_ms, i.queue_ms)

    def wait(self, ticket: int, timeout_s: float = 0.0) -> Info:
        i = TicketInfo()
        st = lib.rplu_session_wait(self.h, ticket, float(timeout_s), ctypes.byref(i))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        return Info(i.state, i.status, i.k_done, i.rel_res, i.latency_ms, i.queue_ms)

    def cancel(self, ticket: int):
        st = lib.rplu_session_cancel(self.h, ticket)
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())

    def fetch(self, ticket: int):
        """(I, J, L n x k_done, U k_done x m) as numpy arrays, or CUDA tensors for
        CUDA inputs; releases the ticket."""
        info = self.poll(ticket)
        n, m, k, dev, cplx = self._shape[ticket]
        kd = max(info.k_done, 0)
        if dev:
            import torch
            tdt = torch.complex64 if cplx else torch.float32
            I = torch.empty(max(kd, 1), dtype=torch.int64, device="cuda")
            J = torch.empty_like(I)
            L = torch.empty((max(kd, 1), n), dtype=tdt, device="cuda")
            U = torch.empty((max(kd, 1), m), dtype=tdt, device="cuda")
            torch.cuda.synchronize()
        else:
            ndt = np.complex64 if cplx else np.float32
            I = np.empty(max(kd, 1), np.int64)
            J = np.empty(max(kd, 1), np.int64)
            L = np.empty((max(kd, 1), n), ndt)
            U = np.empty((max(kd, 1), m), ndt)
        st = lib.rplu_session_fetch(self.h, ticket, _ptr(I), _ptr(J), _ptr(L), _ptr(U))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        self._keep.pop(ticket, None)
        self._shape.pop(ticket, None)
        if dev:
            return I[:kd], J[:kd], L[:kd].t().contiguous(), U[:kd]
        return I[:kd], J[:kd], np.ascontiguousarray(L[:kd].T), U[:kd]

    def release(self, ticket: int):
        """Free a finished ticket's factors without copying them."""
        st = lib.rplu_session_fetch(self.h, ticket, None, None, None, None)
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        self._keep.pop(ticket, None)
        self._shape.pop(ticket, None)

    def completed(self, max_n: int = 1024):
        """[(ticket, Info)] finished since the last call, oldest first."""
        ts = (ctypes.c_int64 * max_n)()
        infos = (TicketInfo * max_n)()
        c = ctypes.c_int32()
        st = lib.rplu_session_completed(self.h, ts, infos, max_n, ctypes.byref(c))
        if st != 0:
            raise RPLUError(st, lib.rplu_last_error().decode())
        return [(int(ts[q]), Info(infos[q].state, infos[q].status, infos[q].k_done, infos[q].rel_res,
                                  infos[q].latency_ms, infos[q].queue_ms)) for q in range(c.value)]

    def stats(self) -> dict:
        out = (ctypes.c_double * 8)()
        lib.rplu_session_stats(self.h, out)
        keys = ["completed", "queued", "running", "arena_used", "arena_bytes", "kernel_launches",
                "large_completed", "cancelled"]
        return dict(zip(keys, [float(v) for v in out]))

    def close(self):
        if getattr(self, "h", None):
            lib.rplu_session_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
