"""Benchmark of the RPLU hot path on GB300.

One step = one pass of the whole hot path over one batch of synthetic input:
  * one dense-form factorization (rplu_dense): A = Q1 diag(sigma) Q2^T,
    32768 x 32768 FP32 in HBM (Q1, Q2 products of 64 Householder reflectors,
    sigma_i = (1+i)^-2), rank k = 256, FP32 Schur update with FP64 row norms,
    sampling and pivot division;
  * one matrix-free factorization (rplu_cauchy) of the complex Cauchy matrix
    A_ij = 1/(x_i - y_j), n = m = 20000, x on two interleaved Archimedean
    spirals plus a 20% Gaussian cluster, y the same recipe rotated by pi/2 and
    shifted by 3; complex64, rank k = 100.
value = factorizations per second (2 per step per GPU), inputs resident in HBM.
e2e   = the same through the same API with pinned HOST inputs and outputs, the
        host<->device copies inside the timed region.
cauchy_like = (extra object) the step's Cauchy matrix factored through its
        generators with exact row norms (rplu_cauchy_like).
cauchy_cur = (extra object) the step's Cauchy matrix in CUR form (Algorithm
        2 as printed: no L, U; pivot rows/columns generated again, core inverse
        by block inversion), with its explicit error.
cauchy_like_bounds = (extra object) Algorithm 3 with rejection-sampled rows
        against the App. C bounds on the Loewner matrices of Sec. 5.2, rank
        1000: ms per factorization, the bounds kernel's FP64 roofline, the
        oracle on a sample of steps.
cur_aaa = (extra object) CUR-AAA rational approximation (Sec. 5.3) of
        tan(20 z^20) from 200 000 samples on the unit disk, eps = 1e-11,
        RPLU and C2PLU pivots: seconds, support size, errors.
batch = (extra object of the same line) 4096 real Cauchy blocks, n, m ~
        U{64..1024}, factored to 1e-6 relative error in one persistent launch
        replayed from a captured CUDA graph; its own roofline (generated
        entries vs the MUFU reciprocal rate), the same jobs one FP64 call each
        for comparison, and rplu_batch end to end from host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank factors its own problems (independent seeds): weak
scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "RPLU factorizations/s at stated rel. error; Schur-pass GB/s vs HBM; p99 latency"
DENSE_N, DENSE_K = 32768, 256
CAUCHY_N, CAUCHY_K = 20000, 100
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
PASS_BLOCK_F32 = 6  # the library's default write-back interval for FP32 data
BATCH_JOBS, BATCH_TOL = 4096, 1e-6
BATCH_FP64_SAMPLE = 256  # jobs run one per call in FP64 for the comparison
BATCH_E2E_CALLS = 3  # timed end-to-end batch calls (after one untimed call)
SERVE_LARGE_POOL, SERVE_LARGE_RANGE, SERVE_BOUND_NU = 4, (8192, 20000), 5.0  # large Cauchy serving requests
# MUFU reciprocal throughput per SM per clock (the XU pipe): measured on this
# GPU model with a chain of rcp.approx.f32 (15.8 per SM per clock at 2.0 GHz),
# the documented rate of 16 for 32-bit reciprocals.
RCP_PER_SM_PER_CLK = 16

# DRAM bytes (read + write) per k_dense_pass_tma launch, mean over one full
# write-back block of the 32768^2 workload, from the ncu capture summarised in
# profiles/dense_pass_32768_dram.md; reported only while csrc/dense.cu and
# csrc/common.cuh (the kernel and the default write-back interval) still have
# the hash they were taken with.
DENSE_UPDATE_TRAFFIC = 5006563499
DENSE_UPDATE_SRC_SHA = "b8030f59b0bcabe6"


# ------------------------------------------------------------------ helpers

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_scalar(x: float, op: str) -> float:
    """max/sum of a scalar over ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dense_pass_bytes(n: int, m: int, k: int, w: int, blk: int) -> float:
    """HBM bytes the per-step dense passes must move over a factorization:
    one read of the unpivoted rows per step, one write-back per block."""
    tot = 0.0
    for t in range(k):
        rows = n - t - 1
        write = (t % blk == blk - 1) and (t + 1 < k)
        tot += rows * m * w * (2.0 if write else 1.0)
    return tot


def src_sha(*names: str) -> str:
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2601_22344_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.out is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.out.flush()
        with open(self.out.name) as f:
            rows = [r.strip().split(", ") for r in f if r.strip()]
        os.unlink(self.out.name)
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                pw.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons)}


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2601_22344_gb300 as rp

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    dn, dk = args.dense_n, args.dense_k
    cn, ck = args.cauchy_n, args.cauchy_k
    # inputs (seeded per rank: independent problems)
    F = W.dense_householder_inverse_square(dn, seed=W.derive_seed(3, rank))
    A = F.to_torch(dev, torch.float32)
    x, y = W.cauchy_spirals_square(cn, seed=W.derive_seed(2, rank))
    xd = torch.from_numpy(x.astype(np.complex64)).to(dev)
    yd = torch.from_numpy(y.astype(np.complex64)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def step(s, prof_d=None, prof_c=None, dense_in=A, xin=xd, yin=yd):
        rd = rp.rplu_dense(dense_in, dk, seed=1000 + s, prof=prof_d)
        rc = rp.rplu_cauchy(xin, yin, ck, seed=2000 + s, prof=prof_c)
        return rd, rc

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()

    prof_d = np.zeros(4)
    prof_c = np.zeros(4)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    barrier()
    torch.cuda.synchronize()
    last = None
    with ClockSampler(gpu_uuid) as clk:
        for s in range(args.steps):
            flush.fill_(float(s))  # write more than L2 between timed steps
            ev[s][0].record()
            rd = rp.rplu_dense(A, dk, seed=1000 + s, prof=prof_d)
            ev[s][1].record()
            rc = rp.rplu_cauchy(xd, yd, ck, seed=2000 + s, prof=prof_c)
            ev[s][2].record()
            last = (rd, rc)
        torch.cuda.synchronize()
    barrier()
    clocks = clk.summary()
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    dense_call_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    cauchy_call_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    local_s = sum(step_ms) / 1e3
    total_s = reduce_scalar(local_s, "max")
    units = reduce_scalar(2.0 * args.steps, "sum")
    value = units / total_s

    # end to end: pinned host inputs and outputs, copies inside the timed region
    A_h = torch.empty(A.shape, dtype=A.dtype, pin_memory=True)
    A_h.copy_(A)
    x_h = torch.empty(xd.shape, dtype=xd.dtype, pin_memory=True)
    y_h = torch.empty(yd.shape, dtype=yd.dtype, pin_memory=True)
    x_h.copy_(xd)
    y_h.copy_(yd)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        step(s, dense_in=A_h, xin=x_h, yin=y_h)
    torch.cuda.synchronize()
    e2e_local = time.perf_counter() - t0
    barrier()
    e2e_s = reduce_scalar(e2e_local, "max")
    e2e_units = reduce_scalar(2.0 * e2e_steps, "sum")
    h2d = A.numel() * 4 + (cn + cn) * 8
    d2h = (dn * dk + dk * dn) * 4 + 2 * dk * 8 + (cn * ck + ck * cn) * 8 + 2 * ck * 8

    # accuracy of the last timed step (outside the timed region)
    rd, rc = last
    dense_rel = math.sqrt(rd.T[-1] / rd.T[0])
    with torch.no_grad():
        xc = xd.to(torch.complex128)
        yc = yd.to(torch.complex128)
        Ac = 1.0 / (xc[:, None] - yc[None, :])
        Rc = Ac - rc.L.to(torch.complex128) @ rc.U.to(torch.complex128)
        cauchy_rel = float(torch.linalg.norm(Rc) / torch.linalg.norm(Ac))
        del Ac, Rc
    cauchy_est = math.sqrt(max(rc.T[-1], 0.0) / rc.T[0])

    # roofline of the dominant kernel: the fused dense Schur pass
    peak, peak_kind = measured_peaks()
    launches = prof_d[1]
    avg_s = prof_d[0] / 1e3 / max(launches, 1)
    # algorithmic bytes per launch: at step t the pass reads every row not yet
    # pivoted ((n - t - 1) rows of m FP32 entries) and writes them back when a
    # block of PASS_BLOCK steps ends (not after the last step); averaged over t < k
    alg_bytes = dense_pass_bytes(dn, dn, dk, 4, PASS_BLOCK_F32) / dk
    achieved = alg_bytes / avg_s / 1e9
    traffic = DENSE_UPDATE_TRAFFIC if DENSE_UPDATE_SRC_SHA == src_sha("dense.cu", "common.cuh") else None
    dense_ms = prof_d[0] / max(prof_d[3], 1)
    mv_ms = prof_c[0] / max(prof_c[3], 1)

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "factorizations/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            **workload_config(args, ws),
            "dense": {"n": dn, "m": dn, "k": dk, "dtype": "f32", "rel_error": dense_rel,
                      "rel_error_kind": "exact ||A-LU||_F/||A||_F (row norms recomputed from S)"},
            "cauchy": {"n": cn, "m": cn, "k": ck, "dtype": "c64", "rel_error": cauchy_rel,
                       "rel_error_estimate": cauchy_est, "rel_error_kind": "explicit, FP64, after the run"},
            "l2": "dense: 4.3 GB operand (> L2); a 256 MB buffer is written between timed steps",
            "step_ms": {"dense_call": dense_call_ms, "dense_update_kernels": dense_ms,
                        "cauchy_call": cauchy_call_ms, "cauchy_matvec_kernels": mv_ms},
        },
        "roofline": {"bound": "hbm", "kernel": "k_dense_pass_tma (fused Schur pass + row norms)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": traffic,
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_s * 1e3},
        "e2e": {"value": e2e_units / e2e_s, "unit": "factorizations/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(prof_d[2] + prof_c[2]),
        "clocks": clocks,
    }
    out["cauchy_roofline"] = _section(cauchy_matvec_roofline, prof_c, cn, cn, clocks.get("sm_mhz"),
                                      torch.cuda.get_device_properties(dev).multi_processor_count)
    out["configs"] = _section(run_precision_configs, args, dev, A, F, xd, yd, rd, rc)
    if isinstance(out["configs"], dict) and "dense_f64_path_32768" in out["configs"]:
        out["configs"]["dense_f64_path_32768"]["fp32_update_ms"] = dense_call_ms
        out["config"]["dense"]["rel_error_explicit"] = out["configs"]["dense_f64_path_32768"]["fp32_update_rel_error"]
    if args.workload == "all":
        out["cauchy_like"] = _section(run_cauchy_like, args, dev, xd, yd, ck, clocks.get("sm_mhz"))
        out["cauchy_cur"] = _section(run_cauchy_cur, args, dev, xd, yd, ck)
    if args.bh_cases > 0 and args.workload == "all":
        out["cauchy_like_bounds"] = _section(run_bh, args, dev, clocks.get("sm_mhz"), with_oracle=rank == 0 and ws == 1)
    if args.aaa_m > 0 and args.workload == "all":
        out["cur_aaa"] = _section(run_aaa, args, dev)
    if args.batch_jobs > 0 and args.workload == "all":
        out["batch"] = _section(run_batch, args, dev, rank, gpu_uuid)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(A, xd, yd, dk, ck)
    if args.serve_seconds > 0 and args.workload == "all":
        out["serving"] = _section(run_serving, args, dev, rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ------------------------------------------------------- the other configs

def dense_explicit_error(A, L, U, block_rows=2048):
    """||A - L U||_F / ||A||_F in FP64 over row blocks of the device operand
    (outside any timed region)."""
    import torch
    num = den = 0.0
    U64 = U.to(torch.float64) if not U.is_complex() else U.to(torch.complex128)
    for r0 in range(0, A.shape[0], block_rows):
        a = A[r0:r0 + block_rows]
        a = a.to(torch.complex128) if a.is_complex() else a.to(torch.float64)
        lb = L[r0:r0 + block_rows]
        lb = lb.to(torch.complex128) if lb.is_complex() else lb.to(torch.float64)
        num += float(torch.linalg.norm(a - lb @ U64) ** 2)
        den += float(torch.linalg.norm(a) ** 2)
    return math.sqrt(num / den) if den > 0 else 0.0


def cauchy_explicit_error(xd, yd, L, U, block_rows=4096):
    """||A - L U||_F / ||A||_F in FP64/complex128 for A_ij = 1/(x_i - y_j)."""
    import torch
    xc, yc = xd.to(torch.complex128), yd.to(torch.complex128)
    U64 = U.to(torch.complex128)
    num = den = 0.0
    for r0 in range(0, xc.shape[0], block_rows):
        a = 1.0 / (xc[r0:r0 + block_rows, None] - yc[None, :])
        num += float(torch.linalg.norm(a - L[r0:r0 + block_rows].to(torch.complex128) @ U64) ** 2)
        den += float(torch.linalg.norm(a) ** 2)
    return math.sqrt(num / den) if den > 0 else 0.0


def _timed_calls(fn, reps):
    """Mean milliseconds of `reps` calls (CUDA events around each, current
    stream), after one untimed call; the last call's result."""
    import torch
    r = fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms), statistics.median(ms), r


def run_precision_configs(args, dev, A32, F, xd, yd, rd32, rc64):
    """The configurations beside the headline pair, each with its explicit
    error: the dense FP64 500 x 400 problem at k = 40 (latency-bound: us per
    step), the spiral Cauchy matrix in complex128 beside the step's complex64,
    and the 32768^2 dense matrix through the FP64 path beside the step's FP32
    update (FP32 Schur update with FP64 row norms, sampling and division)."""
    import torch

    import paper_2601_22344_gb300 as rp

    out = {}
    # dense FP64 500 x 400, sigma_i = 0.8^i, k = 40 (the small dense configuration)
    A1 = torch.from_numpy(W.dense_haar_500x400()).to(dev)
    reps = 50
    mean_ms, med_ms, r1 = _timed_calls(lambda: rp.rplu_dense(A1, 40, seed=7), reps)
    errs = []
    for s_ in range(30):
        g = rp.rplu_dense(A1, 40, seed=100 + s_)
        errs.append(dense_explicit_error(A1, g.L, g.U))
    out["dense_f64_500x400_k40"] = {
        "ms_per_factorization": mean_ms, "median_ms": med_ms, "us_per_step": mean_ms * 1e3 / 40,
        "factorizations_per_s": 1e3 / mean_ms, "calls_timed": reps,
        "rel_error_mean_30_seeds": float(np.mean(errs)), "rel_error_max_30_seeds": float(np.max(errs)),
        "eckart_young_bound": float(math.sqrt(np.sum(0.64 ** np.arange(40, 400)) / np.sum(0.64 ** np.arange(400)))),
        "note": "inputs resident; one rplu_dense call per factorization (allocation, 2 launches per step, sync)"}
    del A1
    # the spiral Cauchy matrix in complex128 (matrix-free), beside the step's complex64
    n = xd.shape[0]
    x128, y128 = xd.to(torch.complex128), yd.to(torch.complex128)
    mean_ms, med_ms, r2 = _timed_calls(lambda: rp.rplu_cauchy(x128, y128, args.cauchy_k, seed=2000), 3)
    out["cauchy_c128_spirals"] = {
        "n": n, "k": args.cauchy_k, "ms_per_factorization": mean_ms, "factorizations_per_s": 1e3 / mean_ms,
        "rel_error": cauchy_explicit_error(x128, y128, r2.L, r2.U),
        "rel_error_c64_same_points_rounded": cauchy_explicit_error(xd, yd, rc64.L, rc64.U),
        "note": "complex128 points = the complex64 points of the step, widened; entries generated in FP64"}
    # the 32768^2 dense matrix through the FP64 path
    A64 = F.to_torch(dev, torch.float64)
    mean_ms, med_ms, r3 = _timed_calls(lambda: rp.rplu_dense(A64, args.dense_k, seed=1000), 2)
    e64 = dense_explicit_error(A64, r3.L, r3.U)
    e32 = dense_explicit_error(A32, rd32.L, rd32.U)
    out["dense_f64_path_32768"] = {
        "n": A64.shape[0], "k": args.dense_k, "ms_per_factorization": mean_ms,
        "factorizations_per_s": 1e3 / mean_ms, "rel_error": e64,
        "fp32_update_rel_error": e32, "fp32_update_ms": None,
        "eckart_young_bound": float(math.sqrt(np.sum((1.0 + np.arange(args.dense_k, A64.shape[0])) ** -4.0) /
                                              np.sum((1.0 + np.arange(A64.shape[0])) ** -4.0))),
        "note": ("FP64 operand (8.6 GB) against the FP32 operand of the step (4.3 GB): errors explicit in FP64 "
                 "against each run's own operand; same generator, different rounding of A")}
    del A64
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ Cauchy-like

def run_cauchy_like(args, dev, xd, yd, ck, clock_mhz):
    """The step's Cauchy matrix (complex64 spirals, n = m = CAUCHY_N) factored
    through its generators (rplu_cauchy_like, G = B = 1): exact row norms every
    step instead of the matrix-free estimate.  Timed with CUDA events, inputs
    resident; explicit FP64 error after the run."""
    import torch

    import paper_2601_22344_gb300 as rp

    n, m = xd.shape[0], yd.shape[0]
    G = torch.ones((n, 1), dtype=xd.dtype, device=dev)
    B = torch.ones((1, m), dtype=xd.dtype, device=dev)
    for q in range(2):
        rp.rplu_cauchy_like(xd, yd, G, B, ck, seed=3000 + q)
    torch.cuda.synchronize()
    reps = 3
    prof = np.zeros(4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for q in range(reps):
        r = rp.rplu_cauchy_like(xd, yd, G, B, ck, seed=3100 + q, prof=prof)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    with torch.no_grad():
        A = 1.0 / (xd.to(torch.complex128)[:, None] - yd.to(torch.complex128)[None, :])
        R = A - r.L.to(torch.complex128) @ r.U.to(torch.complex128)
        explicit = float(torch.linalg.norm(R) / torch.linalg.norm(A))
        del A, R
    norms_ms = prof[0] / max(prof[1], 1)
    entries = float(n) * m  # generated entries per row-norm pass
    mhz = clock_mhz or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * RCP_PER_SM_PER_CLK * mhz * 1e6 / 1e9
    achieved = entries / (norms_ms / 1e3) / 1e9
    return {
        "workload": f"complex64 Cauchy {n}x{m} (the step's spiral matrix) through its generators, k={ck}",
        "ms_per_factorization": ms, "factorizations_per_s": 1e3 / ms, "k_done": int(r.k_done),
        "rel_error_reported": float(np.sqrt(r.T[-1] / r.T[0])), "rel_error_explicit": explicit,
        "row_norm_pass_ms": norms_ms,
        "roofline": {"bound": "alu", "kernel": "k_cl_norms (exact row norms from the generators)",
                     "achieved": achieved, "peak": peak, "unit": "G entries/s", "frac": achieved / peak,
                     "peak_source": (f"one MUFU reciprocal per generated entry: {sms} SMs x {RCP_PER_SM_PER_CLK}/clk "
                                     f"x {mhz:.0f} MHz"), "traffic": None},
    }


# The sparse workload: a Chung-Lu graph's mean degree and power-law exponent
SPARSE_AVG_DEGREE, SPARSE_EXPONENT = 6.0, 2.2

# The multi-level Toeplitz workload of Sec. 4.2: domain side, shift, standard deviation
TOEPLITZ_LENGTH, TOEPLITZ_DELTA, TOEPLITZ_SIGMA = 320.0, 50.0, 80.0

# FP32 lane operations per generated complex64 entry in k_cf_matvec (two
# subtractions, |z|^2 as a multiply and an FMA, two operations for each of the
# real and imaginary parts of z conj(u), two accumulating FMAs), and FP32 lanes
# per SM per clock.
CF_MATVEC_FP32_OPS = 10
FP32_LANES_PER_SM_PER_CLK = 128


def cauchy_matvec_roofline(prof_c, n, m, clock_mhz, sms):
    """Roofline of the matrix-free pass's generated matvec (complex64): n*m
    generated entries per launch over the mean launch time (CUDA events of the
    timed steps), against the FP32 pipe's rate for 10 lane operations per entry;
    the MUFU reciprocal (16 per SM per clock) would allow 1.25x that."""
    if not (prof_c[1] > 0 and prof_c[0] > 0):
        return {"error": "no matvec launch was timed"}
    avg_s = prof_c[0] / 1e3 / prof_c[1]
    mhz = clock_mhz or 2070.0
    peak = sms * FP32_LANES_PER_SM_PER_CLK / CF_MATVEC_FP32_OPS * mhz * 1e6 / 1e9
    achieved = float(n) * m / avg_s / 1e9
    return {"bound": "alu", "kernel": "k_cf_matvec<complex64> (g = A conj(u), entries generated)",
            "achieved": achieved, "peak": peak, "unit": "G entries/s", "frac": achieved / peak,
            "peak_source": (f"{CF_MATVEC_FP32_OPS} FP32 lane operations per entry: {sms} SMs x "
                            f"{FP32_LANES_PER_SM_PER_CLK} lanes/clk / {CF_MATVEC_FP32_OPS} x {mhz:.0f} MHz "
                            f"(sampled SM clock); MUFU: {RCP_PER_SM_PER_CLK}/clk/SM"),
            "avg_launch_ms": avg_s * 1e3, "launches": int(prof_c[1]), "traffic": None}


def _section(fn, *a, **kw):
    """Run one of the secondary workloads after the headline step.  An error
    there is reported in its own object ({"error": ...}, also on stderr) rather
    than losing the headline line; the step's figures above are complete by
    then."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001
        msg = f"{type(e).__name__}: {e}"
        print(f"bench: {fn.__name__} failed: {msg}", file=sys.stderr, flush=True)
        return {"error": msg}


def run_cauchy_cur(args, dev, xd, yd, ck):
    """The step's Cauchy matrix (complex64 spirals, n = m = CAUCHY_N, k =
    CAUCHY_K) factored in CUR form (rplu_cauchy_cur, Algorithm 2 as printed):
    no L or U, the pivot rows and columns generated again every step and the
    core inverse A(I,J)^{-1} updated by block inversion.  Timed with CUDA events,
    inputs resident; the device memory the form keeps against the LU form's L
    and U; explicit FP64 error of A(:,J) core A(I,:) after the run."""
    import torch

    import paper_2601_22344_gb300 as rp

    n, m = xd.shape[0], yd.shape[0]
    for q in range(2):
        rp.rplu_cauchy_cur(xd, yd, ck, seed=4000 + q)
    torch.cuda.synchronize()
    reps = 3
    prof = np.zeros(4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for q in range(reps):
        r = rp.rplu_cauchy_cur(xd, yd, ck, seed=4100 + q, prof=prof)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    kd = int(r.k_done)
    with torch.no_grad():
        A = 1.0 / (xd.to(torch.complex128)[:, None] - yd.to(torch.complex128)[None, :])
        I = torch.as_tensor(r.I).to(dev)
        J = torch.as_tensor(r.J).to(dev)
        C = torch.as_tensor(r.core).to(dev).to(torch.complex128)
        R = A - A[:, J] @ C @ A[I, :]
        explicit = float(torch.linalg.norm(R) / torch.linalg.norm(A))
        del A, R
    w = xd.element_size()
    return {
        "workload": f"complex64 Cauchy {n}x{m} (the step's spiral matrix) in CUR form, k={ck}",
        "ms_per_factorization": ms, "factorizations_per_s": 1e3 / ms, "k_done": kd,
        "matvec_ms": prof[0] / max(prof[1], 1),
        "rel_error_explicit": explicit,
        "kept_bytes": {"cur_core_fp64": 16 * ck * ck, "lu_factors": w * ck * (n + m)},
    }


# ------------------------------------------------- Algorithm 3 (bounds)

BH_NU, BH_LEAF, BH_K = 5.0, 32, 1000
BH_CASES = (("tan", 2000, 3), ("sin", 2000, 3), ("tan", 20000, 1))
FP64_FLOP_PER_SM_PER_CLK = 4  # 1.25 TFLOP/s nominal FP64 over 152 SMs at 2.07 GHz


def _bh_flops(st, n, p, complex_):
    """Algorithmic FLOPs of one bounds launch (Algorithm C.2) from the plan's
    sizes: per exact pair |sum_l g_l b_l|^2 / |x_i - y_j|^2 (a division counts
    as one FLOP), per aggregated entry the 2p^2 FMAs of M_l += alpha H_s, per
    point the quadratic form G(i,:) M_l G(i,:)^*."""
    near = (8 * p + 9) if complex_ else (2 * p + 5)
    far_pt = (10 * p * p) if complex_ else (3 * p * p)
    return st["exact_pairs"] * near + st["aggregated_entries"] * 4 * p * p + n * far_pt


def _oracle_bh_time(x, y, G, B, k_sample, seed):
    """Seconds of the oracle's Algorithm 3 (own quadtrees every step) for the
    first k_sample steps and for none (exact initial norms only)."""
    import oracle
    t = time.perf_counter()
    oracle.rplu_cauchy_like_bh(x, y, G, B, 0, seed=seed, nu=BH_NU, leaf=BH_LEAF)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    oracle.rplu_cauchy_like_bh(x, y, G, B, k_sample, seed=seed, nu=BH_NU, leaf=BH_LEAF)
    t1 = time.perf_counter() - t
    return t0, max(t1 - t0, 0.0) / k_sample


def run_bh(args, dev, clock_mhz, with_oracle=True):
    """Algorithm 3 (rejection-sampled rows against the App. C bounds, nu = 5,
    leaves of 32 points) on the Loewner matrices of Sec. 5.2 (Fig. 7): f(z) =
    tan(20 z^20) on the unit disk (complex128) and sin(1000 z) on [-1, 1]
    (float64), n = m points, rank k = 1000.  Per case: ms per factorization
    through one CUDA graph (inputs resident), the bounds kernel's average
    launch time from a timed run (host-driven loop, CUDA events around each
    launch), its FP64 roofline, mean proposals per step and the residual."""
    import torch

    import paper_2601_22344_gb300 as rp

    mhz = clock_mhz or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP64_FLOP_PER_SM_PER_CLK * mhz * 1e6 / 1e12
    cases = []
    for kind, n, reps in BH_CASES[: args.bh_cases]:
        x, y, G, B = W.loewner_experiment(kind, n, seed=W.derive_seed(6, n))
        complex_ = kind == "tan"
        dt = torch.complex128 if complex_ else torch.float64
        conv = (lambda a: a) if complex_ else (lambda a: np.ascontiguousarray(a.real))
        xd, yd, Gd, Bd = (torch.from_numpy(np.ascontiguousarray(conv(v))).to(dev, dt) for v in (x, y, G, B))
        k = min(args.bh_k, n)
        call = lambda seed, prof=None: rp.rplu_cauchy_like(xd, yd, Gd, Bd, k, seed=seed, bound_nu=BH_NU,  # noqa: E731
                                                            bound_leaf=BH_LEAF, prof=prof)
        call(7000)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for q in range(reps):
            r = call(7100 + q)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        prof = np.zeros(4)
        call(7200, prof)
        torch.cuda.synchronize()
        bounds_ms = prof[0] / max(prof[1], 1)
        st = rp.rplu_bh_plan_stats(xd, yd, nu=BH_NU, leaf=BH_LEAF)
        flops = _bh_flops(st, n, 2, complex_)
        achieved = flops / (bounds_ms / 1e3) / 1e12
        T = r.T
        # relative residual: exact ||S||_F^2 after the last step over the exact ||A||_F^2
        A0 = rp.rplu_cauchy_like(xd, yd, Gd, Bd, 0).T[0]
        case = {
            "workload": (f"Loewner {'tan(20 z^20), unit disk, complex128' if complex_ else 'sin(1000 z), [-1, 1], float64'}"
                         f" n = m = {n}, k = {k}, nu = {BH_NU}, leaf {BH_LEAF}"),
            "ms_per_factorization": ms, "factorizations_per_s": 1e3 / ms, "k_done": int(r.k_done),
            "ms_per_step": ms / max(int(r.k_done), 1),
            "mean_proposals_per_step": float(np.mean(r.attempts)) if r.attempts is not None else None,
            "exact_fallback_steps": int(np.sum(r.attempts == 65)) if r.attempts is not None else None,
            "rel_residual": float(np.sqrt(T[-1] / A0)),
            "plan": st,
            "roofline": {"bound": "alu", "kernel": "k_bh_bounds (Algorithm C.2, FP64)", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "peak_source": (f"nominal FP64 rate: {sms} SMs x {FP64_FLOP_PER_SM_PER_CLK} FLOP/clk x "
                                         f"{mhz:.0f} MHz"),
                         "flops_per_launch": flops, "avg_launch_ms": bounds_ms, "traffic": None},
        }
        if with_oracle and n <= 2000:
            ks = 10
            t0, per_step = _oracle_bh_time(x if complex_ else x.real + 0j, y if complex_ else y.real + 0j,
                                           G, B, ks, 7300)
            fact_s = t0 + k * per_step
            case["cpu_baseline"] = {"value": 1.0 / fact_s, "unit": "factorizations/s", "cores": 1, "kind": "oracle",
                                    "sample": (f"oracle (plain C, complex128, 1 thread) on the same input: the first "
                                               f"{ks} steps ({per_step * 1e3:.1f} ms/step) and the exact initial norms "
                                               f"({t0:.2f} s), extrapolated to {k} steps = {fact_s:.1f} s")}
        cases.append(case)
        del xd, yd, Gd, Bd
    return {"cases": cases}


# ------------------------------------------------------------- CUR-AAA

AAA_M, AAA_D, AAA_EPS, AAA_HOLDOUT = 200_000, 400, 1e-11, 1_000_000


def run_aaa(args, dev):
    """CUR-AAA (Sec. 5.3) in the setting of the paper's Fig. 9: m = 200 000
    samples uniform on the unit disk, f(z) = tan(sqrt(d) z^sqrt(d)) with d =
    400, eps = 1e-11, with RPLU and with C2PLU pivots; wall time of the whole
    rplu_cur_aaa call (split, generators, Algorithm 3 with bounds, both
    Householder fits and evaluations; inputs resident; after one untimed
    call), the support size, and
    the maximum error on the samples and on 10^6 fresh points of the disk."""
    import torch

    import paper_2601_22344_gb300 as rp

    rng = np.random.default_rng(W.derive_seed(8, args.aaa_m))
    m = args.aaa_m
    z = np.sqrt(rng.random(m)) * np.exp(2j * np.pi * rng.random(m))
    s = math.sqrt(AAA_D)
    fn = lambda q: np.tan(s * q ** s)  # noqa: E731
    f = fn(z)
    zh = np.sqrt(rng.random(AAA_HOLDOUT)) * np.exp(2j * np.pi * rng.random(AAA_HOLDOUT))
    fh = fn(zh)
    zd, fd = torch.from_numpy(z).to(dev), torch.from_numpy(f).to(dev)
    zhd = torch.from_numpy(zh).to(dev)
    # one untimed call (the first timed call's arguments) so that first-use costs
    # (module loading, allocator growth) stay out of the timings
    rp.rplu_cur_aaa(zd, fd, eps=AAA_EPS, k_max=2000, seed=9000, pivot="random")
    torch.cuda.synchronize()
    out = []
    for mode in ("random", "c2"):
        torch.cuda.synchronize()
        t = time.perf_counter()
        g = rp.rplu_cur_aaa(zd, fd, eps=AAA_EPS, k_max=2000, seed=9000, pivot=mode)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t
        r = g(zhd, zd, fd).cpu().numpy()
        out.append({
            "pivots": "RPLU" if mode == "random" else "C2PLU",
            "seconds": sec, "support_points": int(g.k), "chosen": g.which,
            "max_err_samples": min(g.err_I, g.err_J), "max_err_other_candidate": max(g.err_I, g.err_J),
            "max_err_holdout": float(np.max(np.abs(r - fh))),
        })
    return {"workload": (f"CUR-AAA, f(z) = tan({s:.0f} z^{s:.0f}) (d = {AAA_D}), {m} samples uniform on the unit "
                         f"disk, eps = {AAA_EPS}, hold-out {AAA_HOLDOUT} points; complex128"),
            "runs": out,
            "paper": "about 50 s for CUR-AAA and about 50 min for AAA on an Apple M3 Max CPU (Sec. 5.3), context only"}


# ----------------------------------------------------------------- batch

def batch_entries(res, ns, ms) -> float:
    """Generated Cauchy entries per batch: every pass (the initial norms and one
    per step) forms all n*m entries of its job."""
    return float(sum((r.k_done + 1) * n * m for r, n, m in zip(res, ns, ms)))


def run_batch(args, dev, rank, gpu_uuid):
    """4096 real Cauchy blocks (n, m ~ U{64..1024}, points in separated unit
    intervals, centres 3-6 apart), each factored to ||S||_F <= 1e-6 ||A||_F,
    FP32 with FP64 sampling: one persistent launch replayed from a captured
    CUDA graph (autotuned shape).  Also: the same jobs one FP64 rplu_dense call
    each (a sample), and rplu_batch end to end from host memory."""
    import torch

    import paper_2601_22344_gb300 as rp
    from paper_2601_22344_gb300 import batch as B

    blocks = W.cauchy_interval_blocks(args.batch_jobs, seed=W.derive_seed(4, rank))
    ns = [len(b.x) for b in blocks]
    ms = [len(b.y) for b in blocks]
    specs = [dict(kind="cauchy", x=torch.from_numpy(b.x.astype(np.float32)).to(dev),
                  y=torch.from_numpy(b.y.astype(np.float32)).to(dev), dtype="f32") for b in blocks]
    seed = W.derive_seed(5, rank)
    plan = B.BatchPlan(specs, rel_tol=BATCH_TOL, seed=seed, tune=bool(args.batch_tune))
    shape = plan.shape()
    s = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        plan.run(s.cuda_stream)
    plan.wait()
    reps = max(args.steps, 3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    with ClockSampler(gpu_uuid) as clk:
        for q in range(reps):
            flush.fill_(float(q))  # write more than L2 between timed replays
            ev[q][0].record(s)
            plan.run(s.cuda_stream)
            ev[q][1].record(s)
        st = plan.wait()
    clocks = clk.summary()
    clock_mhz = clocks.get("sm_mhz")
    batch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    res = plan.results()
    ks = np.array([r.k_done for r in res])
    rr = np.array([r.rel_res for r in res])
    entries = batch_entries(res, ns, ms)
    # explicit FP64 error of sampled jobs (outside the timed region)
    rng = np.random.default_rng(0)
    errs = []
    for b in rng.choice(len(blocks), 16, replace=False):
        A = W.cauchy_dense(blocks[b].x.astype(np.float32), blocks[b].y.astype(np.float32)).astype(np.float64)
        LU = res[b].L.double().cpu().numpy() @ res[b].U.double().cpu().numpy()
        errs.append(float(np.linalg.norm(A - LU) / np.linalg.norm(A)))
    plan.close()
    # the plain alternative: one FP64 rplu_dense call per job, same tolerance
    sample = list(range(0, len(blocks), max(1, len(blocks) // BATCH_FP64_SAMPLE)))[:BATCH_FP64_SAMPLE]
    mats = [torch.from_numpy(W.cauchy_dense(blocks[b].x.astype(np.float32).astype(np.float64),
                                            blocks[b].y.astype(np.float32).astype(np.float64))).to(dev)
            for b in sample]
    rp.rplu_dense(mats[0], min(mats[0].shape), seed=1, rel_tol=BATCH_TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f64_err = []
    for q, b in enumerate(sample):
        r = rp.rplu_dense(mats[q], min(mats[q].shape), seed=B.job_seed(seed, b), rel_tol=BATCH_TOL)
        f64_err.append(math.sqrt(r.T[-1] / r.T[0]))
    torch.cuda.synchronize()
    f64_rate = len(sample) / (time.perf_counter() - t0)
    del mats
    # end to end: host (numpy) points in, host factors out, staging inside the call.  The blocks' points
    # are held as ranges of two packed arrays (as a hierarchical matrix stores them) and passed in one call;
    # one untimed call first (the library's pinned and device staging grow to the batch's size once), then
    # the mean of BATCH_E2E_CALLS calls, each writing into the previous call's output arrays (out=), as a
    # loop over batches would; beside it the same calls with fresh output arrays each
    Xh = np.concatenate([b.x.astype(np.float32) for b in blocks])
    Yh = np.concatenate([b.y.astype(np.float32) for b in blocks])
    hres = B.rplu_batch_cauchy_packed(Xh, Yh, ns, ms, rel_tol=BATCH_TOL, seed=seed)
    t0 = time.perf_counter()
    for _ in range(BATCH_E2E_CALLS):
        hres = B.rplu_batch_cauchy_packed(Xh, Yh, ns, ms, rel_tol=BATCH_TOL, seed=seed, out=hres)
    e2e_s = (time.perf_counter() - t0) / BATCH_E2E_CALLS
    t0 = time.perf_counter()
    for _ in range(BATCH_E2E_CALLS):
        fres = B.rplu_batch_cauchy_packed(Xh, Yh, ns, ms, rel_tol=BATCH_TOL, seed=seed)
    fresh_s = (time.perf_counter() - t0) / BATCH_E2E_CALLS
    del fres
    h2d = sum((n + m) * 4 for n, m in zip(ns, ms))
    d2h = sum(int(kd) * (n + m) * 4 + 2 * 8 * min(n, m) for kd, n, m in zip(hres.k_done, ns, ms))
    value = len(blocks) / (batch_ms / 1e3)
    mhz = clock_mhz or 2070.0
    import torch.cuda as tc
    sms = tc.get_device_properties(dev).multi_processor_count
    peak = sms * RCP_PER_SM_PER_CLK * mhz * 1e6 / 1e9  # G reciprocals/s
    achieved = entries / (batch_ms / 1e3) / 1e9
    return {
        "workload": (f"{len(blocks)} real Cauchy blocks 1/(x_i-y_j), n,m ~ U{{64..1024}}, separated unit "
                     f"intervals (centres 3-6 apart), rank to ||S||_F/||A||_F <= {BATCH_TOL:g}, FP32 with FP64 "
                     f"sampling; one persistent launch from a captured CUDA graph"),
        "value": value, "unit": "factorizations/s", "ms_per_batch": batch_ms, "reps": reps,
        "status": int(st), "shape": shape,
        "k_mean": float(ks.mean()), "k_max": int(ks.max()), "rel_res_max": float(rr.max()),
        "explicit_rel_error_sample": {"jobs": len(errs), "max": max(errs), "mean": statistics.mean(errs)},
        "fp64_one_job_per_call": {"value": f64_rate, "unit": "factorizations/s", "jobs": len(sample),
                                  "rel_res_max": max(f64_err), "speedup_of_batch": value / f64_rate},
        "e2e": {"value": len(blocks) / e2e_s, "unit": "factorizations/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "calls_timed": BATCH_E2E_CALLS,
                "api": ("rplu_batch_cauchy_packed (rplu_batch), numpy host buffers, each call writing into "
                        "the previous call's output arrays (out=); where the device accesses pageable host "
                        "memory in place, one kernel gathers the points from them and one writes the factors "
                        "into them (no pinned staging)"),
                "fresh_output_arrays": {"value": len(blocks) / fresh_s, "unit": "factorizations/s"}},
        "roofline": {"bound": "alu", "kernel": "k_batch (persistent, generated Cauchy entries)",
                     "achieved": achieved, "peak": peak, "unit": "G entries/s", "frac": achieved / peak,
                     "peak_source": (f"one MUFU reciprocal per generated entry: {sms} SMs x "
                                     f"{RCP_PER_SM_PER_CLK}/clk x {mhz:.0f} MHz (sampled SM clock)"),
                     "entries_per_batch": entries, "traffic": None},
        "gpu_launches_per_batch": 1,
        "clocks": clocks,
    }


def run_serving(args, dev, rank):
    """Poisson arrivals of mixed requests into one serving session (continuous
    batching); for each arrival rate: throughput of completed requests, p50 /
    p99 latency (submit to completion), backlog when arrivals stop.  Then one
    rate with a share of large Cauchy requests (n, m up to 20000, above the
    kernel's 4096: Algorithm 3 on the large-request streams)."""
    import threading

    import torch

    from paper_2601_22344_gb300 import serve as SV

    cauchy, dense = W.serving_pool(args.serve_pool, max(4, args.serve_pool // 16), seed=W.derive_seed(6, rank),
                                   cauchy_range=(256, 4096), clouds=True)
    cpool = [(torch.from_numpy(b.x.astype(np.complex64)).to(dev), torch.from_numpy(b.y.astype(np.complex64)).to(dev))
             for b in cauchy]
    dpool = [F.to_torch(dev, torch.float32) for F in dense]
    lrng = np.random.default_rng(W.derive_seed(8, rank))
    lpool = []
    for q in range(SERVE_LARGE_POOL):
        n, m = (int(round(np.exp(lrng.uniform(np.log(SERVE_LARGE_RANGE[0]), np.log(SERVE_LARGE_RANGE[1])))))
                for _ in range(2))
        gen = W.cauchy_spirals if q % 2 == 0 else W.cauchy_smiley
        x, y = gen(n, m, seed=W.derive_seed(9, rank, q))
        lpool.append((torch.from_numpy(x.astype(np.complex64)).to(dev), torch.from_numpy(y.astype(np.complex64)).to(dev)))
    torch.cuda.synchronize()
    sess = SV.Session(bound_nu=SERVE_BOUND_NU)

    def one_rate(rate, large_frac):
        rng = np.random.default_rng(int(rate))
        n_req = max(1, int(rate * args.serve_seconds))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        is_cauchy = rng.random(n_req) < 0.7
        picks = rng.integers(0, 1 << 30, n_req)
        is_large = rng.random(n_req) < large_frac if large_frac > 0 else np.zeros(n_req, bool)
        lat, qms, status, kd, lat_large = [], [], [], [], []
        large_tickets = set()
        large0 = sess.stats()["large_completed"]
        state = {"submitted": 0, "stop": False}
        lock = threading.Lock()

        def collect():
            while True:
                got = sess.completed(4096)
                for t, info in got:
                    sess.release(t)
                    with lock:
                        lat.append(info.latency_ms)
                        qms.append(info.queue_ms)
                        status.append(info.status)
                        kd.append(info.k_done)
                        if t in large_tickets:
                            lat_large.append(info.latency_ms)
                if not got:
                    with lock:
                        if state["stop"]:
                            return
                    time.sleep(0.0002)

        col = threading.Thread(target=collect)
        col.start()
        t0 = time.perf_counter()
        for q in range(n_req):
            delay = t0 + arrivals[q] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            if is_large[q]:
                x, y = lpool[picks[q] % len(lpool)]
                spec = dict(kind="cauchy", x=x, y=y)
            elif is_cauchy[q]:
                x, y = cpool[picks[q] % len(cpool)]
                spec = dict(kind="cauchy", x=x, y=y)
            else:
                A = dpool[picks[q] % len(dpool)]
                spec = dict(kind="dense", A=A)
            with lock:
                t = sess.submit(spec, rel_tol=BATCH_TOL, seed=int(picks[q]))
                if is_large[q]:
                    large_tickets.add(t)
                state["submitted"] += 1
        t_arr = time.perf_counter() - t0
        st = sess.stats()
        backlog = st["queued"] + st["running"]
        deadline = time.perf_counter() + args.serve_drain
        while time.perf_counter() < deadline:
            with lock:
                if len(lat) >= n_req:
                    break
            time.sleep(0.002)
        t_end = time.perf_counter() - t0
        with lock:
            state["stop"] = True
        col.join()
        done = len(lat)
        ok = sum(1 for v in status if v == 0)
        lat_a = np.array(lat) if lat else np.array([np.nan])
        out = {
            "rate_per_s": rate, "seconds": args.serve_seconds, "submitted": n_req, "completed": done,
            "ok": ok, "large_requests": int(sess.stats()["large_completed"] - large0),
            "throughput_per_s": done / t_end, "p50_ms": float(np.percentile(lat_a, 50)),
            "p99_ms": float(np.percentile(lat_a, 99)), "mean_queue_ms": float(np.nanmean(qms)) if qms else None,
            "backlog_when_arrivals_end": backlog, "arrivals_s": t_arr, "drained_s": t_end,
            "mean_k": float(np.mean(kd)) if kd else None,
        }
        if large_frac > 0:
            la = np.array(lat_large) if lat_large else np.array([np.nan])
            out.update({"large_fraction": large_frac, "large_submitted": len(large_tickets),
                        "large_p50_ms": float(np.percentile(la, 50)), "large_p99_ms": float(np.percentile(la, 99))})
        # leave nothing behind for the next rate
        if done < n_req:
            deadline = time.perf_counter() + 120
            while sess.stats()["queued"] + sess.stats()["running"] > 0 and time.perf_counter() < deadline:
                for t, _ in sess.completed(4096):
                    sess.release(t)
                time.sleep(0.01)
            for t, _ in sess.completed(1 << 16):
                sess.release(t)
        return out

    results = [one_rate(rate, 0.0) for rate in args.serve_rates]
    with_large = one_rate(args.serve_large_rate, args.serve_large_frac) if args.serve_large_frac > 0 else None
    sess.close()
    return {
        "workload": (f"Poisson arrivals; 70% complex64 Cauchy requests on the spiral-and-cluster and smiley "
                     f"clouds (half each, n, m log-uniform in [256, 4096]), 30% dense FP32 n x n (n log-uniform "
                     f"in [256, 2048], sigma_i = 0.9^i, Householder-product factors); each to 1e-6 relative "
                     f"error; every request runs in the one persistent serving kernel (Cauchy ones in the "
                     f"generator form with exact norms, up to n, m = 4096; dense ones up to 2048)"),
        "pool": {"cauchy": len(cpool), "dense": len(dpool), "large_cauchy": len(lpool)},
        "rates": results,
        "with_large_cauchy": None if with_large is None else {
            "workload": (f"the same mix at {args.serve_large_rate:g}/s with a share {args.serve_large_frac:g} of "
                         f"the requests replaced by complex64 Cauchy requests on the same clouds with n, m "
                         f"log-uniform in [{SERVE_LARGE_RANGE[0]}, {SERVE_LARGE_RANGE[1]}] (above the kernel's "
                         f"4096): rplu_cauchy_like with unit generators and Algorithm 3 (nu = "
                         f"{SERVE_BOUND_NU:g}) on the session's large-request streams"),
            **with_large},
    }


def run_batch_only(args):
    """The batch workload alone (for profiling): one JSON line with its figures."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    out = {"metric": METRIC, "workload": "batch only", "batch": run_batch(args, dev, rank, gpu_uuid)}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_bh_only(args):
    """Algorithm 3 on the Loewner matrices alone (for profiling): one JSON line."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {"metric": METRIC, "workload": "Cauchy-like with bounds only",
           "cauchy_like_bounds": run_bh(args, dev, None, with_oracle=False)}
    if rank == 0:
        print(json.dumps(out), flush=True)


def toeplitz_sampled_error(N, length, I, J, core, n_sample=2000, seed=0):
    """||A(P,Q) - A(P,J) core A(I,Q)||_F / ||A(P,Q)||_F on random row and column
    samples P, Q of the multi-level Toeplitz matrix (entries from the kernel of
    Eq. kernel at the grid points, formed here in FP64): an estimate of the
    relative Frobenius error that never forms an n x n matrix."""
    n = N ** 3
    h = length / N
    rng = np.random.default_rng(seed)
    P = rng.integers(0, n, n_sample)
    Q = rng.integers(0, n, n_sample)

    def pts(idx):
        idx = np.asarray(idx, dtype=np.int64)
        return np.stack([idx // (N * N), (idx // N) % N, idx % N], axis=1) * h

    def block(rows, cols):
        d = pts(rows)[:, None, :] - pts(cols)[None, :, :]
        return np.exp(-(((d[..., 0] - TOEPLITZ_DELTA) ** 2) + d[..., 1] ** 2 + d[..., 2] ** 2)
                      / (2.0 * TOEPLITZ_SIGMA ** 2))

    A_PQ = block(P, Q)
    approx = block(P, J) @ (core @ block(I, Q))
    return float(np.linalg.norm(A_PQ - approx) / np.linalg.norm(A_PQ))


def run_toeplitz(args, dev, clock_mhz=None):
    """RPLU in CUR form on the multi-level Toeplitz matrix of Sec. 4.2 (the
    drifted Gaussian kernel on an N^3 grid of [0, 320]^3; the paper's N = 128 and
    320, rank 512 for its preconditioner): one factorization, CUDA events around
    the call (inputs are four scalars; outputs resident), the matvec's mean time
    per step and its FP64 roofline (3 N^4 FMAs per matvec against the nominal FP64
    rate), the row-norm estimate of the final error and a sampled explicit one."""
    import torch

    import paper_2601_22344_gb300 as rp

    N, k = args.t3_n, args.t3_k
    length = TOEPLITZ_LENGTH
    rp.rplu_toeplitz3_cur(min(N, 16), 8, seed=1, length=length)  # untimed: first-use costs
    torch.cuda.synchronize()
    prof = np.zeros(4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g = rp.rplu_toeplitz3_cur(N, k, seed=5, length=length, prof=prof)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mv_ms = prof[0] / max(prof[1], 1)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clock_mhz or 2070.0
    peak = sms * FP64_FLOP_PER_SM_PER_CLK * mhz * 1e6 / 1e12
    achieved = 2.0 * 3.0 * float(N) ** 4 / (mv_ms / 1e3) / 1e12
    kd = g.k_done
    I, J = g.I.cpu().numpy(), g.J.cpu().numpy()
    core = g.core.cpu().numpy()
    return {
        "workload": (f"multi-level Toeplitz (drifted Gaussian, shift {TOEPLITZ_DELTA:g}, sd {TOEPLITZ_SIGMA:g}) on a "
                     f"{N}^3 grid of [0, {length:g}]^3, n = {N ** 3}, RPLU in CUR form to k = {k}; FP64"),
        "seconds": ms / 1e3, "k_done": kd, "matvec_ms_per_step": mv_ms,
        "rel_error_estimate": float(np.sqrt(max(g.T[-1], 0.0) / g.T[0])),
        "rel_error_sampled": toeplitz_sampled_error(N, length, I, J, core),
        "device_bytes_kept": int(6 * N ** 3 * 8 + 2 * N ** 3 + kd * kd * 8),
        "roofline": {"bound": "alu", "kernel": "k_t3_conv x 3 (the matvec, FP64)", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": (f"nominal FP64 rate: {sms} SMs x {FP64_FLOP_PER_SM_PER_CLK} FLOP/clk x "
                                     f"{mhz:.0f} MHz"), "traffic": None},
        "paper": ("about 10 minutes for a rank-512 RPLU factorization at N = 320 on an A100 (JAX, FFT matvecs; "
                  "Sec. 4.3), context only"),
    }


def run_toeplitz_only(args):
    """The Toeplitz CUR-form workload alone: one JSON line."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {"metric": METRIC, "workload": "Toeplitz CUR form only", "toeplitz_cur": run_toeplitz(args, dev)}
    if rank == 0:
        print(json.dumps(out), flush=True)


def sparse_sampled_error(S, I, J, core, n_sample=2000, seed=0):
    """||A(P,Q) - A(P,J) core A(I,Q)||_F / ||A(P,Q)||_F over the nonzeros of A
    and as many random entries: a sampled estimate of the relative error of a
    sparse CUR factorization without forming A densely."""
    rng = np.random.default_rng(seed)
    S = S.tocsr()
    coo = S.tocoo()
    pick = rng.integers(0, coo.nnz, n_sample)
    P = np.concatenate([coo.row[pick], rng.integers(0, S.shape[0], n_sample)])
    Q = np.concatenate([coo.col[pick], rng.integers(0, S.shape[1], n_sample)])
    a = np.asarray(S[P, Q]).ravel()
    left = S[P][:, J].toarray()              # A(P, J)
    right = S[I][:, Q].toarray()             # A(I, Q)
    approx = np.einsum("ij,ji->i", left @ core, right)
    return float(np.linalg.norm(a - approx) / max(np.linalg.norm(a), 1e-300))


def run_sparse(args, dev):
    """RPLU in CUR form on a Chung-Lu power-law graph's adjacency (the stand-in
    for the paper's SuiteSparse graphs, Sec. 4.3): one factorization, CUDA
    events around the call, the mean time per step of the CSR walk that forms
    g = A u and the residual column, and its HBM roofline (CSR values and
    indices, the gathered u and column -> pivot map, the per-row vectors), the
    row-norm estimate of the final error and a sampled explicit one."""
    import torch

    import paper_2601_22344_gb300 as rp

    n, k = args.sp_n, args.sp_k
    S = W.chung_lu_graph(n, avg_degree=SPARSE_AVG_DEGREE, exponent=SPARSE_EXPONENT, seed=W.derive_seed(9, n))
    rp.rplu_sparse_cur(S[:2000, :2000], 8, seed=1)  # untimed: first-use costs
    torch.cuda.synchronize()
    prof = np.zeros(4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g = rp.rplu_sparse_cur(S, k, seed=5, prof=prof)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    spmv_ms = prof[0] / max(prof[1], 1)
    nnz = S.nnz
    # per entry: value, column index, the gathered u and column -> pivot map; per row: row pointer,
    # the raw pivot column c, the multiplier l and g written, the pivoted-row flag
    spmv_bytes = nnz * (8 + 4 + 8 + 4) + (n + 1) * 8 + 3 * n * 8 + n
    peak, peak_kind = measured_peaks()
    achieved = spmv_bytes / (spmv_ms / 1e3) / 1e9
    I, J = g.I.cpu().numpy(), g.J.cpu().numpy()
    core = g.core.cpu().numpy()
    return {
        "workload": (f"Chung-Lu graph adjacency, n = {n}, nnz = {nnz} (mean degree {SPARSE_AVG_DEGREE:g}, exponent "
                     f"{SPARSE_EXPONENT:g}), RPLU in CUR form to k = {k}; FP64"),
        "seconds": ms / 1e3, "k_done": g.k_done, "spmv_ms_per_step": spmv_ms,
        "rel_error_estimate": float(np.sqrt(max(g.T[-1], 0.0) / g.T[0])),
        "rel_error_sampled": sparse_sampled_error(S, I, J, core),
        "roofline": {"bound": "hbm", "kernel": "k_sp_colspmv (one CSR walk: g = A u and the residual column)",
                     "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                     "alg_bytes_per_launch": spmv_bytes, "traffic": None},
        "paper": "SuiteSparse graphs with 0.9-36 million rows (Sec. 4.3); not available here, context only",
    }


def run_sparse_only(args):
    """The sparse CUR-form workload alone: one JSON line."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {"metric": METRIC, "workload": "sparse CUR form only", "sparse_cur": run_sparse(args, dev)}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_aaa_only(args):
    """CUR-AAA alone (for profiling): one JSON line."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {"metric": METRIC, "workload": "CUR-AAA only", "cur_aaa": run_aaa(args, dev)}
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_serve_only(args):
    """The serving workload alone (for profiling): one JSON line with its figures."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {"metric": METRIC, "workload": "serving only", "serving": run_serving(args, dev, rank)}
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------ oracle timing

def host_cpu():
    """(usable host cores, CPU model name) of this machine."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return cores, model or "unknown"


def _mem_available():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 16 << 30


def _concurrent(fn, args_list):
    """Run fn(*a) for every a in args_list, one host thread each (the oracle's
    ctypes calls release the GIL); the wall time of each call."""
    from concurrent.futures import ThreadPoolExecutor

    def timed(a):
        t = time.perf_counter()
        fn(*a)
        return time.perf_counter() - t

    if len(args_list) == 1:
        return [timed(args_list[0])]
    with ThreadPoolExecutor(max_workers=len(args_list)) as ex:
        return list(ex.map(timed, args_list))


class OracleStepSample:
    """Bounded samples of the oracle on the benchmark's own inputs, run as it
    stands (plain C, FP64/complex128, one thread per factorization) on
    `threads` host threads at once (each its own draws): the dense oracle
    holds its own n x m FP64 residual, so its thread count is capped by free
    host memory.  A sample runs every thread's factorization to k = 0
    (initialisation) or k = 1; a full factorization is extrapolated as
    t(0) + k (t(1) - t(0)), and the step's throughput on all the threads as
    2 / (t_dense / P_dense + t_cauchy / P_cauchy) (one dense and one Cauchy
    factorization per step, each thread busy with one factorization at a time)."""

    def __init__(self, A64, x, y, dk, ck, threads):
        import oracle
        self.oracle = oracle
        self.A64, self.x, self.y, self.dk, self.ck = A64, x, y, dk, ck
        per_dense = A64.nbytes * 1.05
        self.pd = max(1, min(threads, int(0.6 * _mem_available() // per_dense)))
        self.pc = max(1, threads)
        self.d0 = self.c0 = None
        self.d1, self.c1, self.wall = [], [], []

    def _dense(self, k, seed):
        self.oracle.rplu_dense(self.A64, k, seed=seed)

    def _cauchy(self, k, seed):
        self.oracle.rplu_cauchy(self.x, self.y, k, seed=seed)

    def init_sample(self, seed=0):
        t = time.perf_counter()
        d0 = _concurrent(self._dense, [(0, seed + r) for r in range(self.pd)])
        c0 = _concurrent(self._cauchy, [(0, seed + r) for r in range(self.pc)])
        self.d0, self.c0 = statistics.mean(d0), statistics.mean(c0)
        return time.perf_counter() - t

    def step_sample(self, seed):
        t = time.perf_counter()
        d1 = _concurrent(self._dense, [(1, seed + r) for r in range(self.pd)])
        c1 = _concurrent(self._cauchy, [(1, seed + 7919 + r) for r in range(self.pc)])
        self.d1.append(statistics.mean(d1))
        self.c1.append(statistics.mean(c1))
        w = time.perf_counter() - t
        self.wall.append(w)
        return w

    def summary(self):
        d1, c1 = statistics.mean(self.d1), statistics.mean(self.c1)
        ds, cs = max(d1 - self.d0, 0.0), max(c1 - self.c0, 0.0)
        td, tc = self.d0 + self.dk * ds, self.c0 + self.ck * cs
        value = 2.0 / (td / self.pd + tc / self.pc)
        return {"value": value, "dense_threads": self.pd, "cauchy_threads": self.pc,
                "dense_init_s": self.d0, "dense_step_s": ds, "dense_fact_s": td,
                "cauchy_init_s": self.c0, "cauchy_step_s": cs, "cauchy_fact_s": tc,
                "timed_k": {"dense": 1, "cauchy": 1}, "full_k": {"dense": self.dk, "cauchy": self.ck},
                "sample_wall_s": statistics.mean(self.wall),
                "extrapolation_factor": (td / self.pd + tc / self.pc) / statistics.mean(self.wall)}


def _oracle_inputs(A_dev, x_dev, y_dev):
    A64 = A_dev.double().cpu().numpy()
    x = x_dev.cpu().numpy().astype(np.complex128)
    y = y_dev.cpu().numpy().astype(np.complex128)
    return A64, x, y


def cpu_baseline(A_dev, x_dev, y_dev, dk, ck):
    """The oracle on the host cores: one thread, and every usable core; one
    initialisation sample and one k = 1 sample each (about 10-30 s)."""
    A64, x, y = _oracle_inputs(A_dev, x_dev, y_dev)
    cores, model = host_cpu()
    res = {}
    for label, th in (("one_thread", 1), ("all_cores", cores)):
        smp = OracleStepSample(A64, x, y, dk, ck, th)
        smp.init_sample(seed=1)
        smp.step_sample(seed=1000)
        res[label] = smp.summary()
    del A64
    allc = res["all_cores"]
    return {"value": allc["value"], "unit": "factorizations/s",
            "cores": max(allc["dense_threads"], allc["cauchy_threads"]), "kind": "oracle",
            "host": {"nproc": cores, "cpu_model": model},
            "one_thread": res["one_thread"], "all_cores": allc,
            "sample": (f"oracle (plain C, FP64/complex128) on the same full-size inputs, one initialisation (k=0) "
                       f"and one k=1 sample per factorization, {allc['dense_threads']} dense and "
                       f"{allc['cauchy_threads']} Cauchy factorizations at once on {cores} cores ({model}); "
                       f"extrapolated to k={dk} and k={ck}: the one-thread figure is "
                       f"{res['one_thread']['value']:.3g} factorizations/s")}


def workload_config(args, ws):
    """The benchmark's workload, as both arms print it."""
    dn, dk, cn, ck = args.dense_n, args.dense_k, args.cauchy_n, args.cauchy_k
    return {
        "workload": (f"dense FP32 {dn}x{dn} k={dk} (Householder-product factors, sigma_i=(1+i)^-2) + "
                     f"matrix-free complex64 Cauchy {cn}x{cn} k={ck} (spirals+cluster)"),
        "parallelism": f"independent problems per GPU x{ws}",
    }


# ------------------------------------------------------------ reference arm

def run_reference(args):
    """The oracle as it stands on the host cores, on the same workload: the
    warm-up samples time each factorization's initialisation (k = 0), each
    timed step one k = 1 sample of both factorizations, all on as many threads
    at once as there are cores (the dense ones capped by host memory); the
    factorizations/s are extrapolated to the full k from these samples, and
    the line states the timed k and the extrapolation factor."""
    ws, rank, local = _dist()
    if ws > 1 and rank != 0:
        return
    dn, dk, cn, ck = args.dense_n, args.dense_k, args.cauchy_n, args.cauchy_k
    F = W.dense_householder_inverse_square(dn, seed=W.derive_seed(3, 0))
    A64 = F.dense().astype(np.float32).astype(np.float64)
    x, y = W.cauchy_spirals_square(cn, seed=W.derive_seed(2, 0))
    x = x.astype(np.complex64).astype(np.complex128)
    y = y.astype(np.complex64).astype(np.complex128)
    cores, model = host_cpu()
    smp = OracleStepSample(A64, x, y, dk, ck, cores)
    for w in range(max(args.warmup, 1)):
        smp.init_sample(seed=10 * w)
    for st in range(args.steps):
        smp.step_sample(seed=1000 + 31 * st)
    sm = smp.summary()
    value = sm["value"]
    cfg = workload_config(args, ws)
    cfg["oracle_precision"] = "FP64/complex128 on the FP32/complex64-rounded inputs"
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "factorizations/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": max(args.warmup, 1),
        "ms_per_step": sm["sample_wall_s"] * 1e3,
        "ms_per_step_kind": "wall time of one timed sample step (k = 1 of both factorizations on all threads)",
        "extrapolation": {k_: sm[k_] for k_ in ("timed_k", "full_k", "extrapolation_factor", "dense_init_s",
                                                 "dense_step_s", "cauchy_init_s", "cauchy_step_s",
                                                 "dense_threads", "cauchy_threads")},
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": "factorizations/s",
                         "cores": max(sm["dense_threads"], sm["cauchy_threads"]), "kind": "oracle",
                         "host": {"nproc": cores, "cpu_model": model},
                         "sample": (f"warm-up: k=0 of every factorization; each timed step: k=1 of "
                                    f"{sm['dense_threads']} dense and {sm['cauchy_threads']} Cauchy factorizations "
                                    f"at once; extrapolated to k={dk} and k={ck} "
                                    f"(factor {sm['extrapolation_factor']:.0f} over the sample's wall time)")},
        "e2e": {"value": value, "unit": "factorizations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dense-n", type=int, default=DENSE_N)
    ap.add_argument("--dense-k", type=int, default=DENSE_K)
    ap.add_argument("--cauchy-n", type=int, default=CAUCHY_N)
    ap.add_argument("--cauchy-k", type=int, default=CAUCHY_K)
    ap.add_argument("--batch-jobs", type=int, default=BATCH_JOBS,
                    help="Cauchy blocks of the batch workload (0: skip it)")
    ap.add_argument("--batch-tune", type=int, default=1, help="autotune the batch plan's launch shape")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="arrival window per rate (0: skip serving)")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[500.0, 1000.0, 2000.0, 4000.0])
    ap.add_argument("--serve-pool", type=int, default=256, help="distinct Cauchy request inputs")
    ap.add_argument("--serve-drain", type=float, default=20.0, help="seconds allowed to finish after arrivals")
    ap.add_argument("--serve-large-rate", type=float, default=1000.0,
                    help="arrival rate of the serving run with large Cauchy requests")
    ap.add_argument("--serve-large-frac", type=float, default=0.01,
                    help="share of large Cauchy requests in that run (0: skip it)")
    ap.add_argument("--bh-cases", type=int, default=len(BH_CASES),
                    help="Loewner cases of the bound-based section (0: skip it)")
    ap.add_argument("--bh-k", type=int, default=BH_K, help="rank of the bound-based factorizations")
    ap.add_argument("--aaa-m", type=int, default=AAA_M, help="samples of the CUR-AAA section (0: skip it)")
    ap.add_argument("--t3-n", type=int, default=128, help="grid points per axis of the Toeplitz workload")
    ap.add_argument("--t3-k", type=int, default=512, help="rank of the Toeplitz workload")
    ap.add_argument("--sp-n", type=int, default=1_000_000, help="vertices of the sparse workload's graph")
    ap.add_argument("--sp-k", type=int, default=200, help="rank of the sparse workload")
    ap.add_argument("--workload", choices=["all", "step", "batch", "serve", "bh", "aaa", "toeplitz", "sparse"],
                    default="all",
                    help="all: the benchmark line (step + batch); step or batch alone for profiling; "
                         "toeplitz, sparse: the CUR form on those operators (not part of all)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_only(args)
    elif args.workload == "serve":
        run_serve_only(args)
    elif args.workload == "bh":
        run_bh_only(args)
    elif args.workload == "aaa":
        run_aaa_only(args)
    elif args.workload == "toeplitz":
        run_toeplitz_only(args)
    elif args.workload == "sparse":
        run_sparse_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
