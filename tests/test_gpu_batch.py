"""rplu_batch: each job of a mixed batch equals the same job run alone."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)
from paper_2601_22344_gb300 import batch as B  # noqa: E402


def _jobs(n_jobs, seed):
    blocks = W.cauchy_interval_blocks(n_jobs, seed=seed, size_lo=16, size_hi=200)
    jobs = []
    for b, blk in enumerate(blocks):
        if b % 3 == 2:
            A = W.dense_haar_decay(len(blk.x), len(blk.y), 0.7, seed=b)
            jobs.append(dict(kind="dense", A=A, dtype="f64" if b % 2 else "f32"))
        else:
            jobs.append(dict(kind="cauchy", x=blk.x, y=blk.y, dtype="f64" if b % 2 else "f32"))
    return jobs


def test_batch_equals_single_jobs(orc):
    specs = _jobs(12, seed=3)
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=5)
    for b, (spec, r) in enumerate(zip(specs, res)):
        assert r.status in (rp.RPLU_OK, rp.RPLU_NOT_CONVERGED)
        dt = {"f32": torch.float32, "f64": torch.float64}[spec["dtype"]]
        if spec["kind"] == "dense":
            A = spec["A"]
        else:
            A = W.cauchy_dense(spec["x"].astype(np.float32 if spec["dtype"] == "f32" else np.float64),
                               spec["y"].astype(np.float32 if spec["dtype"] == "f32" else np.float64))
        single = rp.rplu_dense(torch.from_numpy(np.ascontiguousarray(A)).to(dt).cuda(), min(A.shape),
                               seed=B.job_seed(5, b), rel_tol=1e-6)
        assert r.k_done == single.k_done
        assert np.array_equal(r.I, single.I.cpu().numpy())
        tol = 1e-4 if spec["dtype"] == "f32" else 1e-12
        assert np.linalg.norm(r.L - single.L.cpu().numpy()) <= tol * max(np.linalg.norm(r.L), 1e-300)
        assert r.rel_res <= 1e-6 or r.status == rp.RPLU_NOT_CONVERGED
