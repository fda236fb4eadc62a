"""rplu_batch and batch plans (the persistent batch kernel) through the C-ABI:
parity with the oracle job by job, equality with the single-job entry point,
independence of the launch shape and of the other jobs, graph replay, edge
cases, and the full-size batch of 4096 Cauchy blocks on sampled jobs."""
import ctypes

import numpy as np
import pytest

import workloads as W
from parity import GPU_TOL, TIE, assert_factors, assert_pivots, agreed_prefix, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)
from paper_2601_22344_gb300 import batch as B  # noqa: E402

NDT = {"f32": np.float32, "f64": np.float64, "c64": np.complex64}
TDT = {"f32": torch.float32, "f64": torch.float64, "c64": torch.complex64}


def _matrix(spec):
    """The matrix the GPU factors, in the job's precision (Cauchy entries rounded once)."""
    dt = NDT[spec["dtype"]]
    if spec["kind"] == "dense":
        return np.asarray(spec["A"]).astype(dt)
    return W.cauchy_dense(np.asarray(spec["x"]).astype(dt), np.asarray(spec["y"]).astype(dt))


def _mixed(n_jobs, seed, lo=16, hi=200, dtypes=("f32", "f64")):
    blocks = W.cauchy_interval_blocks(n_jobs, seed=seed, size_lo=lo, size_hi=hi)
    specs = []
    for b, blk in enumerate(blocks):
        dt = dtypes[b % len(dtypes)]
        if b % 3 == 2:
            A = W.dense_haar_decay(len(blk.x), len(blk.y), 0.7, seed=b)
            specs.append(dict(kind="dense", A=A, dtype=dt))
        else:
            specs.append(dict(kind="cauchy", x=blk.x, y=blk.y, dtype=dt))
    return specs


def _to_device(specs):
    out = []
    for sp in specs:
        d = dict(sp)
        for key in ("A", "x", "y"):
            if key in d:
                d[key] = torch.from_numpy(np.ascontiguousarray(np.asarray(d[key]).astype(NDT[sp["dtype"]]))).cuda()
        out.append(d)
    return out


def _check_vs_oracle(orc, spec, r, seed, tol_rel=1e-6, mode="random"):
    A = _matrix(spec)
    k_max = min(A.shape)
    o = orc.rplu_dense(A.astype(np.float64), k_max, seed=seed, tol=tol_rel, mode=mode)
    dt = spec["dtype"]
    upto = assert_pivots(r, o, TIE[dt], random_mode=(mode == "random"), min_steps=0, residual_scaled=True)
    assert_factors(r, o, upto, GPU_TOL[dt])
    if upto == len(o["I"]) and upto == r.k_done:
        assert r.k_done == o["k_done"]
        T = o["T"]
        # the residual computed in FP32 differs from the FP64 one by the FP32 rounding of S,
        # of order eps32 * ||A||_F (absolute, relative to ||A||_F)
        assert r.rel_res == pytest.approx(np.sqrt(T[-1] / T[0]), rel=1e-3 if dt == "f32" else 1e-8,
                                          abs=1e-7 if dt == "f32" else 1e-14)
    return upto


@pytest.mark.parametrize("dtypes", [("f64",), ("f32",)])
def test_batch_matches_oracle(orc, dtypes):
    specs = _mixed(18, seed=11, lo=3, hi=150, dtypes=dtypes)
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=7)
    for b, (sp, r) in enumerate(zip(specs, res)):
        assert r.status in (rp.RPLU_OK, rp.RPLU_NOT_CONVERGED), (b, r.status)
        _check_vs_oracle(orc, sp, r, B.job_seed(7, b))


def test_batch_c2_matches_oracle(orc):
    specs = _mixed(6, seed=12, lo=20, hi=90, dtypes=("f64",))
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=1, pivot="c2")
    for b, (sp, r) in enumerate(zip(specs, res)):
        _check_vs_oracle(orc, sp, r, B.job_seed(1, b), mode="c2")


def test_dense_jobs_equal_single_jobs():
    """Dense jobs: the same FMA chain and exact draws as rplu_dense, so
    identical pivots and factors."""
    specs = [sp for sp in _mixed(24, seed=3, lo=16, hi=200) if sp["kind"] == "dense"]
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=5)
    for b, (sp, r) in enumerate(zip(specs, res)):
        A = _matrix(sp)
        single = rp.rplu_dense(torch.from_numpy(np.ascontiguousarray(A)).cuda(), min(A.shape),
                               seed=B.job_seed(5, b), rel_tol=1e-6)
        sI, sJ = to_np(single.I), to_np(single.J)
        same = 0
        while same < min(r.k_done, single.k_done) and r.I[same] == sI[same] and r.J[same] == sJ[same]:
            same += 1
        assert same == r.k_done == single.k_done, (b, same, r.k_done, single.k_done)
        assert np.array_equal(r.L, to_np(single.L)) and np.array_equal(r.U, to_np(single.U)), b


def _generator_form_single(sp, seed):
    """The job run alone through rplu_cauchy_like with unit generators."""
    dt = sp["dtype"]
    x = torch.from_numpy(np.ascontiguousarray(np.asarray(sp["x"]).astype(NDT[dt]))).cuda()
    y = torch.from_numpy(np.ascontiguousarray(np.asarray(sp["y"]).astype(NDT[dt]))).cuda()
    n, m = x.numel(), y.numel()
    G = torch.ones((n, 1), dtype=TDT[dt], device="cuda")
    Bm = torch.ones((1, m), dtype=TDT[dt], device="cuda")
    return rp.rplu_cauchy_like(x, y, G, Bm, min(n, m), seed=seed, rel_tol=1e-6)


@pytest.mark.parametrize("dt", ["f32", "f64", "c64"])
def test_cauchy_jobs_equal_the_generator_form(orc, dt):
    """Cauchy jobs run the generator form in the batch kernel: the pivot rows
    and columns, multipliers and generator updates are those of
    rplu_cauchy_like with unit generators, operation for operation, so the
    factors agree bit for bit as long as the pivots do; the squared row norms
    are summed in another order, so the pivots must agree up to the first step
    the FP64 oracle flags as a near-tie at the working precision."""
    if dt == "c64":
        blocks = W.cauchy_disk_blocks(10, seed=21, size_lo=24, size_hi=240)
    else:
        blocks = W.cauchy_interval_blocks(10, seed=21, size_lo=24, size_hi=240)
    specs = [dict(kind="cauchy", x=b.x, y=b.y, dtype=dt) for b in blocks]
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=13)
    for b, (sp, r) in enumerate(zip(specs, res)):
        g = _generator_form_single(sp, B.job_seed(13, b))
        gI, gJ = to_np(g.I), to_np(g.J)
        same = 0
        while same < min(r.k_done, g.k_done) and r.I[same] == gI[same] and r.J[same] == gJ[same]:
            same += 1
        A = _oracle_matrix_c64(sp) if dt == "c64" else _matrix(sp).astype(np.float64)
        o = orc.rplu_dense(A, min(A.shape), seed=B.job_seed(13, b), tol=1e-6)
        _, tie = agreed_prefix(r, o, TIE[dt], residual_scaled=True)
        assert same >= min(tie, r.k_done, g.k_done), (b, same, tie)
        assert np.array_equal(r.L[:, :same], to_np(g.L)[:, :same]), b
        assert np.array_equal(r.U[:same], to_np(g.U)[:same]), b
        if same == r.k_done == g.k_done:
            assert r.rel_res == pytest.approx(np.sqrt(g.T[-1] / g.T[0]), rel=1e-4, abs=1e-9)


def test_shape_and_neighbours_do_not_change_results():
    specs = _to_device(_mixed(40, seed=21, lo=8, hi=300))
    base = B.BatchPlan(specs, rel_tol=1e-6, seed=3, tune=False)
    base.run()
    assert base.wait() in (rp.RPLU_OK, rp.RPLU_NOT_CONVERGED)
    ref = base.results()
    tuned = B.BatchPlan(specs, rel_tol=1e-6, seed=3, tune=True)
    tuned.run()
    tuned.wait()
    shp = tuned.shape()
    assert shp["threads"] in (128, 256) and shp["tile_rows"] in (4, 8) and shp["write_back"] in (4, 6, 8)
    for a, b in zip(ref, tuned.results()):
        assert a.k_done == b.k_done and torch.equal(a.I, b.I) and torch.equal(a.L, b.L) and torch.equal(a.U, b.U)
    # each job alone (its own seed) equals the same job inside the batch
    for b in (0, 7, 39):
        sp = dict(specs[b])
        sp["seed"] = B.job_seed(3, b)
        alone = B.rplu_batch([sp], rel_tol=1e-6)[0]
        assert alone.k_done == ref[b].k_done
        assert torch.equal(alone.I, ref[b].I) and torch.equal(alone.L, ref[b].L) and torch.equal(alone.U, ref[b].U)
    base.close()
    tuned.close()


def test_plan_replay_and_host_path_agree():
    host_specs = _mixed(10, seed=5, lo=30, hi=160)
    specs = _to_device(host_specs)
    plan = B.BatchPlan(specs, rel_tol=1e-6, seed=9)
    plan.run()
    plan.wait()
    first = plan.results()
    plan.run()
    plan.run()
    plan.wait()
    again = plan.results()
    host = B.rplu_batch(host_specs, rel_tol=1e-6, seed=9)
    for a, b, h in zip(first, again, host):
        assert a.k_done == b.k_done == h.k_done
        assert torch.equal(a.L, b.L) and torch.equal(a.U, b.U)
        assert np.array_equal(to_np(a.I), h.I) and np.array_equal(to_np(a.L), h.L) and np.array_equal(to_np(a.U), h.U)
    plan.close()


def test_edge_cases(orc):
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, 9)
    y = np.concatenate([rng.uniform(4, 5, 6), [x[3]]])  # x_3 == y_6: an infinite entry
    big_dense = W.gaussian(4100, 5, seed=1)              # n > 4096: single-job path
    specs = [
        dict(kind="dense", A=W.gaussian(1, 1, seed=2), dtype="f64"),
        dict(kind="dense", A=W.gaussian(3, 130, seed=3), dtype="f32"),   # ragged: m % 4 != 0
        dict(kind="dense", A=W.gaussian(130, 3, seed=4), dtype="f64"),
        dict(kind="cauchy", x=x, y=y, dtype="f32"),                      # invalid (x_i == y_j)
        dict(kind="dense", A=np.zeros((5, 6)), dtype="f32"),             # zero matrix: stops at once
        dict(kind="dense", A=W.lowrank_product(40, 30, 3, seed=5), dtype="f64"),  # exact rank 3
        dict(kind="dense", A=big_dense, dtype="f64"),
    ]
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=4)
    assert res[3].status == rp.RPLU_ERR_INVALID and res[3].k_done == 0
    assert res[4].status == rp.RPLU_OK and res[4].k_done == 0 and res[4].rel_res == 0.0
    assert res[5].status == rp.RPLU_OK and res[5].k_done == 3
    for b in (0, 1, 2, 5, 6):
        assert res[b].status in (rp.RPLU_OK, rp.RPLU_NOT_CONVERGED), b
        _check_vs_oracle(orc, specs[b], res[b], B.job_seed(4, b))
    # k_max = 0 and rel_tol = 0 (exactly k_max steps)
    r0 = B.rplu_batch([specs[1]], k_max=0)[0]
    assert r0.status == rp.RPLU_OK and r0.k_done == 0
    rk = B.rplu_batch([dict(specs[2], rel_tol=0.0)], k_max=3, seed=2)[0]
    assert rk.k_done == 3
    o = orc.rplu_dense(_matrix(specs[2]), 3, seed=B.job_seed(2, 0))
    assert np.array_equal(rk.I, o["I"]) and np.array_equal(rk.J, o["J"])


def test_full_size_cauchy_blocks_sampled(orc):
    """4096 real Cauchy blocks, n, m ~ U{64..1024}, separated unit intervals, rank to
    1e-6 relative error, FP32: sampled jobs against the oracle, explicit error of every
    sampled factorization, and the reported residual of every job."""
    blocks = W.cauchy_interval_blocks(4096, seed=2026)
    specs = [dict(kind="cauchy", x=b.x, y=b.y, dtype="f32") for b in blocks]
    dspecs = _to_device(specs)
    plan = B.BatchPlan(dspecs, rel_tol=1e-6, seed=1)
    plan.run()
    st = plan.wait()
    res = plan.results()
    assert st == rp.RPLU_OK
    assert all(r.status == rp.RPLU_OK for r in res)
    rr = np.array([r.rel_res for r in res])
    assert np.all(rr <= 1e-6)
    ks = np.array([r.k_done for r in res])
    assert ks.min() >= 1 and ks.max() < 64
    rng = np.random.default_rng(0)
    for b in rng.choice(len(specs), 12, replace=False):
        r = res[b]
        A = _matrix(specs[b])
        err = np.linalg.norm(A.astype(np.float64) - to_np(r.L).astype(np.float64) @ to_np(r.U).astype(np.float64))
        assert err / np.linalg.norm(A.astype(np.float64)) <= 2e-6
        o = orc.rplu_dense(A.astype(np.float64), min(A.shape), seed=B.job_seed(1, int(b)), tol=1e-6)
        same, tie = agreed_prefix(r, o, TIE["f32"], residual_scaled=True)
        assert same >= min(tie, len(o["I"])), (b, same, tie)
        assert_factors(r, o, same, GPU_TOL["f32"])
    plan.close()


def test_points_at_extreme_scales():
    """FP32 Cauchy jobs whose point sets are far apart or huge: every entry
    finite, the factorization accurate against the oracle."""
    rng = np.random.default_rng(8)
    far = dict(kind="cauchy", x=np.r_[rng.uniform(1e18, 2e18, 20), rng.uniform(-1, 1, 40)],
               y=np.r_[rng.uniform(-2e18, -1e18, 12), rng.uniform(3, 5, 45)], dtype="f32")
    near = dict(kind="cauchy", x=rng.uniform(-1, 1, 70), y=rng.uniform(3, 5, 66), dtype="f32")
    res = B.rplu_batch([far, near], rel_tol=1e-6, seed=2)
    for b, (sp, r) in enumerate(zip([far, near], res)):
        A = _matrix(sp).astype(np.float64)
        assert np.all(np.isfinite(A))
        assert r.status == rp.RPLU_OK and r.k_done >= 1
        err = np.linalg.norm(A - r.L.astype(np.float64) @ r.U.astype(np.float64)) / np.linalg.norm(A)
        assert err <= 2e-6, (b, err)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_host_cauchy_batch_equals_device_batch(dt):
    """Host Cauchy jobs of one dtype go through the vectorized marshalling, the
    bulk copies (one pinned copy in, one gathered copy out) and packed result
    views; every job equals the same job given as device tensors, bit for bit."""
    blocks = W.cauchy_interval_blocks(64, seed=17, size_lo=16, size_hi=300)
    host = [dict(kind="cauchy", x=b.x.astype(NDT[dt]), y=b.y.astype(NDT[dt]), dtype=dt) for b in blocks]
    dev = _to_device(host)
    for call in range(2):
        hr = B.rplu_batch(host, rel_tol=1e-6, seed=4)
        dr = B.rplu_batch(dev, rel_tol=1e-6, seed=4)
        for b, (h, d) in enumerate(zip(hr, dr)):
            assert h.status == d.status and h.k_done == d.k_done >= 1, (call, b)
            assert np.array_equal(h.I, to_np(d.I)) and np.array_equal(h.J, to_np(d.J)), (call, b)
            assert np.array_equal(h.L, to_np(d.L)) and np.array_equal(h.U, to_np(d.U)), (call, b)
            assert h.rel_res == d.rel_res


def _complex_mix(n_jobs, seed, lo=16, hi=200):
    """Complex64 jobs: Cauchy blocks on separated unit disks, and dense
    complex matrices with a decaying spectrum."""
    blocks = W.cauchy_disk_blocks(n_jobs, seed=seed, size_lo=lo, size_hi=hi)
    specs = []
    for b, blk in enumerate(blocks):
        if b % 3 == 2:
            n, m = len(blk.x), len(blk.y)
            A = W.dense_haar_decay(n, m, 0.7, seed=b) + 1j * W.dense_haar_decay(n, m, 0.7, seed=b + 1000)
            specs.append(dict(kind="dense", A=A, dtype="c64"))
        else:
            specs.append(dict(kind="cauchy", x=blk.x, y=blk.y, dtype="c64"))
    return specs


def _oracle_matrix_c64(spec):
    """The complex64 job's matrix in complex128: the rounded dense entries, or
    1/(x_i - y_j) of the complex64 points."""
    if spec["kind"] == "dense":
        return np.asarray(spec["A"]).astype(np.complex64).astype(np.complex128)
    x = np.asarray(spec["x"]).astype(np.complex64).astype(np.complex128)
    y = np.asarray(spec["y"]).astype(np.complex64).astype(np.complex128)
    return 1.0 / (x[:, None] - y[None, :])


def test_complex64_jobs_match_oracle(orc):
    """Complex64 Cauchy (separated disks) and dense jobs against the oracle on
    the same points or entries: pivots up to the FP32 near-tie window, the
    residual rows and columns to 1e-5, and the reported residual."""
    specs = _complex_mix(18, seed=31)
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=3)
    for b, (sp, r) in enumerate(zip(specs, res)):
        assert r.status in (rp.RPLU_OK, rp.RPLU_NOT_CONVERGED), (b, r.status)
        A = _oracle_matrix_c64(sp)
        o = orc.rplu_dense(A, min(A.shape), seed=B.job_seed(3, b), tol=1e-6)
        upto = assert_pivots(r, o, TIE["c64"], min_steps=0, residual_scaled=True)
        assert_factors(r, o, upto, GPU_TOL["c64"])
        if sp["kind"] == "cauchy":
            err = np.linalg.norm(A - to_np(r.L).astype(np.complex128) @ to_np(r.U).astype(np.complex128))
            assert err <= 2e-6 * np.linalg.norm(A), (b, err / np.linalg.norm(A))


def test_complex64_dense_jobs_equal_single_jobs():
    """Dense complex64 jobs: the batch kernel's update chain, draws and FP64
    complex multipliers equal rplu_dense's, bit for bit."""
    specs = [sp for sp in _complex_mix(24, seed=8, lo=20, hi=180) if sp["kind"] == "dense"]
    res = B.rplu_batch(specs, rel_tol=1e-6, seed=6)
    for b, (sp, r) in enumerate(zip(specs, res)):
        A = np.ascontiguousarray(np.asarray(sp["A"]).astype(np.complex64))
        single = rp.rplu_dense(torch.from_numpy(A).cuda(), min(A.shape), seed=B.job_seed(6, b), rel_tol=1e-6)
        assert r.k_done == single.k_done, b
        assert np.array_equal(r.I, to_np(single.I)) and np.array_equal(r.J, to_np(single.J)), b
        assert np.array_equal(r.L, to_np(single.L)) and np.array_equal(r.U, to_np(single.U)), b


def test_complex64_job_alone_equals_in_mix():
    """A complex64 job's result does not depend on the batch around it
    (real and complex jobs in one call: one persistent launch per type)."""
    cspecs = _complex_mix(12, seed=40)
    mixed = cspecs + _mixed(8, seed=41)
    res = B.rplu_batch(mixed, rel_tol=1e-6, seed=9)
    for b in (0, 4, 5, 11):
        sp = dict(cspecs[b])
        sp["seed"] = B.job_seed(9, b)
        alone = B.rplu_batch([sp], rel_tol=1e-6)[0]
        assert alone.k_done == res[b].k_done >= 1
        assert np.array_equal(alone.I, res[b].I) and np.array_equal(alone.L, res[b].L)
        assert np.array_equal(alone.U, res[b].U)
    dev = _to_device(cspecs)
    dres = B.rplu_batch(dev, rel_tol=1e-6, seed=9)
    for b in range(len(cspecs)):
        assert np.array_equal(to_np(dres[b].L), res[b].L) and np.array_equal(to_np(dres[b].U), res[b].U), b


def test_packed_ranges_equal_per_job_specs():
    """Cauchy jobs given as ranges of two packed host arrays give the same
    results, bit for bit, as the same jobs given one spec each."""
    blocks = W.cauchy_interval_blocks(40, seed=31, size_lo=16, size_hi=700)
    specs = [dict(kind="cauchy", x=b.x.astype(np.float32), y=b.y.astype(np.float32), dtype="f32") for b in blocks]
    ref = B.rplu_batch(specs, rel_tol=1e-6, seed=8)
    X = np.concatenate([sp["x"] for sp in specs])
    Y = np.concatenate([sp["y"] for sp in specs])
    res = B.rplu_batch_cauchy_packed(X, Y, [len(sp["x"]) for sp in specs], [len(sp["y"]) for sp in specs],
                                     rel_tol=1e-6, seed=8)
    assert len(res) == len(ref)
    for a, b in zip(res, ref):
        assert a.k_done == b.k_done and a.status == b.status
        assert np.array_equal(a.I, b.I) and np.array_equal(a.J, b.J)
        assert np.array_equal(a.L, b.L) and np.array_equal(a.U, b.U)


def test_packed_outputs_reused_equal_fresh_ones():
    """A call writing into an earlier call's output arrays (out=) gives the
    same factors, bit for bit, as one with fresh arrays, whatever the earlier
    call left in them (there: another seed and tolerance, other ranks)."""
    blocks = W.cauchy_interval_blocks(60, seed=17, size_lo=16, size_hi=600)
    X = np.concatenate([b.x for b in blocks]).astype(np.float32)
    Y = np.concatenate([b.y for b in blocks]).astype(np.float32)
    n, m = [len(b.x) for b in blocks], [len(b.y) for b in blocks]
    fresh = B.rplu_batch_cauchy_packed(X, Y, n, m, rel_tol=1e-5, seed=21)
    first = B.rplu_batch_cauchy_packed(X, Y, n, m, rel_tol=1e-7, seed=4)
    assert not np.array_equal(first.k_done, fresh.k_done)
    again = B.rplu_batch_cauchy_packed(X, Y, n, m, rel_tol=1e-5, seed=21, out=first)
    assert np.array_equal(again.k_done, fresh.k_done) and np.array_equal(again.status, fresh.status)
    for a, b in zip(again, fresh):
        assert np.array_equal(a.I, b.I) and np.array_equal(a.J, b.J)
        assert np.array_equal(a.L, b.L) and np.array_equal(a.U, b.U)
        assert a.rel_res == b.rel_res


def _hinted(specs_or_points, mem, out=None):
    """rplu_batch over host jobs with the job table's memory hint set to `mem`:
    packed Cauchy ranges (X, Y, n, m) into packed outputs, or dict specs."""
    from paper_2601_22344_gb300.binding import Job, lib
    o = B._opts("random", None)
    if isinstance(specs_or_points, tuple):
        X, Y, n, m = specs_or_points
        arr = (Job * len(n))()
        keep, packed = B._fill_packed(arr, X, Y, n, m, "f32", 1e-6, 7, None, out)
        B._job_view(arr, len(n))["memory"] = mem
        lib.rplu_batch(arr, len(n), ctypes.byref(o))
        return B.PackedResults(arr, packed, len(n))
    arr = (Job * len(specs_or_points))()
    keep, outs = B._fill(arr, specs_or_points, 1e-6, 7, None)
    B._job_view(arr, len(specs_or_points))["memory"] = mem
    lib.rplu_batch(arr, len(specs_or_points), ctypes.byref(o))
    return B._results(arr, outs)


def test_host_memory_hints_give_equal_results():
    """The memory hint changes only how host buffers move: asked per pointer
    (0), staged through pinned buffers (1), or read and written in place by
    the device where it reaches pageable host memory (3) -- the same factors
    bit for bit, into fresh and into reused output arrays, for packed Cauchy
    ranges and for dense and Cauchy jobs of every type given one spec each."""
    blocks = W.cauchy_interval_blocks(50, seed=23, size_lo=8, size_hi=500)
    X = np.concatenate([b.x for b in blocks]).astype(np.float32)
    Y = np.concatenate([b.y for b in blocks]).astype(np.float32)
    pts = (X, Y, np.array([len(b.x) for b in blocks]), np.array([len(b.y) for b in blocks]))
    rng = np.random.default_rng(4)
    specs = []
    for q, (lo, hi) in enumerate([(3, 40), (30, 300), (200, 700)]):
        n, m = int(rng.integers(lo, hi)), int(rng.integers(lo, hi))
        for dt in ("f32", "f64", "c64"):
            A = W.dense_haar_decay(n, m, 0.8, seed=q)
            if dt == "c64":
                A = A + 1j * W.dense_haar_decay(n, m, 0.8, seed=q + 50)
            specs.append(dict(kind="dense", A=A, dtype=dt))
    specs += [dict(kind="cauchy", x=b.x, y=b.y, dtype="f64") for b in blocks[:6]]

    def same(a, b):
        assert a.k_done == b.k_done and a.status == b.status and a.rel_res == b.rel_res
        assert np.array_equal(a.I, b.I) and np.array_equal(a.J, b.J)
        assert np.array_equal(a.L, b.L) and np.array_equal(a.U, b.U)

    for inputs in (pts, specs):
        ref = _hinted(inputs, 1)
        for mem in (0, 3):
            for res in (_hinted(inputs, mem),) + ((_hinted(pts, mem, out=_hinted(pts, mem)),) if inputs is pts else ()):
                assert len(res) == len(ref)
                for a, b in zip(res, ref):
                    same(a, b)
