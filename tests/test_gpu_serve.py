"""Serving sessions (rplu_session_*) through the C-ABI: continuous batching
returns, for every request, the same result as the request run alone;
admission waits for device memory; cancellation of queued and running
requests; idle kernel exit and relaunch; invalid requests fail alone."""
import time

import numpy as np
import pytest

import workloads as W
from parity import to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)
from paper_2601_22344_gb300 import batch as B  # noqa: E402
from paper_2601_22344_gb300 import serve as S  # noqa: E402


def _requests(n_req, seed, lo=32, hi=400):
    blocks = W.cauchy_interval_blocks(n_req, seed=seed, size_lo=lo, size_hi=hi)
    reqs = []
    for b, blk in enumerate(blocks):
        if b % 3 == 2:
            A = W.dense_haar_decay(len(blk.x), len(blk.y), 0.8, seed=b).astype(np.float32)
            reqs.append(dict(kind="dense", A=torch.from_numpy(A).cuda(), seed=1000 + b))
        else:
            reqs.append(dict(kind="cauchy", x=torch.from_numpy(blk.x.astype(np.float32)).cuda(),
                             y=torch.from_numpy(blk.y.astype(np.float32)).cuda(), seed=1000 + b))
    return reqs


def _alone(spec, k_max=None):
    sp = dict(spec)
    sp["dtype"] = "f32"
    return B.rplu_batch([sp], rel_tol=1e-6, k_max=k_max)[0]


def _same(res, ref):
    I, J, L, U = res
    return (np.array_equal(to_np(I), to_np(ref.I)) and np.array_equal(to_np(J), to_np(ref.J))
            and np.array_equal(to_np(L), to_np(ref.L)) and np.array_equal(to_np(U), to_np(ref.U)))


def test_results_in_the_mix_equal_results_alone():
    reqs = _requests(60, seed=3)
    big = dict(kind="dense", A=torch.from_numpy(W.dense_haar_decay(1100, 300, 0.8, seed=9).astype(np.float32)).cuda(),
               seed=77)
    s = S.Session(max_dim=1024)
    tickets = []
    for q, r in enumerate(reqs[:30]):  # first wave
        tickets.append(s.submit(r))
    tickets.append(s.submit(big))
    time.sleep(0.002)
    for r in reqs[30:]:  # arrives while the first wave is on the GPU
        tickets.append(s.submit(r))
    infos = [s.wait(t, timeout_s=60) for t in tickets]
    assert all(i.state == S.DONE and i.status == rp.RPLU_OK for i in infos), [(i.state, i.status) for i in infos]
    allreq = reqs[:30] + [big] + reqs[30:]
    for t, r, i in zip(tickets, allreq, infos):
        res = s.fetch(t)
        assert len(res[0]) == i.k_done
        if r is big:
            ref = rp.rplu_dense(r["A"], 300, seed=77, rel_tol=1e-6)
            assert i.k_done == ref.k_done and _same(res, ref)
        else:
            ref = _alone(r)
            assert i.k_done == ref.k_done and _same(res, ref), t
            assert i.rel_res == pytest.approx(ref.rel_res, rel=1e-12)
    st = s.stats()
    assert st["completed"] == len(tickets) and st["large_completed"] == 1 and st["arena_used"] == 0
    s.close()


def test_admission_waits_for_memory():
    reqs = _requests(24, seed=5, lo=200, hi=400)
    s = S.Session(hbm_budget=8 << 20, max_dim=512)  # a few requests at a time
    tickets = [s.submit(r) for r in reqs]
    infos, results = [], []
    for t in tickets:  # fetch as they finish: the factors hold arena memory until fetched
        infos.append(s.wait(t, timeout_s=60))
        results.append(s.fetch(t))
    assert all(i.state == S.DONE and i.status == rp.RPLU_OK for i in infos)
    assert max(i.queue_ms for i in infos) > 0.0
    for res, r in zip(results, reqs):
        assert _same(res, _alone(r))
    assert s.stats()["arena_used"] == 0
    s.close()


def test_cancel_queued_and_running():
    rng = np.random.default_rng(4)
    A = torch.from_numpy(rng.standard_normal((1000, 1000)).astype(np.float32)).cuda()  # full rank: 1000 steps
    s = S.Session(hbm_budget=32 << 20, max_dim=1024, dense_kernel_cells=1 << 20)  # runs in the kernel
    long_t = s.submit(dict(kind="dense", A=A, seed=5, rel_tol=0.0))
    queued = [s.submit(dict(kind="dense", A=A, seed=6 + q, rel_tol=0.0)) for q in range(6)]  # memory-bound queue
    for _ in range(2000):
        if s.poll(long_t).state == S.RUNNING:
            break
        time.sleep(0.001)
    s.cancel(long_t)
    s.cancel(queued[-1])
    i = s.wait(long_t, timeout_s=60)
    assert i.state == S.CANCELLED and i.status == rp.RPLU_CANCELLED and 0 <= i.k_done < 1000
    iq = s.wait(queued[-1], timeout_s=60)
    assert iq.state == S.CANCELLED and iq.k_done == 0
    I, J, L, U = s.fetch(long_t)
    if i.k_done > 0:  # the steps done before the cancel are those of the uncancelled run
        ref = _alone(dict(kind="dense", A=A, seed=5, rel_tol=0.0), k_max=i.k_done)
        assert np.array_equal(to_np(I), to_np(ref.I)) and np.array_equal(to_np(U), to_np(ref.U))
    for t in queued[:-1]:
        s.cancel(t)
    for t in queued[:-1]:
        s.wait(t, timeout_s=120)
    s.close()


def test_idle_kernel_exits_and_is_relaunched():
    """CTAs wait for requests with a bounded wait; with nothing published it
    runs out, the kernel ends, and the next request relaunches it."""
    reqs = _requests(4, seed=8)
    s = S.Session(idle_us=50.0)
    a = s.submit(reqs[0])
    assert s.wait(a, timeout_s=30).status == rp.RPLU_OK
    time.sleep(0.05)  # far longer than the idle limit: every CTA has exited
    b = s.submit(reqs[1])
    assert s.wait(b, timeout_s=30).status == rp.RPLU_OK
    assert s.stats()["kernel_launches"] >= 2
    assert _same(s.fetch(b), _alone(reqs[1]))
    s.close()


def test_invalid_request_fails_alone():
    reqs = _requests(6, seed=9)
    x = np.linspace(-1, 1, 50).astype(np.float32)
    y = np.r_[np.linspace(3, 4, 40), [x[7]]].astype(np.float32)  # x_7 == y_40
    bad = dict(kind="cauchy", x=torch.from_numpy(x).cuda(), y=torch.from_numpy(y).cuda(), seed=3)
    s = S.Session()
    ts = [s.submit(r) for r in reqs[:3]] + [s.submit(bad)] + [s.submit(r) for r in reqs[3:]]
    infos = [s.wait(t, timeout_s=30) for t in ts]
    assert infos[3].status == rp.RPLU_ERR_INVALID and infos[3].k_done == 0
    for t, r, i in zip(ts[:3] + ts[4:], reqs, infos[:3] + infos[4:]):
        assert i.status == rp.RPLU_OK and _same(s.fetch(t), _alone(r))
    with pytest.raises(rp.RPLUError):
        s.submit(dict(kind="dense", A=torch.zeros((3, 0), device="cuda")))
    s.close()


def _complex_requests(n_req, seed, lo=32, hi=400):
    """Complex64 requests: Cauchy blocks on separated disks and on spiral
    clouds, and dense complex matrices."""
    disks = W.cauchy_disk_blocks(n_req, seed=seed, size_lo=lo, size_hi=hi)
    reqs = []
    for b, blk in enumerate(disks):
        if b % 4 == 3:
            n, m = len(blk.x), len(blk.y)
            A = (W.dense_haar_decay(n, m, 0.8, seed=b) + 1j * W.dense_haar_decay(n, m, 0.8, seed=b + 50))
            reqs.append(dict(kind="dense", A=torch.from_numpy(A.astype(np.complex64)).cuda(), seed=2000 + b))
        elif b % 4 == 2:
            x, y = W.cauchy_spirals(len(blk.x), len(blk.y), seed=b)
            reqs.append(dict(kind="cauchy", x=torch.from_numpy(x.astype(np.complex64)).cuda(),
                             y=torch.from_numpy(y.astype(np.complex64)).cuda(), seed=2000 + b))
        else:
            reqs.append(dict(kind="cauchy", x=torch.from_numpy(blk.x.astype(np.complex64)).cuda(),
                             y=torch.from_numpy(blk.y.astype(np.complex64)).cuda(), seed=2000 + b))
    return reqs


def test_complex_and_real_requests_in_the_mix_equal_results_alone():
    """Complex64 requests share the session (and its one persistent kernel)
    with FP32 ones; every result equals the request run alone -- rplu_batch for
    the kernel-sized ones, rplu_cauchy_like with unit generators for a Cauchy
    request above cauchy_max_dim -- bit for bit."""
    creqs = _complex_requests(24, seed=12)
    rreqs = _requests(16, seed=13)
    xb, yb = W.cauchy_spirals(1400, 900, seed=5)
    big = dict(kind="cauchy", x=torch.from_numpy(xb.astype(np.complex64)).cuda(),
               y=torch.from_numpy(yb.astype(np.complex64)).cuda(), seed=99)
    s = S.Session(max_dim=1024, cauchy_max_dim=1024)
    order = creqs[:12] + rreqs[:8] + [big] + creqs[12:] + rreqs[8:]
    tickets = []
    for q, r in enumerate(order):
        tickets.append(s.submit(r))
        if q == 20:
            time.sleep(0.002)  # the rest arrives while the first requests are on the GPU
    infos = [s.wait(t, timeout_s=120) for t in tickets]
    assert all(i.state == S.DONE and i.status == rp.RPLU_OK for i in infos), [(i.state, i.status) for i in infos]
    for t, r, i in zip(tickets, order, infos):
        res = s.fetch(t)
        if r is big:
            ones_x = torch.ones((1400, 1), dtype=torch.complex64, device="cuda")
            ones_y = torch.ones((1, 900), dtype=torch.complex64, device="cuda")
            ref = rp.rplu_cauchy_like(r["x"], r["y"], ones_x, ones_y, 900, seed=99, rel_tol=1e-6)
            assert i.k_done == ref.k_done and _same(res, ref)
            continue
        cplx = r["kind"] == "dense" and r["A"].is_complex() or r["kind"] == "cauchy" and r["x"].is_complex()
        sp = dict(r)
        sp["dtype"] = "c64" if cplx else "f32"
        ref = B.rplu_batch([sp], rel_tol=1e-6)[0]
        assert i.k_done == ref.k_done and _same(res, ref), t
        assert i.rel_res == pytest.approx(ref.rel_res, rel=1e-12)
    st = s.stats()
    assert st["completed"] == len(tickets) and st["large_completed"] == 1 and st["arena_used"] == 0
    s.close()


def test_large_cauchy_requests_with_bounds():
    """With bound_nu, Cauchy requests above cauchy_max_dim take Algorithm 3 on
    the large-request streams: the factors equal rplu_cauchy_like's with unit
    generators, the same bound_nu and seed, bit for bit, and rel_res is the
    exact relative residual (||A||_F from an exact-norm pass, not the bounds)."""
    xs, ys = W.cauchy_spirals(2400, 1800, seed=6)
    blk = W.cauchy_interval_blocks(1, seed=8, size_lo=1500, size_hi=2500)[0]
    bigs = [dict(kind="cauchy", x=torch.from_numpy(xs.astype(np.complex64)).cuda(),
                 y=torch.from_numpy(ys.astype(np.complex64)).cuda(), seed=41),
            dict(kind="cauchy", x=torch.from_numpy(blk.x.astype(np.float32)).cuda(),
                 y=torch.from_numpy(blk.y.astype(np.float32)).cuda(), seed=42)]
    small = _requests(6, seed=24) + _complex_requests(4, seed=25)
    s = S.Session(cauchy_max_dim=1024, bound_nu=5.0)
    order = small[:5] + bigs[:1] + small[5:] + bigs[1:]
    tickets = [s.submit(r) for r in order]
    infos = [s.wait(t, timeout_s=120) for t in tickets]
    assert all(i.state == S.DONE and i.status == rp.RPLU_OK for i in infos), [(i.state, i.status) for i in infos]
    for t, r, i in zip(tickets, order, infos):
        res = s.fetch(t)
        if not any(r is b for b in bigs):
            continue
        x, y = r["x"], r["y"]
        n, m = x.numel(), y.numel()
        G = torch.ones((n, 1), dtype=x.dtype, device="cuda")
        Bm = torch.ones((1, m), dtype=x.dtype, device="cuda")
        ref = rp.rplu_cauchy_like(x, y, G, Bm, min(n, m), seed=r["seed"], rel_tol=1e-6, bound_nu=5.0)
        assert i.k_done == ref.k_done and _same(res, ref)
        e = rp.rplu_cauchy_like(x, y, G, Bm, 0, seed=r["seed"])
        assert i.rel_res == pytest.approx(float(np.sqrt(ref.T[-1] / e.T[0])), rel=1e-12)
        A = 1.0 / (x.to(torch.complex128)[:, None] - y.to(torch.complex128)[None, :])
        R = A - ref.L.to(torch.complex128) @ ref.U.to(torch.complex128)
        explicit = float(torch.linalg.norm(R) / torch.linalg.norm(A))
        assert abs(i.rel_res - explicit) <= 1e-3 * explicit + 1e-6
    assert s.stats()["large_completed"] == 2
    s.close()
    with pytest.raises(rp.RPLUError):
        S.Session(bound_nu=0.5)


def test_cauchy_requests_up_to_4096_run_in_the_kernel():
    """Cauchy requests up to n, m = 4096 (the generator form needs O(n + m)
    shared memory) run in the persistent kernel next to small dense ones, and
    equal rplu_batch alone bit for bit."""
    xs, ys = W.cauchy_spirals(3000, 2600, seed=21)
    xr = np.linspace(-1.0, 1.0, 4096).astype(np.float32)
    yr = np.linspace(4.0, 6.0, 4000).astype(np.float32)
    bigs = [dict(kind="cauchy", x=torch.from_numpy(xs.astype(np.complex64)).cuda(),
                 y=torch.from_numpy(ys.astype(np.complex64)).cuda(), seed=31),
            dict(kind="cauchy", x=torch.from_numpy(xr).cuda(), y=torch.from_numpy(yr).cuda(), seed=32)]
    small = _requests(12, seed=22) + _complex_requests(8, seed=23)
    order = small[:6] + bigs[:1] + small[6:14] + bigs[1:] + small[14:]
    s = S.Session()
    is_big = [any(r is b for b in bigs) for r in order]
    tickets = [s.submit(r, k_max=200 if big else None) for r, big in zip(order, is_big)]
    infos = [s.wait(t, timeout_s=120) for t in tickets]
    assert all(i.state == S.DONE and i.status in (rp.RPLU_OK, rp.RPLU_NOT_CONVERGED) for i in infos)
    for t, r, i, big in zip(tickets, order, infos, is_big):
        res = s.fetch(t)
        cplx = r["kind"] == "dense" and r["A"].is_complex() or r["kind"] == "cauchy" and r["x"].is_complex()
        sp = dict(r)
        sp["dtype"] = "c64" if cplx else "f32"
        ref = B.rplu_batch([sp], rel_tol=1e-6, k_max=200 if big else None)[0]
        assert i.k_done == ref.k_done and _same(res, ref), t
    st = s.stats()
    assert st["completed"] == len(tickets) and st["large_completed"] == 0 and st["arena_used"] == 0
    s.close()


def test_exited_ctas_are_replaced_while_a_launch_runs():
    """While one CTA of a launch still factors a long request and the others
    have gone idle and left, new requests get new CTAs (another launch beside
    the running one) instead of waiting for the long request to finish."""
    rng = np.random.default_rng(7)
    A = torch.from_numpy(rng.standard_normal((1000, 1000)).astype(np.float32)).cuda()  # full rank: 1000 steps
    s = S.Session(idle_us=50.0, max_dim=1024, dense_kernel_cells=1 << 20)
    long_t = s.submit(dict(kind="dense", A=A, seed=5, rel_tol=0.0))
    for _ in range(2000):
        if s.poll(long_t).state == S.RUNNING:
            break
        time.sleep(0.001)
    time.sleep(0.01)  # far longer than the idle limit: every other CTA of the launch has left
    n0 = s.stats()["kernel_launches"]
    reqs = _requests(24, seed=17)
    tickets = [s.submit(r) for r in reqs]
    infos = [s.wait(t, timeout_s=60) for t in tickets]
    assert all(i.state == S.DONE and i.status == rp.RPLU_OK for i in infos)
    assert s.poll(long_t).state == S.RUNNING  # they finished before the long request
    assert s.stats()["kernel_launches"] > n0
    for t, r in zip(tickets, reqs):
        assert _same(s.fetch(t), _alone(r))
    s.cancel(long_t)
    s.wait(long_t, timeout_s=60)
    s.close()
