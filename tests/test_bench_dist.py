"""Host logic of bench.py, without a GPU: the cross-rank aggregation (max of
times, sum of units) on a 2-rank gloo process group; a failing secondary
section reported in its object; the generated matvec's roofline arithmetic;
the sampled error estimates of the Toeplitz and sparse sections against
explicit errors on small cases."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx = bench.reduce_scalar(1.5 + rank, "max")
        sm = bench.reduce_scalar(2.0, "sum")
        bench.barrier()
        q.put((rank, mx, sm, bench._dist()))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, d in res:
        assert mx == 2.5 and sm == 4.0
        assert d == (2, rank, rank)


def test_reduce_without_group_is_identity():
    import bench
    assert bench.reduce_scalar(3.0, "max") == 3.0


def test_secondary_section_error_is_reported_not_raised(capsys):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    def ok(a, b=0):
        return {"v": a + b}

    def bad():
        raise RuntimeError("planted")

    assert bench._section(ok, 1, b=2) == {"v": 3}
    assert bench._section(bad) == {"error": "RuntimeError: planted"}
    assert "bad failed" in capsys.readouterr().err


def test_cauchy_matvec_roofline_arithmetic():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np

    import bench
    # 300 launches of 0.148 ms over 20000^2 entries at 2070 MHz on 152 SMs
    r = bench.cauchy_matvec_roofline(np.array([0.148 * 300, 300, 0, 3]), 20000, 20000, 2070.0, 152)
    assert r["achieved"] == pytest.approx(4e8 / 0.148e-3 / 1e9)
    assert r["peak"] == pytest.approx(152 * 12.8 * 2.07e9 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "alu" and r["unit"] == "G entries/s"
    assert "error" in bench.cauchy_matvec_roofline(np.zeros(4), 10, 10, None, 152)


def test_toeplitz_sampled_error_estimates_the_explicit_error():
    """The bench's sampled error of a Toeplitz CUR factorization (entries from
    the kernel formula) tracks the explicit error on the oracle's matrix."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np

    import bench
    from oracle import cur_form as CF
    N, L = 6, 320.0
    op = CF.KroneckerToeplitz(N, length=L)
    o = CF.rplu_cur(op, 30, seed=2)
    A = op.dense().real
    I, J, C = o["I"], o["J"], o["core"].real
    exact = np.linalg.norm(A - A[:, J] @ C @ A[I, :]) / np.linalg.norm(A)
    est = bench.toeplitz_sampled_error(N, L, I, J, C, n_sample=400, seed=1)
    assert abs(est - exact) <= 0.15 * exact


def test_sparse_sampled_error_estimates_the_explicit_error():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np

    import bench
    import workloads as W
    from oracle import cur_form as CF
    S = W.chung_lu_graph(400, avg_degree=5.0, exponent=2.3, seed=6)
    o = CF.rplu_cur(CF.SparseOperator(S), 60, seed=2)
    A = S.toarray()
    I, J, C = o["I"], o["J"], o["core"].real
    exact_on_support = A - A[:, J] @ C @ A[I, :]
    est = bench.sparse_sampled_error(S, I, J, C, n_sample=3000, seed=1)
    # the sample draws half its entries from the nonzeros, so it weighs them more than
    # the Frobenius norm does: compare with the same mixture computed exactly
    nz = A != 0
    mix = np.sqrt((np.mean(exact_on_support[nz] ** 2) + np.mean(exact_on_support ** 2))
                  / (np.mean(A[nz] ** 2) + np.mean(A ** 2)))
    assert abs(est - mix) <= 0.2 * mix


def test_reference_arm_line_on_a_small_case(capsys):
    """The reference arm's line on a small workload: it honours --warmup and
    --steps, states the timed k and the extrapolation factor apart from the
    value, and extrapolates the factorization time linearly in k."""
    import json

    import bench
    bench.main(["--impl", "reference", "--dense-n", "192", "--dense-k", "6", "--cauchy-n", "150",
                "--cauchy-k", "4", "--steps", "2", "--warmup", "2"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 2
    ex = line["extrapolation"]
    assert ex["timed_k"] == {"dense": 1, "cauchy": 1} and ex["full_k"] == {"dense": 6, "cauchy": 4}
    assert ex["dense_threads"] >= 1 and ex["cauchy_threads"] >= 1
    td = ex["dense_init_s"] + 6 * ex["dense_step_s"]
    tc = ex["cauchy_init_s"] + 4 * ex["cauchy_step_s"]
    assert line["value"] == pytest.approx(2.0 / (td / ex["dense_threads"] + tc / ex["cauchy_threads"]), rel=1e-9)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("dense FP32 192x192 k=6")
