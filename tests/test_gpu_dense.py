"""GPU parity of the dense form (rplu_dense through the C-ABI) against the
oracle, on the same seeded inputs and the same draws."""
import numpy as np
import pytest

import workloads as W
from parity import GPU_TOL, TIE, assert_factors, assert_pivots, rel_error, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)

TDT = {"f32": torch.float32, "f64": torch.float64, "c64": torch.complex64, "c128": torch.complex128}
NDT = {"f32": np.float32, "f64": np.float64, "c64": np.complex64, "c128": np.complex128}


def _dev(A, dt):
    return torch.from_numpy(np.ascontiguousarray(A.astype(NDT[dt]))).cuda()


def _oracle_input(A, dt):
    """The oracle runs in FP64/complex128 on exactly the values the GPU sees."""
    return A.astype(NDT[dt]).astype(np.complex128 if np.iscomplexobj(A) or dt.startswith("c") else np.float64)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_dense_haar_500x400_f64_parity(orc, seed):
    A = W.dense_haar_500x400()
    g = rp.rplu_dense(_dev(A, "f64"), 40, seed=seed)
    o = orc.rplu_dense(A, 40, seed=seed)
    assert g.k_done == o["k_done"] == 40
    upto = assert_pivots(g, o, TIE["f64"], min_steps=20)
    assert_factors(g, o, upto, GPU_TOL["f64"])
    if upto == 40:
        assert np.allclose(g.T, o["T"], rtol=1e-10, atol=0)


@pytest.mark.parametrize("dt", ["f64", "c128", "f32", "c64"])
@pytest.mark.parametrize("shape,k", [((1, 1), 1), ((37, 53), 20), ((53, 37), 37), ((130, 7), 7), ((7, 130), 7),
                                     ((401, 403), 30), ((1000, 3), 3), ((257, 129), 64)])
def test_ragged_shapes(orc, dt, shape, k):
    n, m = shape
    A = W.gaussian(n, m, seed=n * 1000 + m, complex_=dt.startswith("c"))
    Ao = _oracle_input(A, dt)
    g = rp.rplu_dense(_dev(A, dt), k, seed=5)
    o = orc.rplu_dense(Ao, k, seed=5)
    assert g.k_done == o["k_done"]
    upto = assert_pivots(g, o, TIE[dt], min_steps=min(k, 3) if dt in ("f64", "c128") else 1, residual_scaled=True)
    assert_factors(g, o, upto, GPU_TOL[dt])
    L, U, I, J = to_np(g.L), to_np(g.U), to_np(g.I), to_np(g.J)
    # exact structure: unit lower triangular L on the pivot rows, zeros in U on earlier pivot columns
    LI = L[I, :]
    assert np.all(np.diag(LI) == 1) and np.all(np.triu(LI, 1) == 0)
    assert np.all(np.tril(U[:, J], -1) == 0)


def test_host_buffers_and_strided_input(orc):
    A = W.gaussian(90, 70, seed=3)
    o = orc.rplu_dense(A, 12, seed=9)
    h = rp.rplu_dense(A, 12, seed=9)                      # numpy in, numpy out (staged)
    assert np.array_equal(h.I, o["I"]) and np.array_equal(h.J, o["J"])
    big = torch.zeros((90, 100), dtype=torch.float64, device="cuda")
    big[:, :70] = torch.from_numpy(A).cuda()
    s = rp.rplu_dense(big[:, :70], 12, seed=9)           # lda = 100
    assert np.array_equal(to_np(s.I), o["I"])
    assert np.array_equal(to_np(s.L), h.L) and np.array_equal(to_np(s.U), h.U)


def test_overwrite_input_matches_copy(orc):
    A = W.gaussian(120, 96, seed=4)
    ref = rp.rplu_dense(_dev(A, "f64"), 20, seed=2)
    t = _dev(A, "f64")
    g = rp.rplu_dense(t, 20, seed=2, overwrite_input=True)
    assert torch.equal(g.I, ref.I) and torch.equal(g.L, ref.L) and torch.equal(g.U, ref.U)


def test_deterministic():
    A = _dev(W.gaussian(300, 250, seed=8), "f32")
    a = rp.rplu_dense(A, 50, seed=77)
    b = rp.rplu_dense(A, 50, seed=77)
    assert torch.equal(a.I, b.I) and torch.equal(a.L, b.L) and torch.equal(a.U, b.U)
    assert np.array_equal(a.T, b.T)


@pytest.mark.parametrize("dt", ["f64", "c128"])
def test_c2_complete_given_modes(orc, dt):
    A = W.gaussian(60, 45, seed=12, complex_=dt == "c128")
    for mode in ("c2", "complete"):
        g = rp.rplu_dense(_dev(A, dt), 30, pivot=mode)
        o = orc.rplu_dense(A, 30, mode=mode)
        assert np.array_equal(to_np(g.I), o["I"]) and np.array_equal(to_np(g.J), o["J"]), mode
        assert_factors(g, o, 30, GPU_TOL[dt])
    gI = np.random.default_rng(0).permutation(60)[:25]
    gJ = np.random.default_rng(1).permutation(45)[:25]
    g = rp.rplu_dense(_dev(A, dt), 25, pivot="given", given=(gI, gJ))
    o = orc.rplu_dense(A, 25, mode="given", given=(gI, gJ))
    assert np.array_equal(to_np(g.I), gI) and np.array_equal(to_np(g.J), gJ)
    assert_factors(g, o, 25, GPU_TOL[dt])


def test_tolerance_stop_and_not_converged(orc):
    A = W.dense_haar_500x400()
    g = rp.rplu_dense(_dev(A, "f64"), 200, seed=3, rel_tol=1e-3)
    o = orc.rplu_dense(A, 200, seed=3, tol=1e-3)
    assert g.k_done == o["k_done"] < 200
    assert g.status == rp.RPLU_OK
    g2 = rp.rplu_dense(_dev(A, "f64"), 5, seed=3, rel_tol=1e-9)
    assert g2.status == rp.RPLU_NOT_CONVERGED and g2.k_done == 5


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_exact_recovery_and_zero_matrix(dt):
    A = W.lowrank_product(200, 150, 7, seed=1)
    g = rp.rplu_dense(_dev(A, dt), 40, seed=1, rel_tol=1e-4 if dt == "f32" else 1e-10)
    assert g.k_done == 7
    assert rel_error(A, g.L, g.U) <= (1e-5 if dt == "f32" else 1e-12)
    z = rp.rplu_dense(torch.zeros((40, 30), dtype=TDT[dt], device="cuda"), 10, seed=0)
    assert z.k_done == 0 and z.T[0] == 0.0
    assert np.all(to_np(z.L) == 0) and np.all(to_np(z.U) == 0)


def test_empty_and_k0(orc):
    e = rp.rplu_dense(torch.zeros((0, 5), dtype=torch.float64, device="cuda"), 0)
    assert e.k_done == 0
    A = W.gaussian(30, 20, seed=2)
    g = rp.rplu_dense(_dev(A, "f64"), 0)
    assert g.k_done == 0 and g.T[0] == pytest.approx(np.sum(A * A), rel=1e-13)


def test_non_finite_input_rejected():
    A = W.gaussian(50, 40, seed=2)
    A[7, 9] = np.nan
    with pytest.raises(rp.RPLUError) as ei:
        rp.rplu_dense(_dev(A, "f64"), 5)
    assert ei.value.status == rp.RPLU_ERR_INVALID
    A[7, 9] = np.inf
    with pytest.raises(rp.RPLUError):
        rp.rplu_dense(_dev(A, "f32"), 5)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_mean_error_within_5_percent_of_oracle(orc, dt):
    A = W.dense_haar_500x400()
    Ao = _oracle_input(A, dt)
    eg, eo = [], []
    Ad = _dev(A, dt)
    for s in range(30):
        g = rp.rplu_dense(Ad, 40, seed=100 + s)
        o = orc.rplu_dense(Ao, 40, seed=100 + s)
        eg.append(rel_error(A, g.L, g.U))
        eo.append(rel_error(A, o["L"], o["U"]))
    assert abs(np.mean(eg) - np.mean(eo)) <= 0.05 * np.mean(eo)


def test_f32_tracks_f64_oracle_on_dense_haar_500x400(orc):
    A = W.dense_haar_500x400()
    Ao = _oracle_input(A, "f32")
    g = rp.rplu_dense(_dev(A, "f32"), 40, seed=11)
    o = orc.rplu_dense(Ao, 40, seed=11)
    upto = assert_pivots(g, o, TIE["f32"], min_steps=5, residual_scaled=True)
    assert_factors(g, o, upto, GPU_TOL["f32"])


@pytest.mark.parametrize("dt", ["f32", "c64", "f64", "c128"])
@pytest.mark.parametrize("blk", [2, 3, 8])
def test_pass_block_is_bitwise_invariant(dt, blk):
    """Writing S back every `blk` steps and applying the pending updates in
    registers gives exactly the numbers of a write-back every step."""
    A = W.gaussian(333, 301, seed=6, complex_=dt.startswith("c"))
    Ad = _dev(A, dt)
    ref = rp.rplu_dense(Ad, 37, seed=3, pass_block=1, return_d=True)
    g = rp.rplu_dense(Ad, 37, seed=3, pass_block=blk, return_d=True)
    assert torch.equal(g.I, ref.I) and torch.equal(g.J, ref.J)
    assert torch.equal(g.L, ref.L) and torch.equal(g.U, ref.U) and torch.equal(g.d, ref.d)
    assert np.array_equal(g.T, ref.T)
    D = W.dense_haar_decay(200, 180, 0.7, seed=2)
    Dd = _dev(D, dt)
    a1 = rp.rplu_dense(Dd, 150, seed=9, pass_block=1, rel_tol=1e-4)
    ab = rp.rplu_dense(Dd, 150, seed=9, pass_block=blk, rel_tol=1e-4)
    assert a1.k_done == ab.k_done < 150
    assert torch.equal(a1.L, ab.L) and torch.equal(a1.U, ab.U)


@pytest.mark.parametrize("dt,shape,k", [("f32", (2600, 2300), 24), ("f32", (4100, 3100), 40), ("f64", (1300, 1100), 24),
                                        ("c64", (1800, 1500), 24), ("c128", (900, 700), 24)])
def test_multi_chunk_many_row_blocks(orc, dt, shape, k):
    """Shapes where the pass's structure changes: more than one column chunk
    (256 16-byte vectors: 1024 FP32, 512 FP64/complex64, 256 complex128
    columns) with a ragged last chunk, several 8-row blocks per CTA, and for
    FP32 the default write-back interval of 8 steps, so that every kernel
    specialised on the number of pending updates (1..8) runs and the
    pivot-chunk mask spans several chunks."""
    n, m = shape
    sigma = (1.0 + np.arange(min(n, m))) ** -2.0
    A = W.dense_householder_decay(n, m, sigma, seed=n + m)
    if dt.startswith("c"):
        A = A + 1j * W.dense_householder_decay(n, m, sigma, seed=n + m + 1)
    Ao = _oracle_input(A, dt)
    g = rp.rplu_dense(_dev(A, dt), k, seed=17)
    o = orc.rplu_dense(Ao, k, seed=17)
    assert g.k_done == o["k_done"] == k
    upto = assert_pivots(g, o, TIE[dt], min_steps=9 if dt == "f32" else 3, residual_scaled=True)
    assert_factors(g, o, upto, GPU_TOL[dt])


def test_bench_matrix_first_steps(orc):
    """The benchmark's own input (dense FP32 32768^2, Householder-product
    factors, sigma_i = (1 + i)^-2) factored to k = 256 exactly as the
    benchmark calls it; its first three steps against the oracle on the same
    FP32 values (the oracle costs about a second per step at this size)."""
    gen = W.dense_householder_inverse_square()
    Ad = gen.to_torch("cuda", torch.float32)
    g = rp.rplu_dense(Ad, 256, seed=1)
    torch.cuda.synchronize()
    assert g.k_done == 256
    Ao = Ad.cpu().numpy().astype(np.float64)
    del Ad
    o = orc.rplu_dense(Ao, 3, seed=1)
    assert np.array_equal(to_np(g.I)[:3], o["I"]) and np.array_equal(to_np(g.J)[:3], o["J"])
    Lg, Ug = to_np(g.L)[:, :3].astype(np.float64), to_np(g.U)[:3].astype(np.float64)
    piv = o["U"][np.arange(3), o["J"]]
    ec = np.linalg.norm((Lg - o["L"]) * piv) / np.linalg.norm(o["L"] * piv)
    eu = np.linalg.norm(Ug - o["U"]) / np.linalg.norm(o["U"])
    assert ec <= GPU_TOL["f32"] and eu <= GPU_TOL["f32"], (ec, eu)
    assert np.allclose(g.T[:4], o["T"], rtol=1e-5, atol=0)
    I = to_np(g.I)
    assert len(set(I.tolist())) == 256 and len(set(to_np(g.J).tolist())) == 256


@pytest.mark.parametrize("dt", ["f32", "c64"])
def test_pinned_host_input_read_in_place_equals_device_input(dt):
    """A in page-locked host memory is read in place by the first kernel; the
    factors equal those of the same matrix in device memory bit for bit, as do
    those of pageable host memory (copied first) and of a row stride that is
    not 16-byte aligned (copied first)."""
    tdt = {"f32": torch.float32, "c64": torch.complex64}[dt]
    A = W.dense_haar_decay(1300, 1100, 0.95, seed=11)
    if dt == "c64":
        A = A + 1j * W.dense_haar_decay(1300, 1100, 0.95, seed=12)
    Ad = torch.from_numpy(A).to(tdt).cuda()
    ref = rp.rplu_dense(Ad, 40, seed=9)
    pinned = torch.empty(Ad.shape, dtype=tdt, pin_memory=True)
    pinned.copy_(Ad)
    wide = torch.empty((1300, 1101), dtype=tdt, pin_memory=True)  # row stride of 1101 elements: not 16-byte aligned
    wide[:, :1100].copy_(Ad)
    for src in (pinned, pinned.numpy().copy(), wide[:, :1100]):
        r = rp.rplu_dense(src, 40, seed=9)
        assert r.k_done == ref.k_done
        for a, b in ((r.I, ref.I), (r.J, ref.J), (r.L, ref.L), (r.U, ref.U)):
            assert np.array_equal(to_np(a), to_np(b))
