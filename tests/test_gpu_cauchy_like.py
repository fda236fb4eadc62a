"""GPU parity of the Cauchy-like (generator) form, rplu_cauchy_like through
the C-ABI, against the oracle's generator form on the same inputs and draws;
plus the exact-norm property at scale: the reported residual equals the
explicit one, and an FP32 run reaches a 1e-6 tolerance."""
import numpy as np
import pytest

import workloads as W
from parity import GPU_TOL, TIE, assert_factors, assert_pivots, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)

NDT = {"f32": np.float32, "f64": np.float64, "c64": np.complex64, "c128": np.complex128}


def _case(kind, seed, n=300, m=260):
    rng = np.random.default_rng(seed)
    if kind == "real_p2":
        x, y = rng.uniform(-1, 1, n), rng.uniform(2.5, 4, m)
        G, B = rng.standard_normal((n, 2)), rng.standard_normal((2, m))
    elif kind == "complex_p3":
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        y = 5 + rng.standard_normal(m) + 1j * rng.standard_normal(m)
        G = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
        B = rng.standard_normal((3, m)) + 1j * rng.standard_normal((3, m))
    elif kind == "cauchy_p1":
        x, y = W.cauchy_spirals(n, m, seed=seed)
        G, B = np.ones((n, 1), complex), np.ones((1, m), complex)
    else:  # loewner, p = 2
        x = np.exp(2j * np.pi * rng.random(n))
        y = 2.5 * np.exp(2j * np.pi * rng.random(m))
        f = lambda z: 1.0 / (1.2 - z) + np.exp(0.3 * z)  # noqa: E731
        G, B = W.loewner_generators(x, y, f(x), f(y))
    return x, y, G, B


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).astype(NDT[dt]))).cuda()


def _oracle_in(a, dt):
    return np.asarray(a).astype(NDT[dt]).astype(np.complex128)


@pytest.mark.parametrize("kind,dt", [("real_p2", "f64"), ("complex_p3", "c128"), ("cauchy_p1", "c128"),
                                     ("loewner", "c128"), ("real_p2", "f32"), ("complex_p3", "c64"),
                                     ("loewner", "c64")])
@pytest.mark.parametrize("seed", [0, 1])
def test_parity_with_the_generator_oracle(orc, kind, dt, seed):
    x, y, G, B = _case(kind, seed)
    k = 25
    g = rp.rplu_cauchy_like(_dev(x, dt), _dev(y, dt), _dev(G, dt), _dev(B, dt), k, seed=seed + 3)
    o = orc.rplu_cauchy_like(_oracle_in(x, dt), _oracle_in(y, dt), _oracle_in(G, dt), _oracle_in(B, dt), k,
                             seed=seed + 3)
    assert g.k_done == o["k_done"] or dt in ("f32", "c64")
    upto = assert_pivots(g, o, TIE[dt], min_steps=min(3, o["k_done"]) if dt in ("f64", "c128") else 1,
                         residual_scaled=True)
    tol = GPU_TOL[dt]
    assert_factors(g, o, upto, tol)
    if upto == o["k_done"] == g.k_done and dt in ("f64", "c128"):
        np.testing.assert_allclose(g.T, o["T"], rtol=1e-9, atol=1e-12 * o["T"][0])


@pytest.mark.parametrize("dt", ["f64", "c128"])
def test_c2_and_given_modes(orc, dt):
    x, y, G, B = _case("complex_p3" if dt == "c128" else "real_p2", 7, n=120, m=90)
    o = orc.rplu_cauchy_like(_oracle_in(x, dt), _oracle_in(y, dt), _oracle_in(G, dt), _oracle_in(B, dt), 15,
                             mode="c2")
    g = rp.rplu_cauchy_like(_dev(x, dt), _dev(y, dt), _dev(G, dt), _dev(B, dt), 15, pivot="c2")
    upto = assert_pivots(g, o, TIE[dt], random_mode=False)
    assert_factors(g, o, upto, GPU_TOL[dt])
    gv = rp.rplu_cauchy_like(_dev(x, dt), _dev(y, dt), _dev(G, dt), _dev(B, dt), 15, pivot="given",
                             given=(o["I"], o["J"]))
    assert np.array_equal(to_np(gv.I), o["I"]) and np.array_equal(to_np(gv.J), o["J"])
    assert_factors(gv, o, 15, GPU_TOL[dt])


def test_reported_residual_is_the_explicit_residual():
    """Spiral Cauchy matrix (the shape of the benchmark's matrix-free workload), complex64, 4000^2:
    the residual the run reports (sum of exact row norms) equals ||A - LU||_F computed explicitly."""
    x, y = W.cauchy_spirals(4000, 4000, seed=11)
    xd, yd = _dev(x, "c64"), _dev(y, "c64")
    G = torch.ones((4000, 1), dtype=torch.complex64, device="cuda")
    B = torch.ones((1, 4000), dtype=torch.complex64, device="cuda")
    g = rp.rplu_cauchy_like(xd, yd, G, B, 60, seed=5)
    A = 1.0 / (xd.to(torch.complex128)[:, None] - yd.to(torch.complex128)[None, :])
    R = A - g.L.to(torch.complex128) @ g.U.to(torch.complex128)
    explicit = float(torch.linalg.norm(R) / torch.linalg.norm(A))
    reported = float(np.sqrt(g.T[-1] / g.T[0]))
    assert abs(reported - explicit) <= 1e-3 * explicit + 1e-6


def test_fp32_reaches_a_1e6_tolerance():
    """Separated real Cauchy blocks: the exact-norm generator form stops at ||S||_F <= 1e-6 ||A||_F in
    FP32 and the explicit error agrees (the FP32 rounding floor of S is about 1e-7)."""
    for b, blk in enumerate(W.cauchy_interval_blocks(4, seed=3, size_lo=500, size_hi=900)):
        n, m = len(blk.x), len(blk.y)
        g = rp.rplu_cauchy_like(_dev(blk.x, "f32"), _dev(blk.y, "f32"), torch.ones((n, 1), device="cuda"),
                                torch.ones((1, m), device="cuda"), min(n, m), seed=b, rel_tol=1e-6)
        assert g.k_done < min(n, m)
        A = W.cauchy_dense(blk.x.astype(np.float32), blk.y.astype(np.float32)).astype(np.float64)
        err = np.linalg.norm(A - to_np(g.L).astype(np.float64) @ to_np(g.U).astype(np.float64)) / np.linalg.norm(A)
        assert err <= 2e-6
        assert np.sqrt(g.T[-1] / g.T[0]) <= 1e-6
