"""Pins of the oracle's Cauchy-like (generator) form, Sec. 5.1.

* It equals the dense oracle run on the materialised matrix: the same pivots
  (away from near-ties) and the same factors, for real and complex
  generators, displacement ranks 1 to 3, a Loewner matrix, and plain Cauchy
  (G = B = 1).
* After k steps the residual A - L U satisfies the Sylvester displacement
  equation X S - S Y = G B with the returned generators (Eq.
  cauchy-like-Sylvester), and the generators vanish exactly on the pivot
  rows and columns.
* The Loewner generators of Sec. 5.2 reproduce (f(x_i) - f(y_j)) / (x_i - y_j).
"""
import numpy as np
import pytest

import workloads as W


def _case(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "real_p2":
        x = rng.uniform(-1, 1, 40)
        y = rng.uniform(2.5, 4, 33)
        G, B = rng.standard_normal((40, 2)), rng.standard_normal((2, 33))
    elif kind == "complex_p3":
        x = rng.standard_normal(31) + 1j * rng.standard_normal(31)
        y = 4 + rng.standard_normal(37) + 1j * rng.standard_normal(37)
        G = rng.standard_normal((31, 3)) + 1j * rng.standard_normal((31, 3))
        B = rng.standard_normal((3, 37)) + 1j * rng.standard_normal((3, 37))
    elif kind == "cauchy_p1":
        x = rng.uniform(-1, 1, 35)
        y = rng.uniform(3, 5, 29)
        G, B = np.ones((35, 1)), np.ones((1, 29))
    else:  # loewner
        x = np.exp(2j * np.pi * rng.random(36))
        y = 2.5 * np.exp(2j * np.pi * rng.random(30))
        f = lambda z: 1.0 / (1.2 - z) + np.exp(0.3 * z)  # noqa: E731
        G, B = W.loewner_generators(x, y, f(x), f(y))
    return x, y, G, B


def _residual_cols(r):
    piv = r["U"][np.arange(r["k_done"]), r["J"]]
    return r["L"] * piv[None, :]


@pytest.mark.parametrize("kind", ["real_p2", "complex_p3", "cauchy_p1", "loewner"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equals_dense_oracle_on_the_materialised_matrix(orc, kind, seed):
    x, y, G, B = _case(kind, seed)
    A = W.cauchy_like_dense(x, y, G, B)
    k = 12
    g = orc.rplu_cauchy_like(x, y, G, B, k, seed=seed + 10)
    d = orc.rplu_dense(A.astype(np.complex128), k, seed=seed + 10)
    # near-tie window: draws within rounding of a CDF boundary may pick the neighbour; the rounding of
    # the residual is absolute (about eps ||A||_F), so relative to the current total it grows as
    # sqrt(T_0 / T_t)
    m = np.minimum(d["row_margin"], d["col_margin"])
    T = d["T"][:len(m)]
    tie = np.nonzero(m < 1e-12 * np.sqrt(T[0] / np.maximum(T, 1e-300)))[0]
    upto = int(tie[0]) if len(tie) else d["k_done"]
    assert np.array_equal(g["I"][:upto], d["I"][:upto]) and np.array_equal(g["J"][:upto], d["J"][:upto])
    if upto == d["k_done"]:
        assert g["k_done"] == d["k_done"]
        np.testing.assert_allclose(g["T"], d["T"], rtol=1e-9, atol=1e-12 * d["T"][0])
    cg, cd = _residual_cols(g)[:, :upto], _residual_cols(d)[:, :upto]
    assert np.linalg.norm(cg - cd) <= 1e-10 * np.linalg.norm(cd)
    assert np.linalg.norm(g["U"][:upto] - d["U"][:upto]) <= 1e-10 * np.linalg.norm(d["U"][:upto])


@pytest.mark.parametrize("kind", ["real_p2", "complex_p3", "loewner"])
def test_displacement_equation_and_exact_zeros(orc, kind):
    x, y, G, B = _case(kind, 5)
    A = W.cauchy_like_dense(x, y, G, B)
    r = orc.rplu_cauchy_like(x, y, G, B, 9, seed=3)
    S = A - r["L"] @ r["U"]
    lhs = x[:, None] * S - S * y[None, :]
    rhs = r["G"] @ r["B"]
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(G @ B)
    assert np.all(r["G"][r["I"]] == 0) and np.all(r["B"][:, r["J"]] == 0)
    # the residual built from the returned generators is the residual of the factors
    S_gen = W.cauchy_like_dense(x, y, r["G"], r["B"])
    assert np.linalg.norm(S_gen - S) <= 1e-11 * np.linalg.norm(A)


def test_loewner_generators_reproduce_the_loewner_matrix():
    rng = np.random.default_rng(4)
    x = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    y = 5 + rng.standard_normal(17)
    fx, fy = np.sin(x), np.sin(y)
    G, B = W.loewner_generators(x, y, fx, fy)
    Lw = (fx[:, None] - fy[None, :]) / (x[:, None] - y[None, :])
    np.testing.assert_allclose(W.cauchy_like_dense(x, y, G, B), Lw, rtol=1e-13, atol=1e-13)
