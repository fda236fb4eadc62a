"""Pins of the oracle's row-norm upper bounds (App. C) and of the Cauchy-like
factorization with Algorithm 3's rejection-sampled row draw.

* The bounds are certified: ||S(i,:)||^2 <= u_i <= nu ||S(i,:)||^2 for every
  row, checked against brute-force norms of the materialised matrix, for
  several point sets, displacement ranks, nu and leaf sizes; with nu = 1
  nothing is aggregated and u equals the exact norms.
* With nu = 1 every first proposal is accepted and the factorization equals
  the exact-norm generator form (same draws).
* The accepted pivot of a step follows |S_ij|^2 / ||S||_F^2 (chi-square over
  many seeds with nu = 5), as rejection sampling guarantees.
* The residual after k steps satisfies the Sylvester displacement equation.
* The Loewner matrix of a rational function of McMillan degree d has rank d
  (Mayo & Antoulas, Linear Algebra Appl. 425, 2007): through its generators
  both the exact-norm form and Algorithm 3 reach a residual at rounding level
  after exactly d steps, and not before.
"""
import numpy as np
import pytest
from scipy import stats

import workloads as W


def _points(kind, seed, n=300, m=260):
    rng = np.random.default_rng(seed)
    if kind == "spirals":
        x, y = W.cauchy_spirals(n, m, seed=seed)
        G, B = np.ones((n, 1)), np.ones((1, m))
    elif kind == "intervals":
        x, y = rng.uniform(-1, 1, n) + 0j, rng.uniform(3, 5, m) + 0j
        G, B = rng.standard_normal((n, 2)), rng.standard_normal((2, m))
    else:  # overlapping complex clouds, p = 3
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        y = 0.5 + rng.standard_normal(m) + 1j * rng.standard_normal(m)
        G = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
        B = rng.standard_normal((3, m)) + 1j * rng.standard_normal((3, m))
    return x, y, G, B


@pytest.mark.parametrize("kind", ["spirals", "intervals", "clouds"])
@pytest.mark.parametrize("nu,leaf", [(1.5, 8), (2.0, 16), (5.0, 32), (5.0, 4)])
def test_bounds_are_certified(orc, kind, nu, leaf):
    x, y, G, B = _points(kind, 1)
    A = W.cauchy_like_dense(x, y, G, B)
    rho = (np.abs(A) ** 2).sum(axis=1)
    u = orc.bh_bounds(x, y, G, B, nu=nu, leaf=leaf)
    assert np.all(u >= rho * (1 - 1e-12)), (u / rho).min()
    assert np.all(u <= nu * rho * (1 + 1e-12)), (u / rho).max()


def test_nu_one_gives_the_exact_norms(orc):
    x, y, G, B = _points("clouds", 2)
    A = W.cauchy_like_dense(x, y, G, B)
    rho = (np.abs(A) ** 2).sum(axis=1)
    np.testing.assert_allclose(orc.bh_bounds(x, y, G, B, nu=1.0, leaf=16), rho, rtol=1e-12)


@pytest.mark.parametrize("kind", ["spirals", "intervals", "clouds"])
def test_nu_one_equals_the_exact_norm_form(orc, kind):
    x, y, G, B = _points(kind, 3, n=120, m=100)
    e = orc.rplu_cauchy_like(x, y, G, B, 12, seed=4)
    b = orc.rplu_cauchy_like_bh(x, y, G, B, 12, seed=4, nu=1.0, leaf=16)
    assert np.all(b["attempts"] == 1)
    assert np.array_equal(b["I"], e["I"]) and np.array_equal(b["J"], e["J"])
    np.testing.assert_allclose(b["U"], e["U"], rtol=1e-10, atol=1e-12 * np.abs(e["U"]).max())
    np.testing.assert_allclose(b["T"][-1], e["T"][-1], rtol=1e-9)


def test_rejection_sampled_pivot_law(orc):
    """The first accepted pivot of a 7 x 6 Cauchy-like matrix, nu = 5, leaf 1,
    over 30000 seeds: chi-square against |a_ij|^2 / ||A||_F^2."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    y = 2 + rng.standard_normal(6) + 1j * rng.standard_normal(6)
    G = rng.standard_normal((7, 2)) + 1j * rng.standard_normal((7, 2))
    B = rng.standard_normal((2, 6)) + 1j * rng.standard_normal((2, 6))
    A = W.cauchy_like_dense(x, y, G, B)
    p = (np.abs(A) ** 2).ravel() / (np.abs(A) ** 2).sum()
    u = orc.bh_bounds(x, y, G, B, nu=5.0, leaf=1)
    rho = (np.abs(A) ** 2).sum(axis=1)
    assert (u / rho).max() > 1.05  # some rows are bounded loosely: rejections happen
    counts = np.zeros(A.size)
    N = 30000
    att = 0
    for s in range(N):
        r = orc.rplu_cauchy_like_bh(x, y, G, B, 1, seed=s, nu=5.0, leaf=1)
        counts[r["I"][0] * A.shape[1] + r["J"][0]] += 1
        att += int(r["attempts"][0])
    assert att > N  # rejection did occur
    chi2 = ((counts - N * p) ** 2 / (N * p)).sum()
    assert stats.chi2.sf(chi2, A.size - 1) > 1e-4, chi2


def test_displacement_equation_after_rejection_steps(orc):
    x, y, G, B = _points("clouds", 6, n=150, m=140)
    A = W.cauchy_like_dense(x, y, G, B)
    r = orc.rplu_cauchy_like_bh(x, y, G, B, 10, seed=2, nu=5.0, leaf=16)
    assert r["k_done"] == 10
    S = A - r["L"] @ r["U"]
    # the exact final residual total is reported last; the others are bounds
    np.testing.assert_allclose(r["T"][-1], (np.abs(S) ** 2).sum(), rtol=1e-9)
    assert np.all(r["T"][:-1] >= 0)
    LI = r["L"][r["I"], :]
    assert np.all(np.diag(LI) == 1) and np.all(np.triu(LI, 1) == 0)
    assert np.linalg.norm(S[r["I"], :]) <= 1e-10 * np.linalg.norm(A)
    assert np.linalg.norm(S[:, r["J"]]) <= 1e-10 * np.linalg.norm(A)


@pytest.mark.parametrize("kind", ["spirals", "intervals", "clouds"])
def test_c2_with_exact_bounds_is_c2(orc, kind):
    """nu = 1 makes the bounds the exact row norms, so the approximate C2PLU of
    Sec. 5.1 (row of the largest bound, then the largest entry of that row)
    is the exact-norm C2 mode of the generator form."""
    x, y, G, B = _points(kind, 5, n=120, m=100)
    e = orc.rplu_cauchy_like(x, y, G, B, 20, mode="c2")
    b = orc.rplu_cauchy_like_bh(x, y, G, B, 20, nu=1.0, leaf=8, mode="c2")
    assert np.array_equal(b["I"], e["I"]) and np.array_equal(b["J"], e["J"])
    np.testing.assert_allclose(b["U"], e["U"], rtol=0, atol=1e-12 * np.abs(e["U"]).max())


@pytest.mark.parametrize("kind", ["spirals", "clouds"])
def test_c2_first_pivot_is_the_argmax_of_the_bounds(orc, kind):
    x, y, G, B = _points(kind, 6)
    u = orc.bh_bounds(x, y, G, B, nu=5.0, leaf=16)
    A = W.cauchy_like_dense(x, y, G, B)
    b = orc.rplu_cauchy_like_bh(x, y, G, B, 3, nu=5.0, leaf=16, mode="c2")
    i0 = int(np.argmax(u))
    assert b["I"][0] == i0 and b["J"][0] == int(np.argmax(np.abs(A[i0]) ** 2))
    assert b["attempts"][0] == 1 and b["T"][0] == pytest.approx(u.sum(), rel=1e-12)


def test_max_stopping_rule(orc):
    """stop "max" (Sec. 5.3): with nu = 1 the bounds are the exact row norms of
    the residual, so the run stops at the first step t where the largest
    squared row norm of A - L U is at most tol^2 times that of A."""
    x, y, G, B = _points("intervals", 7, n=90, m=80)
    A = W.cauchy_like_dense(x, y, G, B)
    tol = 1e-4
    b = orc.rplu_cauchy_like_bh(x, y, G, B, 80, seed=2, nu=1.0, leaf=8, tol=tol, stop="max")
    assert 0 < b["k_done"] < 80
    d0 = (np.abs(A) ** 2).sum(axis=1).max()
    first = None
    for t in range(b["k_done"] + 1):
        S = A - b["L"][:, :t] @ b["U"][:t]
        if (np.abs(S) ** 2).sum(axis=1).max() <= tol * tol * d0 * (1 + 1e-9):
            first = t
            break
    assert first == b["k_done"]


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_loewner_rank_of_a_rational_function(orc, d):
    rng = np.random.default_rng(5)
    z = np.sqrt(rng.random(700)) * np.exp(2j * np.pi * rng.random(700))
    x, y = z[:350], z[350:]
    poles = 1.4 * np.exp(2j * np.pi * np.arange(d) / d + 0.3)
    c = 1.0 + 0.5 * np.arange(d)

    def f(q):
        return sum(cj / (q - pj) for cj, pj in zip(c, poles))

    G, B = W.loewner_generators(x, y, f(x), f(y))
    for r in (orc.rplu_cauchy_like(x, y, G, B, d + 2, seed=2),
              orc.rplu_cauchy_like_bh(x, y, G, B, d + 2, seed=2, nu=5.0, leaf=16)):
        T = r["T"] / r["T"][0]
        assert T[d - 1] > 1e-8
        assert np.all(T[d:] < 1e-24)
