"""Pins for the dense-form oracle (Algorithm 1 with the two-stage draw of
Sec. 4.1) against what the paper and linear algebra fix independently:

* one-step expectation E[A1] = A - A A^* A / ||A||_F^2 (Sec. 3.1), by exact
  enumeration of all pivots with the forced-pivot mode;
* one-step Gram identity (Eq. G1_bound, equality when no entry is zero):
  E||A1||_F^2 = 2 ||A||_F^2 - 2 ||A^* A||_F^2 / ||A||_F^2, and the dense
  unitary case E||A1||_F^2 = 2 (n - 1) (Sec. 3.1);
* the pivot law P(i, j) = |a_ij|^2 / ||A||_F^2 (Sec. 1) by chi-square, and the
  exact joint law of two steps by enumeration;
* interpolation: A - LU vanishes on the pivot rows and columns, and
  LU = A[:, J] A[I, J]^{-1} A[I, :] (the CUR form of Sec. 4.1);
* L unit lower triangular on the pivot rows, U upper triangular on the pivot
  columns, in pivot order (Algorithm 1);
* exact recovery of rank-r inputs; Eckart-Young lower bound (Sec. 2);
* Theorem 1: mean ||A - LU||_F^2 <= 4^k ||A - [[A]]_k||_F^2;
* complete pivoting equals LAPACK's xGETC2 (GE with complete pivoting).
"""
import itertools

import numpy as np
import pytest
from scipy import stats
from scipy.linalg import lapack

import workloads as W


def _residual(A, r):
    return A - r["L"] @ r["U"]


def _one_step(orc, A, i, j):
    """A^(1) for the forced pivot (i, j), from the returned factors; the
    oracle's own updated S must have the same squared norm."""
    r = orc.rplu_dense(A, 1, mode="given", given=([i], [j]))
    R = _residual(A, r)
    assert abs(r["T"][1] - np.sum(np.abs(R) ** 2)) <= 1e-12 * r["T"][0]
    return R


@pytest.mark.parametrize("cplx", [False, True])
def test_one_step_expectation_by_enumeration(orc, cplx):
    A = W.gaussian(7, 5, seed=11, complex_=cplx)
    fro2 = np.sum(np.abs(A) ** 2)
    E = np.zeros_like(A)
    for i, j in itertools.product(range(7), range(5)):
        p = abs(A[i, j]) ** 2 / fro2
        E += p * _one_step(orc, A, i, j)
    closed = A - A @ A.conj().T @ A / fro2
    assert np.max(np.abs(E - closed)) <= 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("cplx", [False, True])
def test_one_step_frobenius_expectation(orc, cplx):
    A = W.gaussian(6, 4, seed=5, complex_=cplx)
    fro2 = np.sum(np.abs(A) ** 2)
    e = 0.0
    for i, j in itertools.product(range(6), range(4)):
        e += abs(A[i, j]) ** 2 / fro2 * np.sum(np.abs(_one_step(orc, A, i, j)) ** 2)
    G = A.conj().T @ A
    closed = 2 * fro2 - 2 * np.sum(np.abs(G) ** 2) / fro2
    assert e == pytest.approx(closed, rel=1e-12)


def test_dense_unitary_example(orc):
    n = 6
    F = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n) / np.sqrt(n)
    e = 0.0
    for i, j in itertools.product(range(n), range(n)):
        e += (1.0 / n ** 2) * np.sum(np.abs(_one_step(orc, F, i, j)) ** 2)
    assert e == pytest.approx(2 * (n - 1), rel=1e-12)


@pytest.mark.parametrize("cplx", [False, True])
def test_pivot_law_chi_square(orc, cplx):
    A = W.gaussian(6, 5, seed=3, complex_=cplx)
    p = (np.abs(A) ** 2 / np.sum(np.abs(A) ** 2)).ravel()
    N = 20000
    counts = np.zeros(30)
    for s in range(N):
        r = orc.rplu_dense(A, 1, seed=1000 + s)
        counts[r["I"][0] * 5 + r["J"][0]] += 1
    chi = stats.chisquare(counts, N * p)
    assert chi.pvalue > 1e-3


def test_two_step_joint_law(orc):
    A = W.gaussian(4, 4, seed=8)
    fro2 = np.sum(A ** 2)
    expected = {}
    for i1, j1 in itertools.product(range(4), range(4)):
        p1 = A[i1, j1] ** 2 / fro2
        A1 = _one_step(orc, A, i1, j1)
        f1 = np.sum(A1 ** 2)
        for i2, j2 in itertools.product(range(4), range(4)):
            if A1[i2, j2] != 0.0:
                expected[(i1, j1, i2, j2)] = p1 * A1[i2, j2] ** 2 / f1
    N = 30000
    counts = {key: 0 for key in expected}
    for s in range(N):
        r = orc.rplu_dense(A, 2, seed=77 + 3 * s)
        key = (r["I"][0], r["J"][0], r["I"][1], r["J"][1])
        assert key in counts  # never a zero-probability pivot
        counts[key] += 1
    keys = sorted(expected)
    exp = np.array([expected[k] for k in keys]) * N
    obs = np.array([counts[k] for k in keys], float)
    big = exp >= 5
    obs_b = np.append(obs[big], obs[~big].sum())
    exp_b = np.append(exp[big], exp[~big].sum())
    assert abs(exp.sum() - N) < 1e-6 * N
    assert stats.chisquare(obs_b, exp_b).pvalue > 1e-3


@pytest.mark.parametrize("cplx", [False, True])
def test_interpolation_and_cur_identity(orc, cplx):
    A = W.gaussian(40, 30, seed=21, complex_=cplx)
    r = orc.rplu_dense(A, 12, seed=4)
    I, J = r["I"], r["J"]
    R = _residual(A, r)
    scale = np.max(np.abs(A))
    assert np.max(np.abs(R[I, :])) <= 1e-12 * scale
    assert np.max(np.abs(R[:, J])) <= 1e-12 * scale
    LU = r["L"] @ r["U"]
    cur = A[:, J] @ np.linalg.solve(A[np.ix_(I, J)], A[I, :])
    assert np.max(np.abs(LU - cur)) <= 1e-9 * scale
    # T_hist holds ||S^(t)||_F^2; its last entry is ||A - LU||_F^2
    assert r["T"][-1] == pytest.approx(np.sum(np.abs(R) ** 2), rel=1e-10)
    assert r["T"][0] == pytest.approx(np.sum(np.abs(A) ** 2), rel=1e-14)


def test_triangular_structure(orc):
    A = W.dense_haar_500x400()
    r = orc.rplu_dense(A, 40, seed=9)
    I, J, L, U = r["I"], r["J"], r["L"], r["U"]
    assert len(set(I)) == 40 and len(set(J)) == 40
    LI = L[I, :]
    UJ = U[:, J]
    assert np.all(np.diag(LI) == 1.0)
    assert np.all(np.triu(LI, 1) == 0.0)
    assert np.all(np.tril(UJ, -1) == 0.0)
    # U(t, j_t) is the pivot value: nonzero
    assert np.all(np.diag(UJ) != 0.0)


@pytest.mark.parametrize("cplx", [False, True])
def test_exact_recovery_rank_r(orc, cplx):
    A = W.lowrank_product(30, 20, 5, seed=2, complex_=cplx)
    r = orc.rplu_dense(A, 5, seed=1)
    assert np.linalg.norm(_residual(A, r)) <= 1e-12 * np.linalg.norm(A)
    r2 = orc.rplu_dense(A, 12, seed=1, tol=1e-10)
    assert r2["k_done"] == 5


def test_eckart_young_lower_bound(orc):
    A = W.dense_haar_500x400()
    s = np.linalg.svd(A, compute_uv=False)
    for k in (5, 20, 40):
        r = orc.rplu_dense(A, k, seed=k)
        best = np.sqrt(np.sum(s[k:] ** 2))
        assert np.linalg.norm(_residual(A, r)) >= best * (1 - 1e-10)


@pytest.mark.parametrize("rho", [0.25, 0.4])
def test_theorem1_doubling_bound(orc, rho):
    n = 200
    sigma = rho ** np.arange(n)
    A = W.dense_with_spectrum(sigma, n, n, seed=31)
    for k in (3, 6):
        errs = [orc.rplu_dense(A, k, seed=s)["T"][-1] for s in range(200)]
        bound = 4.0 ** k * np.sum(sigma[k:] ** 2)
        assert np.mean(errs) <= bound


def test_complete_pivoting_matches_lapack_getc2(orc):
    n = 8
    A = W.gaussian(n, n, seed=17)
    lu, ipiv, jpiv, info = lapack.dgetc2(A.copy())
    assert info == 0
    pr = np.arange(n)
    pc = np.arange(n)
    # scipy's wrapper returns the interchanges 0-based: at step t rows t and
    # ipiv[t] (columns t and jpiv[t]) of the working matrix were swapped
    for t in range(n):
        a, b = t, ipiv[t]
        pr[[a, b]] = pr[[b, a]]
        a, b = t, jpiv[t]
        pc[[a, b]] = pc[[b, a]]
    r = orc.rplu_dense(A, n, mode="complete")
    assert list(r["I"]) == list(pr)
    assert list(r["J"]) == list(pc)
    Lg = np.tril(lu, -1) + np.eye(n)
    Ug = np.triu(lu)
    L = np.zeros((n, n))
    U = np.zeros((n, n))
    L[pr, :] = Lg
    U[:, pc] = Ug
    assert np.max(np.abs(L - r["L"])) <= 1e-12 * np.max(np.abs(L))
    assert np.max(np.abs(U - r["U"])) <= 1e-12 * np.max(np.abs(U))


def test_c2_mode_is_greedy(orc):
    A = W.gaussian(25, 18, seed=40, complex_=True)
    r = orc.rplu_dense(A, 10, mode="c2")
    for t in range(10):
        S = A - r["L"][:, :t] @ r["U"][:t]
        rown = np.sum(np.abs(S) ** 2, axis=1)
        i = int(np.argmax(rown))
        assert r["I"][t] == i
        assert r["J"][t] == int(np.argmax(np.abs(S[i])))


def test_tolerance_stop(orc):
    A = W.dense_haar_500x400()
    tol = 1e-3
    r = orc.rplu_dense(A, 200, seed=3, tol=tol)
    T = r["T"]
    kd = r["k_done"]
    assert kd < 200
    assert T[kd] <= tol ** 2 * T[0] < T[kd - 1]


def test_zero_and_degenerate_inputs(orc):
    Z = np.zeros((5, 4))
    r = orc.rplu_dense(Z, 3, seed=0)
    assert r["k_done"] == 0 and r["T"][0] == 0.0
    e = orc.rplu_dense(np.zeros((0, 3)), 0)
    assert e["k_done"] == 0
    one = orc.rplu_dense(np.array([[2.5]]), 1)
    assert one["k_done"] == 1 and one["L"][0, 0] == 1.0 and one["U"][0, 0] == 2.5
    # a single nonzero entry is always the pivot
    B = np.zeros((4, 6))
    B[2, 5] = -3.0
    rb = orc.rplu_dense(B, 2, seed=5)
    assert rb["k_done"] == 1 and rb["I"][0] == 2 and rb["J"][0] == 5
    with pytest.raises(ValueError):
        orc.rplu_dense(np.ones((3, 2)), 3)
