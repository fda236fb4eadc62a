"""Pins for the matrix-free Cauchy oracle.

* Against the dense oracle on the materialised matrix: same draws give the same
  pivots, the same L and U, and the row-norm estimates d equal the exact squared
  row norms of A - LU (the update formula of Sec. 4.1 "Row norm updates").
  The update subtracts quantities of the size of the original row norms, so an
  estimate carries an absolute error of order eps * ||A_i||^2: pivots are
  compared while ||S||_F^2 / ||A||_F^2 > 1e-9 and each draw is at least 1e-6
  (relative) away from a CDF boundary.
* At sizes where A is never formed: the displacement structure of Sec. 5.1.
  Every residual of a Cauchy matrix is Cauchy-like, with generators updated by
  Eqs. generator_update_g / generator_update_b starting from G = B = 1 (p = 1);
  so (A - LU)_pq must equal G_p B_q / (x_p - y_q) at any (p, q), and
  d_p must equal sum_q |G_p B_q / (x_p - y_q)|^2.
"""
import numpy as np
import pytest

import workloads as W


def _first_tie(*margins, thresh=1e-9):
    m = np.minimum.reduce([np.asarray(x) for x in margins])
    bad = np.nonzero(m < thresh)[0]
    return int(bad[0]) if len(bad) else len(m)


@pytest.mark.parametrize("mode", ["random", "c2"])
def test_matrix_free_equals_dense_oracle(orc, mode):
    x, y = W.cauchy_spirals(70, 55, seed=4)
    A = W.cauchy_dense(x, y)
    k = 25
    rc = orc.rplu_cauchy(x, y, k, seed=6, mode=mode)
    rd = orc.rplu_dense(A, k, seed=6, mode=mode)
    upto = int(np.argmax(np.append(rd["T"] / rd["T"][0], 0.0) <= 1e-9))
    if mode == "random":  # argmax modes draw nothing; their margins are 0
        upto = min(upto, _first_tie(rc["row_margin"], rc["col_margin"], thresh=1e-6),
                   _first_tie(rd["row_margin"], rd["col_margin"], thresh=1e-6))
    assert upto >= 8
    assert list(rc["I"][:upto]) == list(rd["I"][:upto])
    assert list(rc["J"][:upto]) == list(rd["J"][:upto])
    _compare_factors(A, rc, rd, upto)


def test_row_norm_update_matches_exact_norms(orc):
    x, y = W.cauchy_spirals(80, 64, seed=9)
    A = W.cauchy_dense(x, y)
    for k in (1, 5, 30):
        rc = orc.rplu_cauchy(x, y, k, seed=2)
        S = A - rc["L"] @ rc["U"]
        exact = np.sum(np.abs(S) ** 2, axis=1)
        d0 = np.sum(np.abs(A) ** 2, axis=1)
        assert np.max(np.abs(rc["d"] - exact)) <= 1e-9 * np.max(d0)
        assert rc["T"][-1] == pytest.approx(np.sum(rc["d"]), rel=1e-12)


def test_given_mode_reproduces_dense(orc):
    x, y = W.cauchy_smiley(30, 40, seed=1)
    A = W.cauchy_dense(x, y)
    rd = orc.rplu_dense(A, 15, seed=3)
    rc = orc.rplu_cauchy(x, y, 15, mode="given", given=(rd["I"], rd["J"]))
    _compare_factors(A, rc, rd, 15)


def _compare_factors(A, r1, r2, k):
    """L(:,t) = residual column / pivot: both forms carry rounding of order
    eps * max|A| in the residual, so column t may differ by that over |a_t|;
    U rows are residual rows and differ by eps * max|A|; the products agree
    normwise."""
    amax = np.max(np.abs(A))
    piv = np.abs(r2["U"][np.arange(k), r2["J"][:k]])
    for t in range(k):
        assert np.max(np.abs(r1["L"][:, t] - r2["L"][:, t])) <= 1e-12 * amax / piv[t]
    assert np.max(np.abs(r1["U"][:k] - r2["U"][:k])) <= 1e-12 * amax * k
    P1 = r1["L"][:, :k] @ r1["U"][:k]
    P2 = r2["L"][:, :k] @ r2["U"][:k]
    assert np.linalg.norm(P1 - P2) <= 1e-12 * np.linalg.norm(A) * k


def _generators(r):
    """Generator recurrence of Sec. 5.1 for the factors of a Cauchy RPLU run:
    G <- G - L(:,t) G(i_t),  B <- B - B(j_t) U(t,:) / U(t, j_t)."""
    n = r["L"].shape[0]
    m = r["U"].shape[1]
    G = np.ones(n, complex)
    B = np.ones(m, complex)
    for t in range(r["k_done"]):
        i, j = r["I"][t], r["J"][t]
        a = r["U"][t, j]
        gi = G[i]
        bj = B[j]
        G = G - r["L"][:, t] * gi
        B = B - (bj / a) * r["U"][t]
    return G, B


def test_generator_closure_at_scale(orc):
    n, m, k = 2500, 2000, 30
    x, y = W.cauchy_spirals(n, m, seed=12)
    r = orc.rplu_cauchy(x, y, k, seed=8)
    G, B = _generators(r)
    rng = np.random.default_rng(0)
    p = rng.integers(0, n, 400)
    q = rng.integers(0, m, 400)
    lhs = 1.0 / (x[p] - y[q]) - np.einsum("ij,ji->i", r["L"][p], r["U"][:, q])
    rhs = G[p] * B[q] / (x[p] - y[q])
    scale = np.max(np.abs(1.0 / (x[p] - y[q])))
    assert np.max(np.abs(lhs - rhs)) <= 1e-9 * scale
    # row-norm estimates against exact norms of the generator representation
    rows = rng.integers(0, n, 50)
    for pr in rows:
        exact = np.sum(np.abs(G[pr] * B / (x[pr] - y)) ** 2)
        d0 = np.sum(np.abs(1.0 / (x[pr] - y)) ** 2)
        assert abs(r["d"][pr] - exact) <= 1e-8 * max(d0, 1e-300)
    # pivoted rows have zero estimate
    assert np.all(r["d"][r["I"]] == 0.0)


def _schur_closed_form(x, y, I, J, p, q):
    """Entries (p, q) of the Schur complement of the Cauchy matrix
    1/(x_p - y_q) after eliminating rows I and columns J.

    Cauchy's determinant formula, det[1/(x_a - y_b)] = prod_{a<b} (x_b - x_a)
    (y_a - y_b) / prod_{a,b} (x_a - y_b), and the determinant-ratio form of a
    Schur complement, S_pq = det A([I,p],[J,q]) / det A(I,J), give
        S_pq = 1/(x_p - y_q) prod_s (x_p - x_{I_s}) (y_{J_s} - y_q)
                                    / ((x_p - y_{J_s}) (x_{I_s} - y_q)),
    a closed form that shares nothing with the elimination recurrences; it
    vanishes on the eliminated rows and columns by itself."""
    S = 1.0 / (x[p][:, None] - y[q][None, :])
    for i, j in zip(I, J):
        S = S * ((x[p] - x[i])[:, None] * (y[j] - y[q])[None, :]) / ((x[p] - y[j])[:, None] * (x[i] - y[q])[None, :])
    return S


@pytest.mark.parametrize("points", ["spirals", "smiley"])
def test_factors_match_cauchy_determinant_closed_form(orc, points):
    """Every step's U row (the residual row at the pivot), L column (the
    residual column over the pivot) and the final row-norm estimates d against
    the closed-form Schur complements of a Cauchy matrix."""
    gen = W.cauchy_spirals if points == "spirals" else W.cauchy_smiley
    x, y = gen(90, 70, seed=12)
    r = orc.rplu_cauchy(x, y, 14, seed=3)
    kd, I, J = r["k_done"], r["I"], r["J"]
    n, m = len(x), len(y)
    assert kd == 14
    for t in range(kd):
        row = _schur_closed_form(x, y, I[:t], J[:t], np.array([I[t]]), np.arange(m))[0]
        col = _schur_closed_form(x, y, I[:t], J[:t], np.arange(n), np.array([J[t]]))[:, 0]
        rscale = np.max(np.abs(1.0 / (x[I[t]] - y)))
        cscale = np.max(np.abs(1.0 / (x - y[J[t]])))
        piv = row[J[t]]
        assert np.max(np.abs(r["U"][t] - row)) <= 1e-13 * (t + 1) * rscale
        assert np.max(np.abs(r["L"][:, t] - col / piv)) <= 1e-12 * (t + 1) * cscale / abs(piv)
        assert r["L"][I[t], t] == 1.0
    S = _schur_closed_form(x, y, I, J, np.arange(n), np.arange(m))
    d0 = np.sum(np.abs(1.0 / (x[:, None] - y[None, :])) ** 2, axis=1)
    assert np.max(np.abs(r["d"] - np.sum(np.abs(S) ** 2, axis=1))) <= 1e-12 * np.max(d0)


def test_cauchy_rejects_complete_mode(orc):
    x, y = W.cauchy_spirals(10, 10, seed=0)
    with pytest.raises(ValueError):
        orc.rplu_cauchy(x, y, 3, mode="complete")
