"""GPU parity of RPLU in CUR form on sparse matrices (rplu_sparse_cur through
the C-ABI) against the CUR-form oracle (oracle/cur_form.py, SparseOperator,
with its QR core: the library keeps its core as a double-double block-inverse
update, both accurate to about eps cond) on the same draws: the same pivots up
to near-ties, the same row-norm totals, a core equal to A(I,J)^{-1} of the
run's own pivots to eps cond; C2PLU choices that are maxima of their own
residual; forced pivots; exact recovery of a rank-r matrix; bitwise-identical
repeated runs.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cur_form as CF
from parity import to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402

import paper_2601_22344_gb300 as rp  # noqa: E402


def _random_sparse(n, m, density, seed):
    rng = np.random.default_rng(seed)
    return sp.random(n, m, density=density, random_state=rng, data_rvs=lambda k: rng.standard_normal(k)).tocsr()


def _first_tie(o, rel=1e-11):
    T = o["T"]
    kd = o["k_done"]
    thr = rel * T[0] / np.maximum(T[:kd], 1e-300)
    m = np.minimum(o["row_margin"], o["col_margin"])
    bad = np.nonzero(m < thr)[0]
    return int(bad[0]) if len(bad) else kd


def _core_bound(W_, kd):
    """||core A(I,J) - I|| for a core accurate to about eps cond(A(I,J)) (a QR
    of A(I,J), or the double-double update), the FP64 check's own rounding
    included; the FP64 block-inverse update would need eps cond^2."""
    cond = np.linalg.cond(W_) if kd else 1.0
    return max(100 * kd * 1.1e-16 * cond, 1e-12 * max(kd, 1))


def _with_dense_lines(seed):
    """A random sparse matrix with three rows and two columns of more than 1024
    entries: the kernels walk those with a whole CTA, the rest with segments
    of a warp."""
    rng = np.random.default_rng(seed)
    S = _random_sparse(2600, 2200, 0.004, seed).tolil()
    for p in (5, 777, 2599):
        cols = rng.choice(2200, 1500, replace=False)
        S[p, cols] = rng.standard_normal(1500)
    for q in (3, 1800):
        rows = rng.choice(2600, 1300, replace=False)
        S[rows, q] = rng.standard_normal(1300)
    S = S.tocsr()
    S.sort_indices()
    assert (np.diff(S.indptr) > 1024).sum() == 3 and (np.diff(S.tocsc().indptr) > 1024).sum() >= 2
    return S


CASES = {
    "random": lambda: _random_sparse(700, 600, 0.01, 4),
    "graph": lambda: W.chung_lu_graph(3000, avg_degree=5.0, exponent=2.3, seed=6),
    "dense_lines": lambda: _with_dense_lines(11),
}


@pytest.mark.parametrize("case", list(CASES))
def test_parity_with_the_oracle(case):
    S = CASES[case]()
    k = 40
    o = CF.rplu_cur(CF.SparseOperator(S), k, seed=9, core="qr")
    g = rp.rplu_sparse_cur(S, k, seed=9)
    upto = min(_first_tie(o), g.k_done)
    assert upto >= 10
    I, J = to_np(g.I), to_np(g.J)
    assert np.array_equal(I[:upto], o["I"][:upto]) and np.array_equal(J[:upto], o["J"][:upto])
    np.testing.assert_allclose(g.T[:upto + 1], o["T"][:upto + 1], rtol=1e-9, atol=1e-12 * o["T"][0])
    kd = g.k_done
    W_ = S[I][:, J].toarray()
    assert np.linalg.norm(to_np(g.core) @ W_ - np.eye(kd)) <= _core_bound(W_, kd)
    # repeated runs are bitwise identical (fixed summation orders, no atomics)
    g2 = rp.rplu_sparse_cur(S, k, seed=9)
    assert np.array_equal(to_np(g2.I), I) and np.array_equal(to_np(g2.core), to_np(g.core))
    assert np.array_equal(g2.T, g.T)


def test_c2_choices_are_maxima_of_the_residual():
    S = W.chung_lu_graph(400, avg_degree=5.0, exponent=2.3, seed=6)
    A = S.toarray()
    g = rp.rplu_sparse_cur(S, 25, pivot="c2")
    I, J = to_np(g.I), to_np(g.J)
    for t in range(g.k_done):
        R = A - (A[:, J[:t]] @ np.linalg.solve(A[np.ix_(I[:t], J[:t])], A[I[:t], :]) if t else 0.0)
        if np.sum(R ** 2) <= 1e-10 * np.sum(A ** 2):
            break
        w = np.sum(R ** 2, axis=1)
        assert w[I[t]] >= (1 - 1e-9) * w.max(), t
        r = R[I[t]] ** 2
        assert r[J[t]] >= (1 - 1e-9) * r.max(), t


def test_given_pivots_and_exact_recovery():
    S = _random_sparse(300, 250, 0.02, 7)
    o = CF.rplu_cur(CF.SparseOperator(S), 12, seed=2, core="qr")
    g = rp.rplu_sparse_cur(S, 12, pivot="given", given=(o["I"], o["J"]), device="host")
    assert np.array_equal(g.I, o["I"]) and np.array_equal(g.J, o["J"])
    W_ = S[o["I"]][:, o["J"]].toarray()
    assert np.linalg.norm(g.core @ W_ - np.eye(12)) <= _core_bound(W_, 12)
    # block diagonal with 6 rank-one blocks: reproduced after 6 steps
    rng = np.random.default_rng(8)
    B = sp.block_diag([sp.csr_matrix(np.outer(rng.standard_normal(rng.integers(3, 9)),
                                              rng.standard_normal(rng.integers(3, 9)))) for _ in range(6)]).tocsr()
    r = rp.rplu_sparse_cur(B, 8, seed=4, rel_tol=1e-6, device="host")
    assert r.k_done == 6
    A = B.toarray()
    np.testing.assert_allclose(A[:, r.J] @ r.core @ A[r.I, :], A, atol=1e-12 * np.abs(A).max())
