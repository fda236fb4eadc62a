"""Pins of the CUR-form oracle (oracle/cur_form.py: Algorithm 2 of Sec. 4.1
over a general operator).

* Each operator's accesses (rows, columns, blocks, matvec, initial row norms)
  equal those of its matrix formed entry by entry from the definition: the
  Cauchy formula, the sparse matrix's entries, and for the multi-level
  Toeplitz matrix of Sec. 4.2 the drifted Gaussian kernel (Eq. kernel)
  evaluated at every pair of grid points.
* The Kronecker structure of that Toeplitz matrix: its singular values are the
  products of the three one-dimensional factors' singular values, and its row
  norms are products too.
* Algorithm 2 with the same draws reproduces the LU-form oracle (the C oracle's
  rplu_dense on the materialised matrix, and rplu_cauchy): the same pivots up
  to the first near-tie, a core equal to A(I,J)^{-1} to eps cond^2 (the
  block-inverse recurrence multiplies through the previous inverse twice), and
  A(:,J) core A(I,:) equal to L U -- on Cauchy, dense, sparse (random and a
  power-law graph's adjacency) and Toeplitz operators, in RPLU and C2PLU modes;
  where C2PLU's maxima tie, every choice is checked to be a maximum.
* Exact recovery: a sparse matrix of rank r is reproduced after r steps.
* Reading 27: g = A l as printed, without the conjugate, sends complex pivots
  astray.
* Planted mistakes in a copy of the module (core update sign, residual column
  correction, a transposed Toeplitz factor, row norms from the wrong axis) are
  caught by these pins.
"""
import os
import types

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import cur_form as CF

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "cur_form.py")


def _kernel_matrix(N, length=320.0, delta=50.0, sigma=80.0):
    """A_pq = K(x_p - x_q) over all pairs of grid points, K of Eq. kernel."""
    h = length / N
    g = np.arange(N) * h
    pts = np.array([(a, b, c) for a in g for b in g for c in g])
    d = pts[:, None, :] - pts[None, :, :]
    return np.exp(-(((d[..., 0] - delta) ** 2) + d[..., 1] ** 2 + d[..., 2] ** 2) / (2.0 * sigma ** 2))


def _sparse(n, m, seed, density=0.05):
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    S = sp.random(n, m, density=density, random_state=rng, data_rvs=lambda k: rng.standard_normal(k))
    return S.tocsr()


def _operators():
    x, y = W.cauchy_spirals(120, 100, seed=2)
    rng = np.random.default_rng(3)
    Ad = rng.standard_normal((90, 70)) @ np.diag(0.7 ** np.arange(70)) @ rng.standard_normal((70, 70))
    S = _sparse(150, 130, 4)
    G = W.chung_lu_graph(300, avg_degree=5.0, exponent=2.3, seed=6)
    return {
        "graph": (CF.SparseOperator(G), G.toarray().astype(np.complex128)),
        "cauchy": (CF.CauchyOperator(x, y), 1.0 / (x[:, None] - y[None, :])),
        "dense": (CF.DenseOperator(Ad), Ad.astype(np.complex128)),
        "sparse": (CF.SparseOperator(S), S.toarray().astype(np.complex128)),
        "toeplitz": (CF.KroneckerToeplitz(5), _kernel_matrix(5).astype(np.complex128)),
    }


@pytest.mark.parametrize("name", ["cauchy", "dense", "sparse", "graph", "toeplitz"])
def test_operator_accesses_match_the_matrix(name):
    op, A = _operators()[name]
    n, m = A.shape
    assert op.shape == (n, m)
    rng = np.random.default_rng(5)
    scale = np.max(np.abs(A))
    for i in rng.integers(0, n, 5):
        np.testing.assert_allclose(op.row(i), A[i], rtol=0, atol=1e-14 * scale)
    for j in rng.integers(0, m, 5):
        np.testing.assert_allclose(op.col(j), A[:, j], rtol=0, atol=1e-14 * scale)
    I, J = rng.integers(0, n, 7), rng.integers(0, m, 6)
    np.testing.assert_allclose(op.entries(I, J), A[np.ix_(I, J)], rtol=0, atol=1e-14 * scale)
    v = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    np.testing.assert_allclose(op.matvec(v), A @ v, rtol=0, atol=1e-12 * scale * np.sum(np.abs(v)))
    np.testing.assert_allclose(op.row_norms(), np.sum(np.abs(A) ** 2, axis=1), rtol=1e-12, atol=0)


def test_toeplitz_kronecker_closed_forms():
    op = CF.KroneckerToeplitz(6)
    A = _kernel_matrix(6)
    s = np.linalg.svd(A, compute_uv=False)
    s1 = np.linalg.svd(op.T1, compute_uv=False)
    s0 = np.linalg.svd(op.T0, compute_uv=False)
    prod = np.sort(np.einsum("a,b,c->abc", s1, s0, s0).ravel())[::-1]
    np.testing.assert_allclose(s, prod, rtol=0, atol=1e-12 * s[0])
    # the drift makes T1 non-symmetric (a transposed factor is a different matrix)
    assert np.max(np.abs(op.T1 - op.T1.T)) > 0.1


def _near_tie_step(r, thresh):
    """First step whose row or column draw lies within thresh (a scalar or one
    value per step, relative to that step's total) of a CDF boundary."""
    m_ = np.minimum(r["row_margin"], r["col_margin"])
    bad = np.nonzero(m_ < np.broadcast_to(thresh, m_.shape))[0]
    return int(bad[0]) if len(bad) else r["k_done"]


def _argmax_tie_step(A, o, rel=1e-9):
    """First step of an argmax-mode run at which the exact residual's largest
    row norm, or the chosen row's largest squared entry, is within rel of the
    runner-up (the two forms round differently there, so either may win)."""
    for t in range(o["k_done"]):
        S = A - o["L"][:, :t] @ o["U"][:t]
        for w in (np.sum(np.abs(S) ** 2, axis=1), np.abs(S[o["I"][t]]) ** 2):
            top = np.sort(w)[-2:]
            if top[1] - top[0] <= rel * top[1]:
                return t
    return o["k_done"]


def _check_c2_choices_are_maxima(A, c, rel=1e-9):
    """Where the maxima tie several pivot sequences are correct: every step of
    the run picked a row of largest norm, and in it an entry of largest
    modulus, of its own exact residual A - A(:,J) A(I,J)^{-1} A(I,:)."""
    I, J = c["I"], c["J"]
    for t in range(c["k_done"]):
        S = A - (A[:, J[:t]] @ np.linalg.solve(A[np.ix_(I[:t], J[:t])], A[I[:t], :]) if t else 0.0)
        if np.sum(np.abs(S) ** 2) <= 1e-10 * np.sum(np.abs(A) ** 2):
            break  # the updated row norms' rounding (eps ||A||_F^2) decides from here on
        w = np.sum(np.abs(S) ** 2, axis=1)
        assert w[I[t]] >= (1.0 - rel) * w.max(), t
        r = np.abs(S[I[t]]) ** 2
        assert r[J[t]] >= (1.0 - rel) * r.max(), t


def _check_against_lu(op, A, k, seed, mode, lu=None):
    c = CF.rplu_cur(op, k, seed=seed, mode=mode)
    o = lu if lu is not None else oracle.rplu_dense(A, k, seed=seed, mode=mode)
    T = o["T"]
    # pivots are compared while the residual is well above the row-norm update's
    # absolute rounding (eps ||A_i||^2) and away from near-ties
    live = np.nonzero(T[:-1] <= 1e-9 * T[0])[0]
    upto = int(live[0]) if len(live) else o["k_done"]
    if mode == "random":
        # the CUR form's row norms carry an absolute error of order eps ||A||_F^2,
        # i.e. eps T_0 / T_t relative to the step's total
        thr = 1e-11 * T[0] / np.maximum(T[:o["k_done"]], 1e-300)
        upto = min(upto, _near_tie_step(o, thr))
    else:
        upto = min(upto, _argmax_tie_step(A, o))
        _check_c2_choices_are_maxima(A, c)
    # C2PLU on a 0/1 adjacency ties at once (a row's entries are all 1): there
    # the check of every choice against its residual's maxima is the pin
    assert upto >= (3 if mode == "random" else 0), upto
    if upto == 0:
        return c, o, upto
    assert np.array_equal(c["I"][:upto], o["I"][:upto]) and np.array_equal(c["J"][:upto], o["J"][:upto])
    Ik, Jk = c["I"][:upto], c["J"][:upto]
    W_ = A[np.ix_(Ik, Jk)]
    cond = np.linalg.cond(W_)
    if upto == c["k_done"]:
        err = np.linalg.norm(c["core"] @ W_ - np.eye(upto))
        assert err <= max(100 * upto * 1.1e-16 * cond * cond, 1e-13 * upto), (err, cond)
    lu_prod = o["L"][:, :upto] @ o["U"][:upto]
    cur = A[:, Jk] @ np.linalg.solve(W_, A[Ik, :])
    assert np.linalg.norm(cur - lu_prod) <= 1e-9 * np.linalg.norm(A)
    return c, o, upto


@pytest.mark.parametrize("name", ["cauchy", "dense", "sparse", "graph", "toeplitz"])
@pytest.mark.parametrize("mode", ["random", "c2"])
def test_cur_form_reproduces_the_lu_form(name, mode):
    op, A = _operators()[name]
    k = {"cauchy": 25, "dense": 20, "sparse": 25, "graph": 30, "toeplitz": 12}[name]
    _check_against_lu(op, A, k, seed=17, mode=mode)


@pytest.mark.parametrize("seed", [1, 2])
def test_cur_form_reproduces_the_matrix_free_lu_oracle(seed):
    x, y = W.cauchy_spirals(220, 200, seed=seed)
    o = oracle.rplu_cauchy(x, y, 25, seed=seed + 10)
    c = CF.rplu_cur(CF.CauchyOperator(x, y), 25, seed=seed + 10)
    upto = _near_tie_step(o, 1e-11)
    upto = min(upto, int(np.argmax(np.append(o["T"][:-1] / o["T"][0], 0.0) <= 1e-9)))
    assert upto >= 10
    assert np.array_equal(c["I"][:upto], o["I"][:upto]) and np.array_equal(c["J"][:upto], o["J"][:upto])


def test_given_pivots_and_tolerance_stop():
    op, A = _operators()["dense"]
    o = oracle.rplu_dense(A, 15, seed=3)
    c = CF.rplu_cur(op, 15, mode="given", given=(o["I"], o["J"]))
    assert np.array_equal(c["I"], o["I"]) and np.array_equal(c["J"], o["J"])
    np.testing.assert_allclose(c["core"] @ A[np.ix_(o["I"], o["J"])], np.eye(15), atol=1e-8)
    t = CF.rplu_cur(op, 60, seed=3, tol=1e-3)
    T = t["T"]
    assert t["k_done"] < 60 and T[-1] <= 1e-6 * T[0] and np.all(T[:-1] > 1e-6 * T[0])


def test_exact_recovery_of_a_sparse_rank_r_matrix():
    """Block diagonal with r rank-one sparse blocks: after r steps the CUR
    approximation is A itself and the row norms vanish."""
    import scipy.sparse as sp
    rng = np.random.default_rng(8)
    blocks = []
    for _ in range(6):
        u = rng.standard_normal(rng.integers(3, 9)) * (rng.random() + 0.5)
        v = rng.standard_normal(rng.integers(3, 9))
        blocks.append(sp.csr_matrix(np.outer(u, v)))
    S = sp.block_diag(blocks).tocsr()
    A = S.toarray()
    c = CF.rplu_cur(CF.SparseOperator(S), 6, seed=4)
    assert c["k_done"] == 6
    I, J = c["I"], c["J"]
    np.testing.assert_allclose(A[:, J] @ c["core"] @ A[I, :], A, atol=1e-12 * np.abs(A).max())
    # the row norms are updated, not recomputed: what is left is their rounding,
    # of order eps ||A||_F^2
    assert c["T"][-1] <= 1e-14 * c["T"][0]
    c8 = CF.rplu_cur(CF.SparseOperator(S), 8, seed=4, tol=1e-6)
    assert c8["k_done"] == 6


def test_g_without_the_conjugate_diverges():
    """Reading 27: with g = A l as printed (no conjugate) on complex data the
    row-norm estimates go wrong and the pivots leave the oracle's."""
    x, y = W.cauchy_spirals(220, 200, seed=3)
    o = oracle.rplu_cauchy(x, y, 25, seed=7)
    c = CF.rplu_cur(CF.CauchyOperator(x, y), 25, seed=7, conj_g=False)
    n_same = 0
    while n_same < min(len(c["I"]), len(o["I"])) and c["I"][n_same] == o["I"][n_same] \
            and c["J"][n_same] == o["J"][n_same]:
        n_same += 1
    assert n_same < 25


def _mutant(old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("cur_form_mutant")
    exec(compile(src.replace(old, new), "cur_form_mutant", "exec"), mod.__dict__)
    return mod


MUTANTS = [
    ("core_update_sign", "new[:-1, :-1] = Uc + np.outer(e, b) / sigma", "new[:-1, :-1] = Uc - np.outer(e, b) / sigma",
     "lu"),
    ("residual_column_plus", "c = c - ep * cols_J[p_]", "c = c + ep * cols_J[p_]", "lu"),
    ("toeplitz_factor_transposed", 'X = np.einsum("ab,bjk->ajk", self.T1, X)',
     'X = np.einsum("ba,bjk->ajk", self.T1, X)', "access"),
    ("toeplitz_row_norms_wrong_axis", "r1 = np.sum(self.T1 ** 2, axis=1)", "r1 = np.sum(self.T1 ** 2, axis=0)",
     "access"),
]


def _pin(mod, pin):
    """The pin a mutant must fail: the Toeplitz operator's matvec and row norms
    against the kernel matrix ("access"), or Algorithm 2 against the LU oracle
    ("lu": the first 8 pivots, and a core equal to A(I,J)^{-1} at k = 12, where
    cond A(I,J) ~ 1e4 leaves the unmutated recurrence ~1e-8 from it)."""
    if pin == "access":
        op, A = mod.KroneckerToeplitz(5), _kernel_matrix(5).astype(np.complex128)
        v = np.random.default_rng(1).standard_normal(op.shape[1]) + 0j
        np.testing.assert_allclose(op.matvec(v), A @ v, rtol=0, atol=1e-10)
        np.testing.assert_allclose(op.row_norms(), np.sum(np.abs(A) ** 2, axis=1), rtol=1e-12)
        return
    x, y = W.cauchy_spirals(120, 100, seed=2)
    A = 1.0 / (x[:, None] - y[None, :])
    c = mod.rplu_cur(mod.CauchyOperator(x, y), 12, seed=17)
    o = oracle.rplu_dense(A, 12, seed=17)
    assert np.array_equal(c["I"][:8], o["I"][:8]) and np.array_equal(c["J"][:8], o["J"][:8])
    k = c["k_done"]
    W_ = A[np.ix_(c["I"], c["J"])]
    assert np.linalg.norm(c["core"] @ W_ - np.eye(k)) <= 1e-6


@pytest.mark.parametrize("pin", ["access", "lu"])
def test_mutant_pins_pass_on_the_oracle(pin):
    _pin(CF, pin)


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_are_caught(name, old, new, pin):
    mod = _mutant(old, new)
    with pytest.raises(AssertionError):
        _pin(mod, pin)


@pytest.mark.parametrize("name", ["cauchy", "toeplitz"])
def test_qr_core_agrees_and_is_the_stable_variant(name):
    """Sec. 4.1: the block-inverse update may be unstable when A(I,J) is ill
    conditioned; a QR of A(I,J) is the stable alternative.  Both cores give the
    same pivots while A(I,J) is well conditioned; the QR core's error grows like
    eps cond, the updated inverse's like eps cond^2."""
    op = CF.CauchyOperator(*W.cauchy_spirals(120, 100, seed=2)) if name == "cauchy" \
        else CF.KroneckerToeplitz(6, length=30.0)
    A = op.dense()
    for k in (8, 14):
        a = CF.rplu_cur(op, k, seed=17)
        q = CF.rplu_cur(op, k, seed=17, core="qr")
        assert np.array_equal(a["I"], q["I"]) and np.array_equal(a["J"], q["J"])
        Wm = A[np.ix_(q["I"], q["J"])]
        cond = np.linalg.cond(Wm)
        e_inv = np.linalg.norm(a["core"] @ Wm - np.eye(k))
        e_qr = np.linalg.norm(q["core"] @ Wm - np.eye(k))
        assert e_qr <= 100 * k * 1.1e-16 * cond
        assert e_inv <= 100 * k * 1.1e-16 * cond * cond
        if cond > 1e6:
            assert e_qr * 100 <= e_inv


def test_toeplitz_operator_at_the_papers_grid():
    """At N = 128 (n = 2.1e6, the paper's smaller grid) the Kronecker row norms and
    the mode-product matvec equal direct sums of the kernel over all grid points
    for sampled rows."""
    N = 128
    op = CF.KroneckerToeplitz(N)
    h = 320.0 / N
    g = np.arange(N) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    rng = np.random.default_rng(3)
    rows = rng.integers(0, N ** 3, 4)
    d = op.row_norms()
    u = rng.standard_normal(N ** 3)
    Au = op.matvec(u).real
    for p in rows:
        diff = pts[p] - pts
        k = np.exp(-(((diff[:, 0] - 50.0) ** 2) + diff[:, 1] ** 2 + diff[:, 2] ** 2) / (2.0 * 80.0 ** 2))
        assert d[p] == pytest.approx(np.sum(k * k), rel=1e-12)
        assert Au[p] == pytest.approx(np.dot(k, u), rel=1e-9, abs=1e-12 * np.sum(np.abs(k * u)))
