"""Algorithm 2 as printed (RPLU in CUR form, Sec. 4.1), written out step by
step in numpy with the oracle's draws, against the oracle's matrix-free LU
form: the same pivots, a core equal to A(I,J)^{-1}, and A(:,J) core A(I,:)
equal to L U.  This pins the CUR-form recurrences the GPU's rplu_cauchy_cur
uses -- the residual row r - A(I,:)^T U^T r(J), the residual column
c - A(:,J) U c(I), the row-norm update through g - A(:,J) U g(I), and the
block-inverse core update (Eq. block-inverse-update) -- including reading
27: g = A conj(l), not A l."""
import numpy as np
import pytest

import oracle
import workloads as W


def _cauchy_row(x, y, i):
    return 1.0 / (x[i] - y)


def _cauchy_col(x, y, j):
    return 1.0 / (x - y[j])


def cur_form(x, y, k, seed, conj_g=True):
    x = np.asarray(x, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    n, m = len(x), len(y)
    d = np.array([np.sum(np.abs(_cauchy_row(x, y, p)) ** 2) for p in range(n)])
    T0 = float(np.cumsum(d)[-1])
    Uc = np.zeros((0, 0), dtype=np.complex128)
    I, J, T_hist = [], [], []
    row_used = np.zeros(n, bool)
    col_used = np.zeros(m, bool)
    for t in range(k):
        T = float(np.cumsum(d)[-1])
        T_hist.append(T)
        if not T > 0.0:
            break
        ok = False
        for attempt in range(64):
            i, _ = oracle.inverse_cdf(d, oracle.u01(seed, t, 0, attempt) * T, T)
            z = _cauchy_row(x, y[J], i) if J else np.zeros(0, np.complex128)  # A(i, J)
            b = z @ Uc                                                        # b^T = A(i,J) U
            r = _cauchy_row(x, y, i)
            for s_, bs in enumerate(b):
                r = r - bs * _cauchy_row(x, y, I[s_])                          # r - A(I,:)^T U^T r(J)
            wcol = np.where(col_used, 0.0, np.abs(r) ** 2)
            R = float(np.cumsum(wcol)[-1])
            if not R > 0.0:
                d[i] = 0.0
                T = float(np.cumsum(d)[-1])
                if not T > 0.0:
                    break
                continue
            j, _ = oracle.inverse_cdf(wcol, oracle.u01(seed, t, 1, attempt) * R, R)
            ok = True
            break
        if not ok:
            break
        a = r[j]
        u = np.where(col_used, 0.0, r)
        w = np.array([_cauchy_row(x, y, I[s_])[j] for s_ in range(len(I))], dtype=np.complex128)  # A(I, j)
        e = Uc @ w
        c = _cauchy_col(x, y, j)
        for p_, ep in enumerate(e):
            c = c - ep * _cauchy_col(x, y, J[p_])                              # c - A(:,J) U c(I)
        row_used[i] = True
        col_used[j] = True
        lmul = np.where(row_used, 0.0, c / a)
        lmul[i] = 1.0
        # g = A conj(u) - A(:,J) U (A(I,:) conj(u))  =  S^(t) conj(u)
        cu = np.conj(u) if conj_g else u
        g = np.array([_cauchy_row(x, y, p) @ cu for p in range(n)])
        gI = g[I] if I else np.zeros(0, np.complex128)
        h = Uc @ gI
        for p_, hp in enumerate(h):
            g = g - hp * _cauchy_col(x, y, J[p_])
        un2 = float(np.sum(np.abs(u) ** 2))
        d = np.maximum(0.0, d - 2.0 * np.real(np.conj(lmul) * g) + np.abs(lmul) ** 2 * un2)
        d[row_used] = 0.0
        # block inverse: [[U + e b^T/a, -e/a], [-b^T/a, 1/a]]
        t1 = len(I) + 1
        new = np.zeros((t1, t1), dtype=np.complex128)
        new[:-1, :-1] = Uc + np.outer(e, b) / a
        new[:-1, -1] = -e / a
        new[-1, :-1] = -b / a
        new[-1, -1] = 1.0 / a
        Uc = new
        I.append(i)
        J.append(j)
    return np.array(I, np.int64), np.array(J, np.int64), Uc, np.array(T_hist), T0


@pytest.mark.parametrize("seed", [1, 2])
def test_cur_form_reproduces_the_lu_form(seed):
    x, y = W.cauchy_spirals(220, 200, seed=seed)
    k = 25
    o = oracle.rplu_cauchy(x, y, k, seed=seed + 10)
    I, J, Uc, T, _ = cur_form(x, y, k, seed + 10)
    # the same pivots up to the first step whose draw the oracle reports as a near-tie
    m_ = np.minimum(o["row_margin"], o["col_margin"])
    thr = 1e-11 * o["T"][0] / np.maximum(o["T"][:-1], 1e-300)
    bad = np.nonzero(m_ < thr)[0]
    upto = int(bad[0]) if len(bad) else o["k_done"]
    assert upto >= 10
    assert np.array_equal(I[:upto], o["I"][:upto]) and np.array_equal(J[:upto], o["J"][:upto])
    A = W.cauchy_dense(x, y)
    Ik, Jk = I[:upto], J[:upto]
    Wm = A[np.ix_(Ik, Jk)]
    cond = np.linalg.cond(Wm)
    if upto == len(I):
        assert np.linalg.norm(Uc @ Wm - np.eye(upto)) <= 100 * upto * 1.1e-16 * cond * cond
    lu = o["L"][:, :upto] @ o["U"][:upto]
    cur = A[:, Jk] @ np.linalg.solve(Wm, A[Ik, :])
    assert np.linalg.norm(cur - lu) <= 1e-9 * np.linalg.norm(A)


def test_g_without_the_conjugate_diverges():
    """Reading 27: with g = A l as printed (no conjugate) on complex data the
    row-norm estimates go wrong and the pivots leave the oracle's."""
    x, y = W.cauchy_spirals(220, 200, seed=3)
    o = oracle.rplu_cauchy(x, y, 25, seed=7)
    I, J, _, T, _ = cur_form(x, y, 25, 7, conj_g=False)
    n_same = 0
    while n_same < min(len(I), len(o["I"])) and I[n_same] == o["I"][n_same] and J[n_same] == o["J"][n_same]:
        n_same += 1
    assert n_same < 25
