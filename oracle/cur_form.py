"""Oracle for RPLU in CUR form (Algorithm 2, Sec. 4.1) over a general
operator: TEST INFRASTRUCTURE ONLY (imported by tests/; never by the library).

Algorithm 2 touches A only through a few accesses, which every operator below
provides in FP64 / complex128:
  shape               (n, m)
  row(i), col(j)      A(i,:) and A(:,j)
  entries(I, J)       the block A(I,J)
  matvec(v)           A v
  row_norms()         ||A(i,:)||^2 for every i (the initial row norms)

Operators:
  DenseOperator       a stored matrix.
  CauchyOperator      A_pq = 1/(x_p - y_q), entries generated (Sec. 5.1, p = 1).
  SparseOperator      a scipy.sparse matrix (Sec. 4.3: sparse graph matrices).
  KroneckerToeplitz   the multi-level Toeplitz matrix of Sec. 4.2: the drifted
                      Gaussian kernel of Eq. kernel on a Cartesian N^3 grid,
                      A_pq = K(x_p - x_q).  K is a product of one-dimensional
                      Gaussians, so A = T_1 (x) T_2 (x) T_3 exactly (Kronecker
                      product of three N x N Toeplitz matrices, x the slowest
                      index) and a matvec is three mode products.

The factorization (rplu_cur) follows Algorithm 2's steps in its order:
  step 1  row i by the row norms n_k; the residual row
          r^ = r - A(I,:)^T U^T r(J)  (here: b^T = A(i,J) U, r^ = r - b^T A(I,:));
          column j by |r^|^2 with the pivoted columns masked; the residual
          column c^ = c - A(:,J) U c(I);
  step 2  l = r^ / r^_j (pivoted columns zero); g = A conj(l) - A(:,J) U g(I)
          (reading: the conjugate, which Algorithm 2 omits, is the one of the
          row-norm formula of Sec. 4.1; without it complex data go wrong);
          n_{k+1} = n_k - 2 Re((g) conj(c^)) + ||l||^2 |c^|^2, clamped at 0,
          pivoted rows set to 0;
  step 3  the core U = A(I,J)^{-1} by the block-inverse update of Eq.
          block-inverse-update, sigma = omega - z^T U w.
Draws, redraws and the stop rule are those of the LU oracle (rplu_oracle.c):
U01(seed, t, s, a), the smallest index whose prefix sum exceeds u * total,
at most 64 row draws per step (a row whose masked weights sum to zero gets
n_i = 0 and is drawn again), stop when the total is 0 or <= tol^2 * initial.
Modes: "random" (RPLU), "c2" (C2PLU: the first maximum instead of each draw),
"given" (caller's pivots).
"""
from __future__ import annotations

import numpy as np

MAX_ATTEMPTS = 64


# ----------------------------------------------------------------- operators

class DenseOperator:
    def __init__(self, A):
        self.A = np.asarray(A, dtype=np.complex128)
        self.shape = self.A.shape

    def row(self, i):
        return self.A[i].copy()

    def col(self, j):
        return self.A[:, j].copy()

    def entries(self, I, J):
        return self.A[np.ix_(np.asarray(I, int), np.asarray(J, int))]

    def matvec(self, v):
        return self.A @ v

    def row_norms(self):
        return np.sum(np.abs(self.A) ** 2, axis=1)

    def dense(self):
        return self.A.copy()


class CauchyOperator:
    def __init__(self, x, y):
        self.x = np.asarray(x, dtype=np.complex128)
        self.y = np.asarray(y, dtype=np.complex128)
        self.shape = (len(self.x), len(self.y))

    def row(self, i):
        return 1.0 / (self.x[i] - self.y)

    def col(self, j):
        return 1.0 / (self.x - self.y[j])

    def entries(self, I, J):
        return 1.0 / (self.x[np.asarray(I, int)][:, None] - self.y[np.asarray(J, int)][None, :])

    def matvec(self, v):
        out = np.empty(self.shape[0], dtype=np.complex128)
        for p in range(self.shape[0]):
            out[p] = np.sum(v / (self.x[p] - self.y))
        return out

    def row_norms(self):
        return np.array([np.sum(np.abs(1.0 / (xp - self.y)) ** 2) for xp in self.x])

    def dense(self):
        return 1.0 / (self.x[:, None] - self.y[None, :])


class SparseOperator:
    def __init__(self, S):
        import scipy.sparse as sp

        self.csr = sp.csr_matrix(S, dtype=np.complex128)
        self.csc = self.csr.tocsc()
        self.shape = self.csr.shape

    def row(self, i):
        out = np.zeros(self.shape[1], dtype=np.complex128)
        lo, hi = self.csr.indptr[i], self.csr.indptr[i + 1]
        out[self.csr.indices[lo:hi]] = self.csr.data[lo:hi]
        return out

    def col(self, j):
        out = np.zeros(self.shape[0], dtype=np.complex128)
        lo, hi = self.csc.indptr[j], self.csc.indptr[j + 1]
        out[self.csc.indices[lo:hi]] = self.csc.data[lo:hi]
        return out

    def entries(self, I, J):
        return self.csr[np.asarray(I, int)][:, np.asarray(J, int)].toarray()

    def matvec(self, v):
        return self.csr @ v

    def row_norms(self):
        return np.asarray(abs(self.csr).power(2).sum(axis=1)).ravel()

    def dense(self):
        return self.csr.toarray()


class KroneckerToeplitz:
    """A_pq = K(x_p - x_q) on the grid {0, h, ..., (N-1) h}^3 with the drifted
    Gaussian K(d) = exp(-((d_1 - delta)^2 + d_2^2 + d_3^2) / (2 sigma^2))
    (Eq. kernel); p = (a N + b) N + c for the grid point (a h, b h, c h)."""

    def __init__(self, N: int, length: float = 320.0, delta: float = 50.0, sigma: float = 80.0):
        self.N = int(N)
        self.h = length / self.N
        self.delta, self.sigma = float(delta), float(sigma)
        n = self.N ** 3
        self.shape = (n, n)
        d = (np.arange(self.N)[:, None] - np.arange(self.N)[None, :]) * self.h
        self.T1 = np.exp(-((d - self.delta) ** 2) / (2.0 * self.sigma ** 2))
        self.T0 = np.exp(-(d ** 2) / (2.0 * self.sigma ** 2))

    def _digits(self, p):
        p = np.asarray(p, dtype=np.int64)
        return p // (self.N * self.N), (p // self.N) % self.N, p % self.N

    def row(self, i):
        a, b, c = self._digits(i)
        return np.kron(np.kron(self.T1[a], self.T0[b]), self.T0[c]).astype(np.complex128)

    def col(self, j):
        a, b, c = self._digits(j)
        return np.kron(np.kron(self.T1[:, a], self.T0[:, b]), self.T0[:, c]).astype(np.complex128)

    def entries(self, I, J):
        ai, bi, ci = self._digits(I)
        aj, bj, cj = self._digits(J)
        return (self.T1[np.ix_(ai, aj)] * self.T0[np.ix_(bi, bj)] * self.T0[np.ix_(ci, cj)]).astype(np.complex128)

    def matvec(self, v):
        N = self.N
        X = np.asarray(v, dtype=np.complex128).reshape(N, N, N)
        X = np.einsum("ab,bjk->ajk", self.T1, X)
        X = np.einsum("ab,ibk->iak", self.T0, X)
        X = np.einsum("ab,ijb->ija", self.T0, X)
        return X.reshape(-1)

    def row_norms(self):
        r1 = np.sum(self.T1 ** 2, axis=1)
        r0 = np.sum(self.T0 ** 2, axis=1)
        return np.kron(np.kron(r1, r0), r0)

    def dense(self):
        return np.kron(np.kron(self.T1, self.T0), self.T0).astype(np.complex128)


# ------------------------------------------------------------- Algorithm 2

def _qr_solve(W, v):
    """W^{-1} v through a Householder QR of W (R x = Q^* v)."""
    if W.shape[0] == 0:
        return np.zeros(0, dtype=np.complex128)
    Q, R = np.linalg.qr(W)
    return np.linalg.solve(np.triu(R), Q.conj().T @ v)


def _qr_solve_t(W, z):
    """z^T W^{-1}, i.e. the solution b of W^T b = z, through a QR of W^T."""
    return _qr_solve(W.T, z)


def _first_max(w):
    return int(np.argmax(w)) if len(w) and np.max(w) > 0.0 else -1


def rplu_cur(op, k: int, seed: int = 0, mode: str = "random", tol: float = 0.0, given=None,
             conj_g: bool = True, core: str = "inverse") -> dict:
    """RPLU (or C2PLU) in CUR form on the operator `op` (module header).

    Returns I, J (pivots in order), core (A(I,J)^{-1}, k_done x k_done),
    T (the total of the row norms before each step and after the last),
    d (the final row norms), row_margin / col_margin (distance of each draw
    from the nearest CDF boundary, relative to the total; 0 in other modes)
    and k_done.  conj_g=False evaluates g = A l as Algorithm 2 prints it (for
    the test that shows why the conjugate is needed).  core="inverse" keeps
    U = A(I,J)^{-1} by the block-inverse update (Eq. block-inverse-update);
    core="qr" keeps W = A(I,J) and applies W^{-1} through a QR factorization
    of W recomputed every step (the variant Sec. 4.1 prefers for stability;
    numpy's QR, a LAPACK Householder QR), the returned core then being
    W^{-1} from that QR."""
    import oracle

    n, m = op.shape
    if k < 0 or k > min(n, m):
        raise ValueError("k must be in 0..min(n, m)")
    d = np.asarray(op.row_norms(), dtype=np.float64).copy()
    T0 = float(np.sum(d))
    I, J = [], []
    rows_I, cols_J = [], []              # A(I_s,:) and A(:,J_s), regenerated in the GPU path
    Uc = np.zeros((0, 0), dtype=np.complex128)
    Wc = np.zeros((0, 0), dtype=np.complex128)  # A(I,J), kept when core="qr"
    row_used = np.zeros(n, dtype=bool)
    col_used = np.zeros(m, dtype=bool)
    T_hist, rmarg, cmarg = [], [], []
    for t in range(k):
        T = float(np.sum(d))
        T_hist.append(T)
        if not T > 0.0 or (tol > 0.0 and T <= tol * tol * T0):
            break
        found = False
        rm = cm = 0.0
        for attempt in range(MAX_ATTEMPTS):
            # step 1: row i, its residual row, column j
            if mode == "given":
                i = int(given[0][t])
            elif mode == "c2":
                i = _first_max(d)
            else:
                i, rm = oracle.inverse_cdf(d, oracle.u01(seed, t, 0, attempt) * T, T)
            z = op.entries([i], J)[0] if J else np.zeros(0, np.complex128)   # A(i, J)
            b = z @ Uc if core == "inverse" else _qr_solve_t(Wc, z)            # b^T = A(i,J) U
            r = op.row(i)
            for s_, bs in enumerate(b):
                r = r - bs * rows_I[s_]
            if mode == "given":
                j = int(given[1][t])
                found = True
                break
            wcol = np.where(col_used, 0.0, np.abs(r) ** 2)
            R = float(np.sum(wcol))
            if not R > 0.0:
                d[i] = 0.0
                T = float(np.sum(d))
                if not T > 0.0:
                    break
                continue
            if mode == "c2":
                j = _first_max(wcol)
            else:
                j, cm = oracle.inverse_cdf(wcol, oracle.u01(seed, t, 1, attempt) * R, R)
            found = True
            break
        if not found:
            break
        w = op.entries(I, [j])[:, 0] if I else np.zeros(0, np.complex128)    # A(I, j)
        sigma = r[j]                                                           # omega - z^T U w
        if sigma == 0:
            raise ValueError("zero pivot")
        e = Uc @ w if core == "inverse" else _qr_solve(Wc, w)
        c = op.col(j)
        for p_, ep in enumerate(e):
            c = c - ep * cols_J[p_]                                            # c^ = c - A(:,J) U c(I)
        u = np.where(col_used, 0.0, r)
        row_used[i] = True
        col_used[j] = True
        # step 2: row norms of the next residual
        l = np.where(row_used, 0.0, c / sigma)
        l[i] = 1.0
        g = op.matvec(np.conj(u) if conj_g else u)                             # A conj(u)
        if I:
            h = Uc @ g[np.asarray(I)] if core == "inverse" else _qr_solve(Wc, g[np.asarray(I)])
            for p_, hp in enumerate(h):
                g = g - hp * cols_J[p_]                                        # minus A(:,J) U g(I)
        un2 = float(np.sum(np.abs(u) ** 2))
        d = np.maximum(0.0, d - 2.0 * np.real(np.conj(l) * g) + np.abs(l) ** 2 * un2)
        d[row_used] = 0.0
        # step 3: block-inverse update of the core (Eq. block-inverse-update)
        t1 = len(I) + 1
        new = np.zeros((t1, t1), dtype=np.complex128)
        new[:-1, :-1] = Uc + np.outer(e, b) / sigma
        new[:-1, -1] = -e / sigma
        new[-1, :-1] = -b / sigma
        new[-1, -1] = 1.0 / sigma
        Uc = new
        # W = A(I,J) grown by the new row z^T (columns J) and column w (rows I)
        Wn = np.zeros((t1, t1), dtype=np.complex128)
        Wn[:-1, :-1] = Wc
        Wn[:-1, -1] = w
        Wn[-1, :-1] = z
        Wn[-1, -1] = op.entries([i], [j])[0, 0]  # omega = A(i, j)
        Wc = Wn
        I.append(i)
        J.append(j)
        rows_I.append(op.row(i))
        cols_J.append(op.col(j))
        rmarg.append(rm)
        cmarg.append(cm)
    kd = len(I)
    if len(T_hist) == kd:
        T_hist.append(float(np.sum(d)))
    if core == "qr":
        Uc = _qr_solve(Wc, np.eye(kd, dtype=np.complex128)) if kd else Wc
    return {"I": np.array(I, np.int64), "J": np.array(J, np.int64), "core": Uc, "T": np.array(T_hist[:kd + 1]),
            "d": d, "row_margin": np.array(rmarg), "col_margin": np.array(cmarg), "k_done": kd, "T0": T0}
