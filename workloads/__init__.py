"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the oracle side (tests, CPU baseline) and the CUDA side
(tests, bench): it generates matrices and point sets and nothing else.  It holds
none of the RPLU arithmetic (no sampling, no Schur update, no row-norm update).

Workloads (paper sections in brackets):
  * dense matrices with a prescribed decaying spectrum, A = Q1 diag(sigma) Q2^T
    (Sec. 3, the Fig. 3 bound experiment uses sigma_k = rho^k on 200x200);
  * Cauchy matrices A_ij = 1/(x_i - y_j) on planar point clouds: two
    interleaved Archimedean spirals plus a Gaussian cluster, and a smiley
    (Fig. 1, Sec. 1; Cauchy-like matrices Sec. 5.1 with p = 1, G = B = 1);
  * batches of real Cauchy blocks on separated intervals (hierarchical-matrix
    off-diagonal blocks, Sec. 5.1);
  * exact low-rank products X Y^T.

All randomness comes from numpy's PCG64 (np.random.default_rng(seed)), which is
platform independent, so x86 and aarch64 hosts produce the same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 2601223440


def derive_seed(*parts: int) -> int:
    """Deterministic 63-bit seed from integer parts (workload id, job id, ...)."""
    ss = np.random.SeedSequence([BASE_SEED, *[int(p) for p in parts]])
    return int(ss.generate_state(1, dtype=np.uint64)[0] >> np.uint64(1))


# ---------------------------------------------------------------------------
# Dense matrices with a prescribed spectrum
# ---------------------------------------------------------------------------

def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed n x n orthogonal matrix: QR of a Gaussian matrix with
    the signs of R's diagonal moved into Q (Mezzadri 2007)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def dense_haar_decay(n: int, m: int, rho: float, seed: int) -> np.ndarray:
    """A = Q1 diag(sigma) Q2^T with Q1 (n x n), Q2 (m x m) Haar orthogonal and
    sigma_i = rho**i, i = 0..min(n,m)-1.  FP64, C-contiguous (row-major)."""
    rng = np.random.default_rng(seed)
    q1 = haar_orthogonal(n, rng)
    q2 = haar_orthogonal(m, rng)
    r = min(n, m)
    sigma = rho ** np.arange(r, dtype=np.float64)
    return np.ascontiguousarray((q1[:, :r] * sigma[None, :]) @ q2[:, :r].T)


def dense_with_spectrum(sigma: np.ndarray, n: int, m: int, seed: int) -> np.ndarray:
    """A = Q1 diag(sigma) Q2^T with Haar Q1, Q2 and the given singular values."""
    rng = np.random.default_rng(seed)
    r = len(sigma)
    q1 = haar_orthogonal(n, rng)[:, :r]
    q2 = haar_orthogonal(m, rng)[:, :r]
    return np.ascontiguousarray((q1 * np.asarray(sigma)[None, :]) @ q2.T)


def householder_wy(v: np.ndarray):
    """Compact WY form of H_1 H_2 ... H_k, H_i = I - tau_i v_i v_i^T with
    tau_i = 2 / (v_i^T v_i):  the product equals I - V T V^T, T upper
    triangular (Schreiber & Van Loan 1989).  v has shape (n, k)."""
    n, k = v.shape
    tau = 2.0 / np.einsum("ij,ij->j", v, v)
    t = np.zeros((k, k))
    for j in range(k):
        t[j, j] = tau[j]
        if j:
            t[:j, j] = -tau[j] * (t[:j, :j] @ (v[:, :j].T @ v[:, j]))
    return v, t


@dataclass
class LowRankPlusDiag:
    """A = D + X Y^T, D the n x m matrix with sigma on its main diagonal."""
    n: int
    m: int
    sigma: np.ndarray  # (min(n,m),)
    X: np.ndarray      # (n, r)
    Y: np.ndarray      # (m, r)

    def rows(self, r0: int, r1: int) -> np.ndarray:
        """Rows r0:r1 of A in FP64."""
        out = self.X[r0:r1] @ self.Y.T
        idx = np.arange(r0, min(r1, len(self.sigma)))
        out[idx - r0, idx] += self.sigma[idx]
        return out

    def entries(self, p: np.ndarray, q: np.ndarray) -> np.ndarray:
        """A[p, q] for index arrays p, q of equal length (FP64)."""
        p = np.asarray(p)
        q = np.asarray(q)
        val = np.einsum("ij,ij->i", self.X[p], self.Y[q])
        diag = (p == q) & (p < len(self.sigma))
        val[diag] += self.sigma[p[diag]]
        return val

    def dense(self) -> np.ndarray:
        return self.rows(0, self.n)

    def to_torch(self, device, dtype, block_rows: int = 2048):
        """Materialise A on a torch device: each row block is formed in FP64 and
        rounded once to `dtype`."""
        import torch
        out = torch.empty((self.n, self.m), dtype=dtype, device=device)
        X = torch.from_numpy(self.X).to(device)
        Yt = torch.from_numpy(np.ascontiguousarray(self.Y.T)).to(device)
        sig = torch.from_numpy(self.sigma).to(device)
        for r0 in range(0, self.n, block_rows):
            r1 = min(self.n, r0 + block_rows)
            blk = X[r0:r1] @ Yt
            d1 = min(r1, len(self.sigma))
            if d1 > r0:
                ar = torch.arange(r0, d1, device=device)
                blk[ar - r0, ar] += sig[r0:d1]
            out[r0:r1] = blk.to(dtype)
        return out


def householder_decay(n: int, m: int, sigma: np.ndarray, seed: int,
                      n_reflectors: int = 64) -> LowRankPlusDiag:
    """A = Q1 diag(sigma) Q2^T where Q1 (n x n) and Q2 (m x m) are products of
    `n_reflectors` Householder reflectors with Gaussian vectors.

    With Q1 = I - V1 T1 V1^T, Q2 = I - V2 T2 V2^T, P1 = V1 T1, P2 = V2 T2^T... the
    product expands to D plus a rank-2k term:
        A = D + (P1 M - D V2) P2'^T - P1 (D^T V1)^T,  M = V1^T D V2,
    with P2' = V2 T2 (so that Q2^T = I - V2 T2^T V2^T = I - V2 P2'^T ... ).
    Returned as D + X Y^T with X = [P1 M - D V2, -P1], Y = [V2 T2, D^T V1]."""
    rng = np.random.default_rng(seed)
    k = n_reflectors
    v1 = rng.standard_normal((n, k))
    v2 = rng.standard_normal((m, k))
    V1, T1 = householder_wy(v1)
    V2, T2 = householder_wy(v2)
    r = min(n, m)
    sigma = np.asarray(sigma, dtype=np.float64)[:r]
    # D V2 (n x k): row i < r scaled by sigma_i, rows >= r are zero
    DV2 = np.zeros((n, k))
    DV2[:r] = sigma[:, None] * V2[:r]
    DtV1 = np.zeros((m, k))
    DtV1[:r] = sigma[:, None] * V1[:r]
    P1 = V1 @ T1
    M = V1.T @ DV2
    X = np.hstack([P1 @ M - DV2, -P1])
    Y = np.hstack([V2 @ T2, DtV1])
    return LowRankPlusDiag(n, m, sigma, np.ascontiguousarray(X), np.ascontiguousarray(Y))


def dense_householder_decay(n: int, m: int, sigma: np.ndarray, seed: int,
                            n_reflectors: int = 64) -> np.ndarray:
    return householder_decay(n, m, sigma, seed, n_reflectors).dense()


def lowrank_product(n: int, m: int, r: int, seed: int, complex_: bool = False) -> np.ndarray:
    """Exact rank-r matrix X Y^T with Gaussian factors (complex if asked)."""
    rng = np.random.default_rng(seed)
    if complex_:
        x = rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))
        y = rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))
    else:
        x = rng.standard_normal((n, r))
        y = rng.standard_normal((m, r))
    return np.ascontiguousarray(x @ y.T)


def gaussian(n: int, m: int, seed: int, complex_: bool = False) -> np.ndarray:
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, m))
    if complex_:
        a = a + 1j * rng.standard_normal((n, m))
    return np.ascontiguousarray(a)


# ---------------------------------------------------------------------------
# Cauchy point sets
# ---------------------------------------------------------------------------

def spiral_cluster(n: int, rng: np.random.Generator) -> np.ndarray:
    """n complex points: 40% and 40% on two interleaved Archimedean spirals
    r = theta/(4 pi), theta ~ U[0, 8 pi] (the second rotated by pi), and 20%
    from a Gaussian cluster N(0, 0.05^2) per component at the origin."""
    n1 = (2 * n) // 5
    n2 = (2 * n) // 5
    n3 = n - n1 - n2
    th1 = rng.uniform(0.0, 8 * math.pi, n1)
    th2 = rng.uniform(0.0, 8 * math.pi, n2)
    s1 = (th1 / (4 * math.pi)) * np.exp(1j * th1)
    s2 = (th2 / (4 * math.pi)) * np.exp(1j * (th2 + math.pi))
    c = 0.05 * (rng.standard_normal(n3) + 1j * rng.standard_normal(n3))
    pts = np.concatenate([s1, s2, c])
    return pts[rng.permutation(n)]


def cauchy_spirals(n: int, m: int, seed: int):
    """Points for the spiral Cauchy workload: x from the spiral+cluster recipe,
    y from the same recipe with its own draws, rotated by pi/2 and shifted by 3
    (y <- i*y + 3).  Returns complex128 arrays (x, y)."""
    rng = np.random.default_rng(seed)
    x = spiral_cluster(n, rng)
    y = 1j * spiral_cluster(m, rng) + 3.0
    return np.ascontiguousarray(x), np.ascontiguousarray(y)


def smiley(n: int, rng: np.random.Generator) -> np.ndarray:
    """n complex points on a smiley: unit circle 50%, two eyes 10% each (discs of
    radius 0.1 at (+-0.35, 0.35)), mouth arc 30% (radius 0.6, 200..340 deg)."""
    nf = n // 2
    ne = n // 10
    nm = n - nf - 2 * ne
    face = np.exp(1j * rng.uniform(0, 2 * math.pi, nf))

    def disc(c, k):
        rad = 0.1 * np.sqrt(rng.uniform(0, 1, k))
        ang = rng.uniform(0, 2 * math.pi, k)
        return c + rad * np.exp(1j * ang)

    eyes = np.concatenate([disc(-0.35 + 0.35j, ne), disc(0.35 + 0.35j, ne)])
    ang = np.deg2rad(rng.uniform(200, 340, nm))
    mouth = 0.6 * np.exp(1j * ang)
    pts = np.concatenate([face, eyes, mouth])
    return pts[rng.permutation(n)]


def cauchy_smiley(n: int, m: int, seed: int):
    rng = np.random.default_rng(seed)
    x = smiley(n, rng)
    y = 1j * smiley(m, rng) + 3.0
    return np.ascontiguousarray(x), np.ascontiguousarray(y)


def cauchy_dense(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Materialise A_ij = 1/(x_i - y_j) (test helper for small sizes)."""
    return 1.0 / (np.asarray(x)[:, None] - np.asarray(y)[None, :])


@dataclass
class CauchyBlock:
    x: np.ndarray  # FP64 points (n,), real or complex
    y: np.ndarray  # FP64 points (m,)


def cauchy_interval_blocks(n_blocks: int, seed: int, size_lo: int = 64, size_hi: int = 1024):
    """Real Cauchy blocks 1/(x_i - y_j): n, m ~ U{size_lo..size_hi}
    independently; x ~ U[c_x - 1, c_x + 1], y ~ U[c_y - 1, c_y + 1] with
    |c_x - c_y| ~ U[3, 6] (separated unit intervals, i.e. 1-D unit discs)."""
    rng = np.random.default_rng(seed)
    blocks = []
    for _ in range(n_blocks):
        n = int(rng.integers(size_lo, size_hi + 1))
        m = int(rng.integers(size_lo, size_hi + 1))
        cx = rng.uniform(-10, 10)
        cy = cx + rng.choice([-1.0, 1.0]) * rng.uniform(3.0, 6.0)
        x = rng.uniform(cx - 1, cx + 1, n)
        y = rng.uniform(cy - 1, cy + 1, m)
        blocks.append(CauchyBlock(x, y))
    return blocks


def _unit_disk(rng: np.random.Generator, k: int) -> np.ndarray:
    """k points uniform in the unit disk (radius sqrt(U), angle U[0, 2 pi))."""
    r = np.sqrt(rng.random(k))
    a = rng.uniform(0.0, 2.0 * np.pi, k)
    return r * np.exp(1j * a)


def cauchy_disk_blocks(n_blocks: int, seed: int, size_lo: int = 64, size_hi: int = 1024):
    """Complex Cauchy blocks 1/(x_i - y_j): n, m ~ U{size_lo..size_hi}
    independently; x uniform in the unit disk around c_x, y in the unit disk
    around c_y, |c_x - c_y| ~ U[3, 6] in a uniform direction (separated
    2-D unit discs, the complex variant of the interval blocks)."""
    rng = np.random.default_rng(seed)
    blocks = []
    for _ in range(n_blocks):
        n = int(rng.integers(size_lo, size_hi + 1))
        m = int(rng.integers(size_lo, size_hi + 1))
        cx = complex(rng.uniform(-10, 10), rng.uniform(-10, 10))
        cy = cx + rng.uniform(3.0, 6.0) * np.exp(1j * rng.uniform(0.0, 2.0 * np.pi))
        blocks.append(CauchyBlock(cx + _unit_disk(rng, n), cy + _unit_disk(rng, m)))
    return blocks


def loewner_generators(x: np.ndarray, y: np.ndarray, fx: np.ndarray, fy: np.ndarray):
    """Generators (G n x 2, B 2 x m) of the Loewner matrix
    L_ij = (fx_i - fy_j) / (x_i - y_j): G = [fx/alpha, alpha], B = [alpha; -fy/alpha]
    with alpha = sqrt(max(max|fx|, max|fy|)) (the scaling stated in Sec. 5.2)."""
    fx = np.asarray(fx)
    fy = np.asarray(fy)
    alpha = np.sqrt(max(np.max(np.abs(fx)), np.max(np.abs(fy))))
    G = np.stack([fx / alpha, np.full(len(fx), alpha, dtype=np.result_type(fx, float))], axis=1)
    B = np.stack([np.full(len(fy), alpha, dtype=np.result_type(fy, float)), -fy / alpha], axis=0)
    return G, B


def loewner_experiment(kind: str, n: int, seed: int):
    """Inputs of the Loewner experiments of Sec. 5.2 (Fig. 7), n = m points:
    kind "sin": f(z) = sin(1000 z), x and y uniform on [-1, 1] (real data);
    kind "tan": f(z) = tan(20 z^20), x and y uniform on the unit disk
    {|z| <= 1} (complex data).  Returns (x, y, G, B) with the generators of
    loewner_generators.  Draws whose x_i coincides with some y_j (probability
    zero) are not filtered."""
    rng = np.random.default_rng(seed)
    if kind == "sin":
        x = rng.uniform(-1.0, 1.0, n)
        y = rng.uniform(-1.0, 1.0, n)
        f = lambda z: np.sin(1000.0 * z)  # noqa: E731
    elif kind == "tan":
        x = np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
        y = np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
        f = lambda z: np.tan(20.0 * z ** 20)  # noqa: E731
    else:
        raise ValueError(kind)
    G, B = loewner_generators(x, y, f(x), f(y))
    return x, y, G, B


def cauchy_like_dense(x, y, G, B) -> np.ndarray:
    """Materialise A_ij = sum_l G[i,l] B[l,j] / (x_i - y_j) (test helper)."""
    return (np.asarray(G) @ np.asarray(B)) / (np.asarray(x)[:, None] - np.asarray(y)[None, :])


def serving_pool(n_cauchy: int, n_dense: int, seed: int, cauchy_range=(64, 4096), dense_range=(256, 2048),
                 dense_decay: float = 0.9, clouds: bool = False):
    """Request inputs for the serving workload.  Cauchy requests, n and m drawn
    log-uniformly from cauchy_range: with clouds, complex points on the
    spiral-and-cluster and smiley clouds (half each; cauchy_spirals and
    cauchy_smiley, own draws per request), else real points on separated unit
    intervals (as cauchy_interval_blocks).  Dense requests: square n x n with n
    log-uniform in dense_range, A = Q1 diag(dense_decay^i) Q2^T with Q1, Q2
    products of 64 Householder reflectors, returned as LowRankPlusDiag
    factories (materialised where they are used)."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(cauchy_range[0]), np.log(cauchy_range[1])
    cauchy = []
    for q in range(n_cauchy):
        n = int(round(np.exp(rng.uniform(lo, hi))))
        m = int(round(np.exp(rng.uniform(lo, hi))))
        if clouds:
            gen = cauchy_spirals if q % 2 == 0 else cauchy_smiley
            x, y = gen(n, m, seed=derive_seed(seed, 7, q))
            cauchy.append(CauchyBlock(x, y))
            continue
        cx = rng.uniform(-10, 10)
        cy = cx + rng.choice([-1.0, 1.0]) * rng.uniform(3.0, 6.0)
        cauchy.append(CauchyBlock(rng.uniform(cx - 1, cx + 1, n), rng.uniform(cy - 1, cy + 1, m)))
    lo, hi = np.log(dense_range[0]), np.log(dense_range[1])
    dense = []
    for q in range(n_dense):
        n = int(round(np.exp(rng.uniform(lo, hi))))
        dense.append(householder_decay(n, n, dense_decay ** np.arange(n), seed=derive_seed(seed, q)))
    return cauchy, dense


def chung_lu_graph(n: int, avg_degree: float, exponent: float, seed: int):
    """Symmetric 0/1 adjacency (scipy CSR, float64) of a Chung-Lu random graph
    with a power-law degree sequence: expected degrees w_p proportional to
    (p + 1)^(-1/(exponent - 1)), scaled to the mean avg_degree (Chung & Lu,
    "Connected components in random graphs with given expected degree
    sequences", 2002).  Sampled in the usual fast form: a Poisson(sum(w)/2)
    number of edges whose endpoints are drawn independently in proportion to
    w; repeated edges and self loops are dropped.  Stands in for the paper's
    sparse network matrices (Sec. 4.3: talk, traffic and circuit graphs with
    10^6 - 10^7 rows and a few nonzeros per row)."""
    import scipy.sparse as sp

    if n < 2 or avg_degree <= 0 or exponent <= 2.0:
        raise ValueError("need n >= 2, avg_degree > 0 and exponent > 2")
    rng = np.random.default_rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (exponent - 1.0))
    w *= avg_degree * n / w.sum()
    n_edges = int(rng.poisson(w.sum() / 2.0))
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    a = np.searchsorted(cdf, rng.random(n_edges), side="right")
    b = np.searchsorted(cdf, rng.random(n_edges), side="right")
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo.astype(np.int64) * n + hi)
    lo, hi = key // n, key % n
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    S = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    perm = rng.permutation(n)  # hubs spread over the index range
    return S[perm][:, perm].tocsr()


def toeplitz_kernel_grid(N: int) -> dict:
    """The multi-level Toeplitz workload of Sec. 4.2: the drifted Gaussian
    kernel of Eq. kernel (shift 50 along the first axis, standard deviation 80)
    on the Cartesian grid {0, h, ..., (N - 1) h}^3 of [0, 320]^3, h = 320 / N,
    n = N^3 (the paper uses N = 128 and 320).  Parameters only: the matrix
    A_pq = K(x_p - x_q) is formed by whoever consumes it."""
    return {"N": int(N), "length": 320.0, "delta": 50.0, "sigma": 80.0, "h": 320.0 / N, "n": int(N) ** 3}


# ---------------------------------------------------------------------------
# Named workloads (sizes and recipes of the paper-shaped inputs)
# ---------------------------------------------------------------------------

def dense_haar_500x400(seed: int = 1) -> np.ndarray:
    """Dense FP64 500 x 400, Haar factors, sigma_i = 0.8**i (rank 40 target)."""
    return dense_haar_decay(500, 400, 0.8, seed)


def dense_householder_inverse_square(n: int = 32768, seed: int = 3) -> LowRankPlusDiag:
    """Dense n x n, Householder-product factors (64 reflectors each side),
    sigma_i = (1 + i)**-2 (rank 256 target)."""
    sigma = (1.0 + np.arange(n, dtype=np.float64)) ** -2
    return householder_decay(n, n, sigma, seed, 64)


def cauchy_spirals_square(n: int = 20000, seed: int = 2):
    """Complex Cauchy on spirals + cluster, n = m = 20000 (rank 100 target)."""
    return cauchy_spirals(n, n, seed)
