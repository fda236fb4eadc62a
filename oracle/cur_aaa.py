"""Oracle for CUR-AAA (Sec. 5.3, Algorithm "CUR-AAA using RPLU"): TEST
INFRASTRUCTURE ONLY (imported by tests/; never by the library).

Steps, in the paper's order:
  1. split the m samples Z at random into X (ceil(m/2)) and Y (floor(m/2));
  2. form the generators G, B of the Loewner matrix L~_ij = (f(x_i) - f(y_j)) /
     (x_i - y_j) (Eq. loewner-generators, alpha = sqrt(max(max|f^x|, max|f^y|)));
  3. run Algorithm 3 (rejection-sampled RPLU, or the approximate C2PLU) until
     max(u) <= eps^2 max(u at step 0);
  4. for each of the two pivot sets (rows I -> points X[I], columns J ->
     points Y[J]) take them as support points T and compute the barycentric
     weights as the right singular vector of the smallest singular value of
     the Loewner matrix L_ij = (f(z_i) - f(t_j)) / (z_i - t_j) over the
     samples z_i not in T (Eq. Laaa);
  5. evaluate both rational functions (Eq. aaa-barycentric) on all of Z and
     return the one with the smaller maximum error.

The random split (step 1) is this build's reading of "partition randomly":
sample i goes to X when pi(i) < ceil(m/2), pi a keyed permutation of
[0, m): a 4-round Feistel network on 2h-bit words (2^(2h) >= m) whose round
function is the SplitMix64 output function (Steele, Lea & Flood 2014) of
seed XOR K_r XOR R, restricted to [0, m) by cycle walking (Black & Rogaway,
"Ciphers with arbitrary finite domains", 2002).  X and Y keep the samples'
index order.  Step 4 uses numpy's SVD (LAPACK), step 3 the C oracle.
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
PART_KEY = 0x632BE59BD9B4E019  # the split's stream: seed XOR this constant


def _mix64(z: int) -> int:
    """SplitMix64 output function (the finaliser applied to the state)."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def half_bits(m: int) -> int:
    """h with 2^(2h) >= m (at least 1)."""
    h = 1
    while (1 << (2 * h)) < m:
        h += 1
    return h


def feistel_index(i: int, m: int, seed: int) -> int:
    """pi(i): the keyed permutation of [0, m) described in the module header."""
    h = half_bits(m)
    mask = (1 << h) - 1
    key = (seed ^ PART_KEY) & M64
    x = i
    while True:
        left, right = x >> h, x & mask
        for r in range(4):
            f = _mix64(key ^ ((GAMMA * (r + 1)) & M64) ^ right) & mask
            left, right = right, left ^ f
        x = (left << h) | right
        if x < m:
            return x


def random_halves(m: int, seed: int):
    """Indices of X (pi(i) < ceil(m/2)) and of Y, each in increasing order."""
    half = (m + 1) // 2
    inx = np.array([feistel_index(i, m, seed) < half for i in range(m)], dtype=bool)
    idx = np.arange(m)
    return idx[inx], idx[~inx]


def loewner_generators(fx, fy):
    """G (n x 2), B (2 x m) of L~ (Eq. loewner-generators)."""
    fx = np.asarray(fx, dtype=np.complex128)
    fy = np.asarray(fy, dtype=np.complex128)
    alpha = np.sqrt(max(np.abs(fx).max(), np.abs(fy).max()))
    G = np.stack([fx / alpha, np.full(len(fx), alpha, dtype=np.complex128)], axis=1)
    B = np.stack([np.full(len(fy), alpha, dtype=np.complex128), -fy / alpha], axis=0)
    return G, B


def aaa_weights(z, f, support):
    """Barycentric weights for the support points z[support] (step 4): the right
    singular vector of the smallest singular value of the Loewner matrix over
    the other samples.  Returns (w, sigma_min)."""
    z = np.asarray(z, dtype=np.complex128)
    f = np.asarray(f, dtype=np.complex128)
    mask = np.ones(len(z), dtype=bool)
    mask[support] = False
    zi, fi = z[mask], f[mask]
    t, ft = z[support], f[support]
    Lw = (fi[:, None] - ft[None, :]) / (zi[:, None] - t[None, :])
    _, s, vh = np.linalg.svd(Lw, full_matrices=False)
    return np.conj(vh[-1]), s[-1]


def barycentric(zq, t, ft, w):
    """r(zq) of Eq. aaa-barycentric; at a support point the sample value."""
    zq = np.asarray(zq, dtype=np.complex128)
    r = np.empty(len(zq), dtype=np.complex128)
    for a, zz in enumerate(zq):
        d = zz - t
        hit = np.nonzero(d == 0)[0]
        if len(hit):
            r[a] = ft[hit[0]]
        else:
            c = w / d
            r[a] = np.sum(c * ft) / np.sum(c)
    return r


def cur_aaa(z, f, eps: float, seed: int = 0, mode: str = "random", nu: float = 5.0, leaf: int = 32,
            k_max: int | None = None) -> dict:
    """CUR-AAA (Sec. 5.3).  Returns the chosen support (indices into z), its
    weights, both maximum errors over Z, which pivot set won ("I": rows /
    X side, "J": columns / Y side) and the factorization's pivots."""
    import oracle

    z = np.asarray(z, dtype=np.complex128)
    f = np.asarray(f, dtype=np.complex128)
    m = len(z)
    X, Y = random_halves(m, seed)
    G, B = loewner_generators(f[X], f[Y])
    k = min(len(X), len(Y)) if k_max is None else min(k_max, len(X), len(Y))
    o = oracle.rplu_cauchy_like_bh(z[X], z[Y], G, B, k, seed=seed, nu=nu, leaf=leaf, tol=eps, mode=mode, stop="max")
    out = {"X": X, "Y": Y, "I": o["I"], "J": o["J"], "k": o["k_done"], "factorization": o}
    cand = {}
    for name, sup in (("I", X[o["I"]]), ("J", Y[o["J"]])):
        w, smin = aaa_weights(z, f, sup)
        r = barycentric(z, z[sup], f[sup], w)
        cand[name] = (sup, w, float(np.max(np.abs(f - r))), smin)
    out["err_I"], out["err_J"] = cand["I"][2], cand["J"][2]
    out["sigma_min_I"], out["sigma_min_J"] = cand["I"][3], cand["J"][3]
    win = "I" if cand["I"][2] < cand["J"][2] else "J"
    out["which"] = win
    out["support"], out["weights"] = cand[win][0], cand[win][1]
    return out
