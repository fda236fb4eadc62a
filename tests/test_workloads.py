"""The synthetic input generators produce what their recipes state."""
import numpy as np
import pytest

import workloads as W


def test_householder_wy_equals_explicit_product():
    rng = np.random.default_rng(0)
    v = rng.standard_normal((30, 6))
    V, T = W.householder_wy(v)
    Q = np.eye(30)
    for j in range(6):
        vj = v[:, j:j + 1]
        Q = Q @ (np.eye(30) - 2.0 * (vj @ vj.T) / (vj.T @ vj))
    assert np.allclose(np.eye(30) - V @ T @ V.T, Q, atol=1e-13)


@pytest.mark.parametrize("n,m", [(60, 60), (70, 50), (40, 55)])
def test_householder_decay_spectrum_and_entries(n, m):
    r = min(n, m)
    sigma = (1.0 + np.arange(r)) ** -2
    F = W.householder_decay(n, m, sigma, seed=4, n_reflectors=8)
    A = F.dense()
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(np.sort(s)[::-1], np.sort(sigma)[::-1], rtol=1e-10, atol=1e-14)
    rng = np.random.default_rng(1)
    p = rng.integers(0, n, 200)
    q = rng.integers(0, m, 200)
    q[:20] = p[:20] % m
    assert np.allclose(F.entries(p, q), A[p, q], atol=1e-14)
    assert np.allclose(F.rows(5, 17), A[5:17], atol=1e-14)


def test_householder_decay_matches_explicit_construction():
    n, m, k = 25, 20, 5
    sigma = 0.7 ** np.arange(20)
    F = W.householder_decay(n, m, sigma, seed=9, n_reflectors=k)
    rng = np.random.default_rng(9)
    v1 = rng.standard_normal((n, k))
    v2 = rng.standard_normal((m, k))

    def prod(v):
        Q = np.eye(v.shape[0])
        for j in range(v.shape[1]):
            vj = v[:, j:j + 1]
            Q = Q @ (np.eye(v.shape[0]) - 2.0 * (vj @ vj.T) / (vj.T @ vj))
        return Q

    D = np.zeros((n, m))
    D[np.arange(20), np.arange(20)] = sigma
    assert np.allclose(F.dense(), prod(v1) @ D @ prod(v2).T, atol=1e-13)


def test_haar_decay_spectrum():
    A = W.dense_haar_500x400()
    assert A.shape == (500, 400) and A.flags["C_CONTIGUOUS"]
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, 0.8 ** np.arange(400), rtol=1e-9, atol=1e-14)


def test_spiral_points_recipe():
    x, y = W.cauchy_spirals(1000, 800, seed=2)
    assert x.shape == (1000,) and y.shape == (800,)
    r = np.abs(x)
    assert np.sum(r < 0.25) >= 200  # the 20% cluster (plus inner spiral turns)
    assert r.max() <= 2.0 + 1e-12
    assert np.allclose(np.mean(y), 3.0, atol=0.2)
    assert np.min(np.abs(x[:, None] - y[None, :])) > 0


def test_interval_blocks_recipe():
    blocks = W.cauchy_interval_blocks(50, seed=1)
    for b in blocks:
        assert 64 <= len(b.x) <= 1024 and 64 <= len(b.y) <= 1024
        cx, cy = np.mean(b.x), np.mean(b.y)
        assert 1.0 <= abs(cx - cy) <= 8.0
        assert np.max(b.x) - np.min(b.x) <= 2.0 and np.max(b.y) - np.min(b.y) <= 2.0


def test_determinism():
    assert np.array_equal(W.cauchy_spirals(50, 50, 7)[0], W.cauchy_spirals(50, 50, 7)[0])
    assert W.derive_seed(1, 2) == W.derive_seed(1, 2) != W.derive_seed(2, 1)


def test_chung_lu_graph_is_a_power_law_adjacency():
    S = W.chung_lu_graph(20000, avg_degree=6.0, exponent=2.2, seed=3)
    assert S.shape == (20000, 20000)
    assert (S != S.T).nnz == 0 and S.diagonal().sum() == 0 and set(np.unique(S.data)) == {1.0}
    deg = np.asarray(S.sum(axis=1)).ravel()
    assert 4.0 < deg.mean() < 6.5           # repeated edges are dropped: a little below 6
    assert deg.max() > 50 * deg.mean()      # hubs: a heavy tail
    assert np.mean(deg <= 2) > 0.3          # most vertices have few edges
    # the same seed gives the same graph, another seed another one
    assert (S != W.chung_lu_graph(20000, 6.0, 2.2, seed=3)).nnz == 0
    assert (S != W.chung_lu_graph(20000, 6.0, 2.2, seed=4)).nnz > 0


def test_toeplitz_kernel_grid_parameters():
    g = W.toeplitz_kernel_grid(128)
    assert g["n"] == 128 ** 3 and g["h"] == 2.5 and g["delta"] == 50.0 and g["sigma"] == 80.0


def test_disk_blocks_recipe():
    bl = W.cauchy_disk_blocks(200, seed=5, size_lo=20, size_hi=60)
    for b in bl:
        assert np.iscomplexobj(b.x) and np.iscomplexobj(b.y)
        assert 20 <= len(b.x) <= 60 and 20 <= len(b.y) <= 60
        cx, cy = b.x.mean(), b.y.mean()
        # every point within its unit disk; the disks' centres 3 to 6 apart, so they never meet
        assert np.abs(b.x[:, None] - b.y[None, :]).min() >= 1.0 - 1e-12
        assert np.max(np.abs(b.x - cx)) <= 2.0 and np.max(np.abs(b.y - cy)) <= 2.0
