"""Pins of the CUR-AAA oracle (Sec. 5.3, oracle/cur_aaa.py).

* The random split is a split: the keyed Feistel map is a bijection of
  [0, m) for every m tried, X has ceil(m/2) samples, X and Y partition Z.
* The whole pipeline (generators, Algorithm 3 with the max stopping rule,
  weights, barycentric evaluation) yields rational approximants that match
  analytic functions on the unit disk to near the tolerance, on the samples
  and on points it never saw, for both pivot rules; a planted mistake in the
  generators or in the weights ruins that.
* The weights solve the linearisation: ||L w|| is the smallest singular value
  of the Loewner matrix, and r interpolates f at the support points.
"""
import numpy as np
import pytest

from oracle import cur_aaa as CA


@pytest.mark.parametrize("m", [1, 2, 3, 5, 16, 17, 100, 1000, 4097])
def test_feistel_split_is_a_bijection_and_balanced(m):
    seed = 12345 + m
    img = [CA.feistel_index(i, m, seed) for i in range(m)]
    assert sorted(img) == list(range(m))
    X, Y = CA.random_halves(m, seed)
    assert len(X) == (m + 1) // 2 and len(Y) == m // 2
    assert np.array_equal(np.sort(np.concatenate([X, Y])), np.arange(m))
    if m >= 100:  # a shuffle, not a prefix
        assert 0.25 < np.mean(X < m // 2) < 0.75


def test_different_seeds_give_different_splits():
    a, _ = CA.random_halves(500, 1)
    b, _ = CA.random_halves(500, 2)
    assert not np.array_equal(a, b)


def _disk(m, seed):
    rng = np.random.default_rng(seed)
    return np.sqrt(rng.random(m)) * np.exp(2j * np.pi * rng.random(m))


FUNCS = {
    "tan": lambda z: np.tan(z),                       # poles at +-pi/2, outside the disk
    "exp_pole": lambda z: np.exp(z) + 1.0 / (1.3 - z),
    "log": lambda z: np.log(2.0 - z),                 # branch point at 2
}


@pytest.mark.parametrize("name", list(FUNCS))
@pytest.mark.parametrize("mode", ["random", "c2"])
def test_approximants_are_accurate(name, mode):
    z = _disk(1500, 3)
    f = FUNCS[name](z)
    out = CA.cur_aaa(z, f, eps=1e-10, seed=7, mode=mode, leaf=16)
    k = out["k"]
    assert 3 <= k <= 60
    err = min(out["err_I"], out["err_J"])
    scale = np.abs(f).max()
    assert err <= 1e-7 * scale, (out["err_I"], out["err_J"], k)
    assert out["which"] == ("I" if out["err_I"] < out["err_J"] else "J")
    # points the fit never saw
    zh = _disk(3000, 99) * 0.999
    t = z[out["support"]]
    r = CA.barycentric(zh, t, f[out["support"]], out["weights"])
    assert np.max(np.abs(r - FUNCS[name](zh))) <= 1e-6 * scale


def test_weights_solve_the_linearisation():
    z = _disk(800, 5)
    f = FUNCS["exp_pole"](z)
    out = CA.cur_aaa(z, f, eps=1e-9, seed=2, leaf=16)
    sup, w = out["support"], out["weights"]
    mask = np.ones(len(z), bool)
    mask[sup] = False
    L = (f[mask][:, None] - f[sup][None, :]) / (z[mask][:, None] - z[sup][None, :])
    smin = np.linalg.svd(L, compute_uv=False)[-1]
    assert abs(np.linalg.norm(w) - 1.0) < 1e-12
    assert np.linalg.norm(L @ w) == pytest.approx(smin, rel=1e-6, abs=1e-14 * np.linalg.norm(L))
    r = CA.barycentric(z[sup], z[sup], f[sup], w)
    assert np.array_equal(r, f[sup])


def test_planted_mistakes_are_caught(monkeypatch):
    z = _disk(800, 6)
    f = FUNCS["tan"](z)
    good = CA.cur_aaa(z, f, eps=1e-10, seed=4, leaf=16)
    assert min(good["err_I"], good["err_J"]) <= 1e-7

    orig = CA.loewner_generators

    def wrong_sign(fx, fy):  # B = [alpha; +fy/alpha]: the matrix is no longer Loewner
        G, B = orig(fx, fy)
        return G, np.stack([B[0], -B[1]])

    monkeypatch.setattr(CA, "loewner_generators", wrong_sign)
    bad = CA.cur_aaa(z, f, eps=1e-10, seed=4, leaf=16)
    monkeypatch.setattr(CA, "loewner_generators", orig)
    assert bad["k"] > 2 * good["k"] or min(bad["err_I"], bad["err_J"]) > 1e-5

    orig_w = CA.aaa_weights

    def unconjugated(zz, ff, sup):  # weights without the conjugate of the singular vector
        w, s = orig_w(zz, ff, sup)
        return np.conj(w), s

    monkeypatch.setattr(CA, "aaa_weights", unconjugated)
    bad = CA.cur_aaa(z, f, eps=1e-10, seed=4, leaf=16)
    assert min(bad["err_I"], bad["err_J"]) > 1e-5


@pytest.mark.parametrize("name,f", [
    ("mobius", lambda z: (2 * z + 1) / (z - 1.7)),
    ("type33", lambda z: 1 + 1 / (z - 1.5) + 2 / (z + 2) - 1 / (z - 2j)),
])
def test_rational_functions_of_equal_degrees_are_recovered(name, f):
    """A rational function of type (d, d) is its own best approximant: with the
    support CUR-AAA picks (at least d + 1 points here) the barycentric form
    reproduces it to rounding on the samples and off them."""
    rng = np.random.default_rng(1)
    z = np.sqrt(rng.random(1200)) * np.exp(2j * np.pi * rng.random(1200))
    fz = f(z)
    out = CA.cur_aaa(z, fz, eps=1e-12, seed=3, leaf=16)
    scale = np.abs(fz).max()
    assert min(out["err_I"], out["err_J"]) <= 1e-12 * scale
    zh = _disk(500, 9) * 0.99
    r = CA.barycentric(zh, z[out["support"]], fz[out["support"]], out["weights"])
    assert np.max(np.abs(r - f(zh))) <= 1e-10 * scale
