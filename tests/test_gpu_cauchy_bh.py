"""GPU parity of Algorithm 3's bound-based row draw (rplu_cauchy_like with
bound_nu, and rplu_bh_bounds) through the C-ABI:

* the bounds of App. C equal the oracle's (its own trees and lists, pinned
  against brute force) and are certified against brute-force row norms;
* the factorization equals the oracle's step for step (proposals, rejections,
  the exact fallback after 64 rejections, columns, factors, sum(u) history),
  up to the first step whose draws or acceptance decisions the oracle reports
  as near-ties;
* with nu = 1 the bounds are the exact norms, every first proposal is accepted
  and the result equals the exact-norm generator form;
* at 4000^2 the reported final residual is the explicit one."""
import numpy as np
import pytest

import workloads as W
from parity import GPU_TOL, TIE, assert_factors, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)

NDT = {"f32": np.float32, "f64": np.float64, "c64": np.complex64, "c128": np.complex128}


def _case(kind, seed, n=300, m=260):
    rng = np.random.default_rng(seed)
    if kind == "intervals":  # real, p = 2
        x, y = rng.uniform(-1, 1, n), rng.uniform(2.5, 4, m)
        G, B = rng.standard_normal((n, 2)), rng.standard_normal((2, m))
    elif kind == "clouds":  # overlapping complex clouds, p = 3
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        y = 0.5 + rng.standard_normal(m) + 1j * rng.standard_normal(m)
        G = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
        B = rng.standard_normal((3, m)) + 1j * rng.standard_normal((3, m))
    elif kind == "spirals":  # plain Cauchy, p = 1
        x, y = W.cauchy_spirals(n, m, seed=seed)
        G, B = np.ones((n, 1), complex), np.ones((1, m), complex)
    elif kind == "close":  # nearly touching intervals, p = 1
        x, y = rng.uniform(0, 1, n) + 0j, rng.uniform(1.0005, 2, m) + 0j
        G, B = np.ones((n, 1), complex), np.ones((1, m), complex)
    else:  # Loewner matrix on the unit disk (Sec. 5.2), p = 2
        x = np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
        y = np.sqrt(rng.random(m)) * np.exp(2j * np.pi * rng.random(m))
        f = lambda z: np.tan(2 * z ** 4)  # noqa: E731
        G, B = W.loewner_generators(x, y, f(x), f(y))
    return x, y, G, B


def _cast(a, dt):
    a = np.asarray(a)
    if dt in ("f32", "f64"):
        a = a.real
    return np.ascontiguousarray(a.astype(NDT[dt]))


def _dev(a, dt):
    return torch.from_numpy(_cast(a, dt)).cuda()


def _oracle_in(a, dt):
    return _cast(a, dt).astype(np.complex128)


def _bh_prefix(g, o, tie):
    """Agreed pivot prefix and the first step flagged as a near-tie: any row
    proposal, the column draw, or any acceptance decision of the step within
    the window (residual-scaled for the draws; for the acceptance the bounds
    carry absolute rounding of the size of the initial generators, so the
    window grows as T_0 / T_t)."""
    gI, gJ = to_np(g.I), to_np(g.J)
    k = min(len(gI), len(o["I"]))
    T = np.maximum(np.asarray(o["T"][:k]), 1e-300)
    thr = tie * np.sqrt(T[0] / T)
    bad = (np.minimum(o["row_margin"][:k], o["col_margin"][:k]) < thr) | (o["acc_margin"][:k] < tie * T[0] / T)
    tie_step = int(np.nonzero(bad)[0][0]) if bad.any() else k
    same = 0
    while same < k and gI[same] == o["I"][same] and gJ[same] == o["J"][same]:
        same += 1
    return same, tie_step


@pytest.mark.parametrize("kind", ["intervals", "clouds", "spirals", "close", "disk"])
@pytest.mark.parametrize("nu,leaf", [(5.0, 32), (2.0, 8), (5.0, 4), (1.0, 16)])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_bounds_equal_the_oracle_and_are_certified(orc, kind, nu, leaf, dt):
    if kind == "intervals":
        dt = {"c128": "f64", "c64": "f32"}[dt]
    x, y, G, B = _case(kind, 2)
    u = to_np(rp.rplu_bh_bounds(_dev(x, dt), _dev(y, dt), _dev(G, dt), _dev(B, dt), nu=nu, leaf=leaf))
    xo, yo, Go, Bo = (_oracle_in(v, dt) for v in (x, y, G, B))
    uo = orc.bh_bounds(xo, yo, Go, Bo, nu=nu, leaf=leaf)
    rtol = 1e-11 if dt in ("f64", "c128") else 2e-5
    np.testing.assert_allclose(u, uo, rtol=rtol, atol=0)
    rho = (np.abs(W.cauchy_like_dense(xo, yo, Go, Bo)) ** 2).sum(axis=1)
    assert np.all(u >= rho * (1 - rtol)) and np.all(u <= nu * rho * (1 + rtol))


def test_bounds_from_host_arrays_equal_device(orc):
    x, y, G, B = _case("disk", 5)
    ud = to_np(rp.rplu_bh_bounds(_dev(x, "c128"), _dev(y, "c128"), _dev(G, "c128"), _dev(B, "c128")))
    uh = rp.rplu_bh_bounds(x.astype(np.complex128), y.astype(np.complex128), G.astype(np.complex128),
                           B.astype(np.complex128))
    assert np.array_equal(ud, uh)


@pytest.mark.parametrize("kind", ["intervals", "clouds", "spirals", "disk"])
@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_parity_with_the_rejection_oracle(orc, kind, seed, dt):
    if kind == "intervals":
        dt = {"c128": "f64", "c64": "f32"}[dt]
    x, y, G, B = _case(kind, seed)
    k, nu, leaf = 25, 5.0, 16
    g = rp.rplu_cauchy_like(_dev(x, dt), _dev(y, dt), _dev(G, dt), _dev(B, dt), k, seed=seed + 7, bound_nu=nu,
                            bound_leaf=leaf)
    o = orc.rplu_cauchy_like_bh(*(_oracle_in(v, dt) for v in (x, y, G, B)), k, seed=seed + 7, nu=nu, leaf=leaf)
    same, tie_step = _bh_prefix(g, o, TIE[dt])
    assert same >= min(tie_step, o["k_done"]), (same, tie_step, to_np(g.I)[:same + 1], o["I"][:same + 1])
    if dt in ("f64", "c128"):
        assert same >= min(3, o["k_done"])
    upto = min(same, tie_step)
    assert np.array_equal(g.attempts[:upto], o["attempts"][:upto])
    assert_factors(g, o, upto, GPU_TOL[dt])
    if dt in ("f64", "c128"):
        np.testing.assert_allclose(g.T[:upto], o["T"][:upto], rtol=1e-9, atol=1e-13 * o["T"][0])
        if upto == o["k_done"] == g.k_done:
            np.testing.assert_allclose(g.T[-1], o["T"][-1], rtol=1e-9, atol=1e-12 * o["T"][0])


@pytest.mark.parametrize("kind", ["close", "disk"])
def test_exact_fallback_after_64_rejections(orc, kind):
    """nu = 1e6 with 4-point leaves: bounds loose enough that some steps reject
    all 64 proposals and take the exact-norm draw; the GPU takes it at the same
    steps with the same result."""
    x, y, G, B = _case(kind, 0, n=200, m=200)
    k = 30
    g = rp.rplu_cauchy_like(_dev(x, "c128"), _dev(y, "c128"), _dev(G, "c128"), _dev(B, "c128"), k, seed=1,
                            bound_nu=1e6, bound_leaf=4)
    o = orc.rplu_cauchy_like_bh(x, y, G, B, k, seed=1, nu=1e6, leaf=4)
    assert (o["attempts"] == 65).any()
    same, tie_step = _bh_prefix(g, o, TIE["c128"])
    upto = min(same, tie_step)
    assert same >= min(tie_step, o["k_done"]) and (g.attempts[:upto] == 65).any()
    assert np.array_equal(g.attempts[:upto], o["attempts"][:upto])
    assert_factors(g, o, upto, GPU_TOL["c128"])


@pytest.mark.parametrize("kind", ["clouds", "disk"])
def test_nu_one_equals_the_exact_norm_form(kind):
    x, y, G, B = _case(kind, 4, n=400, m=350)
    args = [_dev(v, "c128") for v in (x, y, G, B)]
    e = rp.rplu_cauchy_like(*args, 40, seed=9)
    b = rp.rplu_cauchy_like(*args, 40, seed=9, bound_nu=1.0, bound_leaf=16)
    assert np.all(b.attempts == 1)
    assert np.array_equal(to_np(e.I), to_np(b.I)) and np.array_equal(to_np(e.J), to_np(b.J))
    np.testing.assert_allclose(to_np(b.U), to_np(e.U), rtol=0, atol=1e-12 * np.abs(to_np(e.U)).max())
    np.testing.assert_allclose(b.T[:-1], e.T[:-1], rtol=1e-10)


def test_reported_residual_and_acceptance_rate_at_scale():
    """Spiral Cauchy matrix, complex64, 4000^2, nu = 5: the final T_hist entry
    is the exact residual (checked explicitly), the mean number of proposals
    per step is at most nu, and the sum of the bounds stays within [1, nu] of
    the exact squared norm at the start."""
    x, y = W.cauchy_spirals(4000, 4000, seed=11)
    xd, yd = _dev(x, "c64"), _dev(y, "c64")
    G = torch.ones((4000, 1), dtype=torch.complex64, device="cuda")
    B = torch.ones((1, 4000), dtype=torch.complex64, device="cuda")
    g = rp.rplu_cauchy_like(xd, yd, G, B, 60, seed=5, bound_nu=5.0)
    e = rp.rplu_cauchy_like(xd, yd, G, B, 0, seed=5)
    A = 1.0 / (xd.to(torch.complex128)[:, None] - yd.to(torch.complex128)[None, :])
    R = A - g.L.to(torch.complex128) @ g.U.to(torch.complex128)
    explicit = float(torch.linalg.norm(R) / torch.linalg.norm(A))
    reported = float(np.sqrt(g.T[-1] / e.T[0]))
    assert abs(reported - explicit) <= 1e-3 * explicit + 1e-6
    assert g.attempts.mean() <= 5.0 and np.all(g.attempts <= 65)
    assert e.T[0] * (1 - 1e-5) <= g.T[0] <= 5.0 * e.T[0] * (1 + 1e-5)


def test_tolerance_stop_is_conservative():
    """The stop test compares sum(u) >= ||S||_F^2: when it fires, the exact
    residual is below the tolerance too."""
    for b, blk in enumerate(W.cauchy_interval_blocks(3, seed=4, size_lo=600, size_hi=900)):
        n, m = len(blk.x), len(blk.y)
        g = rp.rplu_cauchy_like(_dev(blk.x, "f64"), _dev(blk.y, "f64"), torch.ones((n, 1), dtype=torch.float64,
                                device="cuda"), torch.ones((1, m), dtype=torch.float64, device="cuda"),
                                min(n, m), seed=b, rel_tol=1e-8, bound_nu=5.0)
        assert g.k_done < min(n, m)
        A = W.cauchy_dense(blk.x, blk.y)
        err = np.linalg.norm(A - to_np(g.L) @ to_np(g.U)) / np.linalg.norm(A)
        assert err <= 1e-8 and np.sqrt(g.T[-1] / g.T[0]) <= 1e-8


def test_invalid_bound_arguments():
    x, y, G, B = (_dev(v, "c128") for v in _case("clouds", 1, n=50, m=40))
    with pytest.raises(rp.RPLUError):
        rp.rplu_cauchy_like(x, y, G, B, 5, bound_nu=0.5)
    with pytest.raises(rp.RPLUError):
        rp.rplu_cauchy_like(x, y, G, B, 5, bound_nu=5.0, pivot="given", given=([0, 1, 2, 3, 4], [0, 1, 2, 3, 4]))
    with pytest.raises(rp.RPLUError):
        rp.rplu_cauchy_like(x, y, G, B, 5, bound_nu=float("inf"))
    with pytest.raises(rp.RPLUError):
        rp.rplu_bh_bounds(x, y, G, B, nu=0.9)
    with pytest.raises(rp.RPLUError):
        rp.rplu_bh_bounds(x, y, G, B, leaf=0)


def test_plan_stats():
    """rplu_bh_plan_stats reports the plan the factorization uses: with nu = 1
    only pairs of single-point boxes (d_max = d_min) are aggregated, one pair
    each (no coincident points here), and every other pair is exact; with
    nu = 5 most pairs are aggregated."""
    x, y, G, B = _case("clouds", 3, n=500, m=400)
    s1 = rp.rplu_bh_plan_stats(_dev(x, "c128"), _dev(y, "c128"), nu=1.0, leaf=16)
    assert s1["exact_pairs"] + s1["aggregated_entries"] == 500 * 400
    assert s1["max_target_leaf"] <= 16 and s1["target_leaves"] >= 500 // 16
    s5 = rp.rplu_bh_plan_stats(x, y, nu=5.0, leaf=16)
    assert s5["aggregated_entries"] > 0 and s5["exact_pairs"] < 500 * 400 // 2
    assert s5["source_leaves"] < s5["source_nodes"]


@pytest.mark.parametrize("kind", ["intervals", "clouds", "spirals", "disk"])
def test_c2_with_bounds_matches_the_oracle(orc, kind):
    """The approximate C2PLU of Sec. 5.1 (row of the largest bound, largest
    entry of that row): pivots identical to the oracle's up to the first step
    whose arg-max gap lies within the rounding window of the bounds."""
    dt = "f64" if kind == "intervals" else "c128"
    x, y, G, B = _case(kind, 3)
    g = rp.rplu_cauchy_like(_dev(x, dt), _dev(y, dt), _dev(G, dt), _dev(B, dt), 25, pivot="c2", bound_nu=5.0,
                            bound_leaf=16)
    o = orc.rplu_cauchy_like_bh(*(_oracle_in(v, dt) for v in (x, y, G, B)), 25, nu=5.0, leaf=16, mode="c2")
    T = np.maximum(np.asarray(o["T"][:-1]), 1e-300)
    bad = (o["row_margin"] < 1e-12 * T[0] / T) | (o["col_margin"] < 1e-12 * np.sqrt(T[0] / T))
    tie_step = int(np.nonzero(bad)[0][0]) if bad.any() else o["k_done"]
    gI, gJ = to_np(g.I), to_np(g.J)
    same = 0
    while same < min(len(gI), o["k_done"]) and gI[same] == o["I"][same] and gJ[same] == o["J"][same]:
        same += 1
    assert same >= tie_step, (same, tie_step)
    upto = min(same, tie_step)
    assert np.array_equal(g.attempts[:upto], o["attempts"][:upto])
    assert_factors(g, o, upto, GPU_TOL[dt])


@pytest.mark.parametrize("mode", ["random", "c2"])
def test_max_stopping_rule_matches_the_oracle(orc, mode):
    """bound_stop="max" (the CUR-AAA rule of Sec. 5.3): the run stops at the
    same step as the oracle's."""
    x, y, G, B = _case("intervals", 8, n=400, m=350)
    args = [_dev(v, "f64") for v in (x, y, G, B)]
    g = rp.rplu_cauchy_like(*args, 200, seed=4, rel_tol=1e-7, bound_nu=5.0, bound_leaf=16, bound_stop="max",
                            pivot=mode)
    o = orc.rplu_cauchy_like_bh(*(_oracle_in(v, "f64") for v in (x, y, G, B)), 200, seed=4, nu=5.0, leaf=16,
                                tol=1e-7, mode=mode, stop="max")
    assert 0 < o["k_done"] < 200
    if mode == "random":
        same, tie_step = _bh_prefix(g, o, TIE["f64"])
    else:
        T = np.maximum(np.asarray(o["T"][:-1]), 1e-300)
        bad = (o["row_margin"] < 1e-12 * T[0] / T) | (o["col_margin"] < 1e-12 * np.sqrt(T[0] / T))
        tie_step = int(np.nonzero(bad)[0][0]) if bad.any() else o["k_done"]
        gI, gJ = to_np(g.I), to_np(g.J)
        same = 0
        while same < min(len(gI), o["k_done"]) and gI[same] == o["I"][same] and gJ[same] == o["J"][same]:
            same += 1
    assert same >= min(tie_step, o["k_done"])
    if tie_step >= o["k_done"]:  # the same pivots throughout: the same stopping step
        assert g.k_done == o["k_done"]
