"""GPU parity of CUR-AAA (Sec. 5.3; rplu_cur_aaa and rplu_barycentric through
the C-ABI) against the numpy oracle (oracle/cur_aaa.py): the same split, the
same support points (pivots of Algorithm 3, up to near-ties), the same choice
between the row and column candidates, weights that give the same rational
function (the weights are a singular vector, unique up to a unit factor),
and accurate approximants at a larger size."""
import numpy as np
import pytest

from parity import to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)
from oracle import cur_aaa as CA  # noqa: E402


def _disk(m, seed):
    rng = np.random.default_rng(seed)
    return np.sqrt(rng.random(m)) * np.exp(2j * np.pi * rng.random(m))


FUNCS = {
    "tan": lambda z: np.tan(z),
    "exp_pole": lambda z: np.exp(z) + 1.0 / (1.3 - z),
    "tan4": lambda z: np.tan(2 * z ** 4),
}


@pytest.mark.parametrize("name", list(FUNCS))
@pytest.mark.parametrize("mode", ["random", "c2"])
def test_parity_with_the_oracle(name, mode):
    z = _disk(1500, 3)
    f = FUNCS[name](z)
    o = CA.cur_aaa(z, f, eps=1e-10, seed=7, mode=mode, leaf=16)
    zd, fd = torch.from_numpy(z).cuda(), torch.from_numpy(f).cuda()
    g = rp.rplu_cur_aaa(zd, fd, eps=1e-10, seed=7, pivot=mode, leaf=16)
    fo = o["factorization"]
    # the same pivots up to the first step where the oracle saw a near-tie in a draw
    T = np.maximum(np.asarray(fo["T"][:-1]), 1e-300)
    if mode == "random":
        ties = (np.minimum(fo["row_margin"], fo["col_margin"]) < 1e-12 * np.sqrt(T[0] / T)) | \
               (fo["acc_margin"] < 1e-12 * T[0] / T)
    else:
        ties = (fo["row_margin"] < 1e-12 * T[0] / T) | (fo["col_margin"] < 1e-12 * np.sqrt(T[0] / T))
    tie_step = int(np.nonzero(ties)[0][0]) if ties.any() else fo["k_done"]
    gsup = to_np(g.support)
    osup_I, osup_J = o["X"][fo["I"]], o["Y"][fo["J"]]
    scale = np.abs(f).max()
    # the GPU's own result is a good approximant in every case
    assert min(g.err_I, g.err_J) <= 1e-7 * scale
    zh = _disk(2000, 77) * 0.999
    rg = to_np(g(torch.from_numpy(zh).cuda(), zd, fd))
    assert np.max(np.abs(rg - FUNCS[name](zh))) <= 1e-6 * scale
    agreed = g.k == o["k"] and np.array_equal(gsup, osup_I if g.which == "I" else osup_J)
    if not agreed:
        # pivots may differ only after a near-tie step
        assert tie_step < min(g.k, o["k"]), (g.k, o["k"], tie_step)
        return
    assert g.which == o["which"]
    assert np.array_equal(gsup, o["support"])
    assert g.err_I == pytest.approx(o["err_I"], rel=0.5, abs=1e-12 * scale)
    assert g.err_J == pytest.approx(o["err_J"], rel=0.5, abs=1e-12 * scale)
    # the same rational function: weights agree up to a unit factor, values agree
    wg, wo = to_np(g.weights), o["weights"]
    assert abs(abs(np.vdot(wo, wg)) - 1.0) < 1e-6
    ro = CA.barycentric(zh, z[o["support"]], f[o["support"]], o["weights"])
    assert np.max(np.abs(rg - ro)) <= max(10 * min(o["err_I"], o["err_J"]), 1e-10 * scale)


def test_barycentric_matches_the_formula():
    rng = np.random.default_rng(1)
    t = rng.standard_normal(17) + 1j * rng.standard_normal(17)
    ft = rng.standard_normal(17) + 1j * rng.standard_normal(17)
    w = rng.standard_normal(17) + 1j * rng.standard_normal(17)
    zq = np.concatenate([rng.standard_normal(300) + 1j * rng.standard_normal(300), t[[0, 5, 16]]])
    z = np.concatenate([t, zq])  # support indices 0..16 into z
    r = to_np(rp.rplu_barycentric(z, np.concatenate([ft, np.zeros(len(zq))]), np.arange(17), w, zq))
    ro = CA.barycentric(zq, t, ft, w)
    np.testing.assert_allclose(r, ro, rtol=1e-12, atol=0)
    assert np.array_equal(r[-3:], ft[[0, 5, 16]])


def test_accuracy_at_scale():
    """20 000 samples on the unit disk, f = tan(2 z^4): the approximant is
    accurate on the samples and on points it never saw."""
    z = _disk(20000, 11)
    f = FUNCS["tan4"](z)
    zd, fd = torch.from_numpy(z).cuda(), torch.from_numpy(f).cuda()
    g = rp.rplu_cur_aaa(zd, fd, eps=1e-10, seed=3)
    scale = np.abs(f).max()
    assert 10 <= g.k <= 80
    assert min(g.err_I, g.err_J) <= 1e-7 * scale
    zh = _disk(20000, 12) * 0.999
    r = to_np(g(torch.from_numpy(zh).cuda(), zd, fd))
    assert np.max(np.abs(r - FUNCS["tan4"](zh))) <= 1e-6 * scale


def test_invalid_arguments():
    z = _disk(100, 2)
    with pytest.raises(rp.RPLUError):
        rp.rplu_cur_aaa(z, np.ones(100), eps=1e-8)  # constant f: zero Loewner matrix
    with pytest.raises(rp.RPLUError):
        rp.rplu_cur_aaa(z, np.tan(z), eps=0.0)
    with pytest.raises(rp.RPLUError):
        rp.rplu_cur_aaa(z[:1], np.tan(z[:1]), eps=1e-8)
