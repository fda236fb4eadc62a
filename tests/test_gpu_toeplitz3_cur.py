"""GPU parity of RPLU in CUR form on the multi-level Toeplitz matrix of
Sec. 4.2 (rplu_toeplitz3_cur through the C-ABI) against the CUR-form oracle
(oracle/cur_form.py, KroneckerToeplitz, with its QR core: the library keeps
its core as a double-double block-inverse update, both accurate to about
eps cond) on the same draws: the same pivots up to near-ties, the same
row-norm totals, a core equal to A(I,J)^{-1} of the run's own pivots to
eps cond; C2PLU choices that are maxima of their own residual; forced pivots;
the tolerance stop.
"""
import numpy as np
import pytest

from oracle import cur_form as CF
from parity import to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402


def _first_tie(o, rel=1e-11):
    """First step whose draw the oracle saw within the row-norm estimate's
    rounding (eps T_0, relative to the step's total) of a CDF boundary."""
    T = o["T"]
    kd = o["k_done"]
    thr = rel * T[0] / np.maximum(T[:kd], 1e-300)
    m = np.minimum(o["row_margin"], o["col_margin"])
    bad = np.nonzero(m < thr)[0]
    return int(bad[0]) if len(bad) else kd


def _core_bound(A_IJ, kd):
    """||core A(I,J) - I|| for a core accurate to about eps cond(A(I,J)) (a QR
    of A(I,J), or the double-double update), the FP64 check's own rounding
    included; the FP64 block-inverse update would need eps cond^2."""
    cond = np.linalg.cond(A_IJ) if kd else 1.0
    return max(100 * kd * 1.1e-16 * cond, 1e-12 * max(kd, 1))


# (N, length, k) with A(I,J) still well enough conditioned (cond <= ~1e5) that the
# core bound eps cond^2 means something; length 30 and 60 give the paper's
# spacing h = 2.5 (fast decay), length 320 a coarse grid (slow decay)
@pytest.mark.parametrize("N,length,k", [(5, 320.0, 20), (16, 320.0, 30), (12, 30.0, 8), (24, 60.0, 12)])
def test_parity_with_the_oracle(N, length, k):
    op = CF.KroneckerToeplitz(N, length=length)
    o = CF.rplu_cur(op, k, seed=21, core="qr")
    g = rp.rplu_toeplitz3_cur(N, k, seed=21, length=length)
    upto = min(_first_tie(o), g.k_done)
    live = np.nonzero(o["T"][:-1] <= 1e-9 * o["T"][0])[0]
    if len(live):
        upto = min(upto, int(live[0]))
    assert upto >= 3
    I, J = to_np(g.I), to_np(g.J)
    assert np.array_equal(I[:upto], o["I"][:upto]) and np.array_equal(J[:upto], o["J"][:upto])
    np.testing.assert_allclose(g.T[:upto + 1], o["T"][:upto + 1], rtol=1e-9, atol=1e-12 * o["T"][0])
    # the core is A(I,J)^{-1} of the run's own pivots (its definition)
    kd = g.k_done
    W = op.entries(I, J).real
    C = to_np(g.core)
    assert np.linalg.norm(C @ W - np.eye(kd)) <= _core_bound(W, kd)


def test_c2_choices_are_maxima_of_the_residual():
    """The grid's mirror symmetry makes C2PLU's maxima tie; every GPU choice
    must be a maximum of its own exact residual."""
    N = 5
    op = CF.KroneckerToeplitz(N)
    A = op.dense().real
    g = rp.rplu_toeplitz3_cur(N, 15, pivot="c2")
    I, J = to_np(g.I), to_np(g.J)
    for t in range(g.k_done):
        S = A - (A[:, J[:t]] @ np.linalg.solve(A[np.ix_(I[:t], J[:t])], A[I[:t], :]) if t else 0.0)
        if np.sum(S ** 2) <= 1e-10 * np.sum(A ** 2):
            break
        w = np.sum(S ** 2, axis=1)
        assert w[I[t]] >= (1 - 1e-9) * w.max(), t
        r = S[I[t]] ** 2
        assert r[J[t]] >= (1 - 1e-9) * r.max(), t


def test_given_pivots_and_tolerance_stop():
    N = 8
    op = CF.KroneckerToeplitz(N, length=20.0)
    o = CF.rplu_cur(op, 6, seed=3, core="qr")
    g = rp.rplu_toeplitz3_cur(N, 6, length=20.0, pivot="given", given=(o["I"], o["J"]))
    assert np.array_equal(to_np(g.I), o["I"]) and np.array_equal(to_np(g.J), o["J"])
    W = op.entries(o["I"], o["J"]).real
    assert np.linalg.norm(to_np(g.core) @ W - np.eye(6)) <= _core_bound(W, 6)
    np.testing.assert_allclose(to_np(g.core), o["core"].real, rtol=0, atol=_core_bound(W, 6) * np.abs(o["core"]).max())
    t = rp.rplu_toeplitz3_cur(N, 200, seed=3, length=20.0, rel_tol=1e-5)
    assert t.k_done < 200 and t.T[-1] <= 1e-10 * t.T[0] and np.all(t.T[:-1] > 1e-10 * t.T[0])


def test_host_outputs_and_invalid_arguments():
    g = rp.rplu_toeplitz3_cur(4, 6, seed=1, device="host")
    assert isinstance(g.I, np.ndarray) and g.k_done == 6 and g.core.shape == (6, 6)
    with pytest.raises(rp.RPLUError):
        rp.rplu_toeplitz3_cur(4, 65)  # k > N^3
