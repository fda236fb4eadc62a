"""GPU parity of the CUR form of the matrix-free Cauchy factorization
(rplu_cauchy_cur through the C-ABI, Algorithm 2 as printed) against the
oracle's matrix-free LU form on the same draws: the same pivots (up to
near-ties and the row-norm estimate's resolution), A(:,J) core A(I,:) equal
to the oracle's L U, and the core equal to A(I,J)^{-1} formed from the
materialised matrix (its plain definition)."""
import numpy as np
import pytest

import workloads as W
from parity import assert_pivots, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_22344_gb300 as rp  # noqa: E402
from paper_2601_22344_gb300 import binding as _binding  # noqa: E402,F401  (raises if librplu.so is missing)

NDT = {"f32": np.float32, "f64": np.float64, "c64": np.complex64, "c128": np.complex128}


def _pts(dt, n, m, seed):
    if dt in ("c128", "c64"):
        x, y = W.cauchy_spirals(n, m, seed=seed)
    else:
        b = W.cauchy_interval_blocks(1, seed=seed, size_lo=max(n, m), size_hi=max(n, m))[0]
        x, y = b.x[:n], b.y[:m]
    return np.ascontiguousarray(x.astype(NDT[dt])), np.ascontiguousarray(y.astype(NDT[dt]))


def _window(o, floor):
    T = o["T"]
    below = np.nonzero(T[:-1] <= floor * T[0])[0]
    return int(below[0]) if len(below) else len(T) - 1


@pytest.mark.parametrize("dt", ["c128", "f64", "c64"])
def test_parity_with_the_oracle(orc, dt):
    xs, ys = _pts(dt, 600, 550, 3)
    # the separated real intervals decay to rounding within a few steps (A(I,J) then
    # has condition ~1/eps and no inverse carries information); the spirals decay slowly
    k = 4 if dt == "f64" else 30
    g = rp.rplu_cauchy_cur(torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda(), k, seed=4)
    o = orc.rplu_cauchy(xs, ys, k, seed=4)
    fp64 = dt in ("f64", "c128")
    win = _window(o, 1e-9 if fp64 else 1e-3)
    same = assert_pivots(g, o, 1e-12 if fp64 else 1e-5, min_steps=min(win, 3),
                         estimate_eps=1e-13 if fp64 else 1e-6)
    A = W.cauchy_dense(xs.astype(np.complex128), ys.astype(np.complex128))
    # the core is A(I,J)^{-1} for the run's own pivots (its definition), up to the
    # rounding of the block-inverse recurrence (of order eps cond^2: each update
    # multiplies through the previous inverse twice) and, for FP32 data, the
    # entries' own rounding (of order eps32 cond)
    I, J = to_np(g.I), to_np(g.J)
    kd = g.k_done
    C = to_np(g.core).astype(np.complex128)
    Wm = A[np.ix_(I, J)]
    cond = np.linalg.cond(Wm)
    bound = 10 * kd * (1.1e-16 * cond * cond + (0.0 if fp64 else 1.2e-7 * cond))
    assert np.linalg.norm(C @ Wm - np.eye(kd)) <= max(bound, 1e-13 * kd)
    # where the pivots agree throughout: CUR = the oracle's LU
    if same == o["k_done"] == kd:
        cur = A[:, J] @ C @ A[I, :]
        lu = o["L"] @ o["U"]
        assert np.linalg.norm(cur - lu) <= max(bound, 1e-12) * np.linalg.norm(A)


def test_given_and_c2_modes(orc):
    xs, ys = _pts("c128", 300, 280, 7)
    o = orc.rplu_cauchy(xs, ys, 20, mode="c2")
    g = rp.rplu_cauchy_cur(torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda(), 20, pivot="c2")
    assert_pivots(g, o, 1e-12, random_mode=False)
    gv = rp.rplu_cauchy_cur(xs, ys, 20, pivot="given", given=(o["I"], o["J"]))
    assert np.array_equal(to_np(gv.I), o["I"]) and np.array_equal(to_np(gv.J), o["J"])
    A = W.cauchy_dense(xs, ys)
    C = to_np(gv.core)
    np.testing.assert_allclose(C @ A[np.ix_(o["I"], o["J"])], np.eye(20), atol=1e-8)


def test_matches_the_lu_form_at_scale():
    """Spiral matrix, complex64, 4000^2, k = 60: the CUR form follows the GPU's
    LU form step for step while the FP32 row-norm estimates agree, and its
    approximation A(:,J) core A(I,:) is that of its own pivots with the exact
    inverse of A(I,J) (an FP64 solve on the materialised matrix)."""
    x, y = W.cauchy_spirals(4000, 4000, seed=11)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    yd = torch.from_numpy(y.astype(np.complex64)).cuda()
    lu = rp.rplu_cauchy(xd, yd, 60, seed=5)
    cu = rp.rplu_cauchy_cur(xd, yd, 60, seed=5)
    same = 0
    while same < 60 and to_np(lu.I)[same] == to_np(cu.I)[same] and to_np(lu.J)[same] == to_np(cu.J)[same]:
        same += 1
    assert same >= 10
    assert cu.core.dtype == torch.complex128
    A = 1.0 / (xd.to(torch.complex128)[:, None] - yd.to(torch.complex128)[None, :])
    I = torch.as_tensor(to_np(cu.I)).cuda()
    J = torch.as_tensor(to_np(cu.J)).cuda()
    nA = torch.linalg.norm(A)
    e_cur = float(torch.linalg.norm(A - A[:, J] @ cu.core @ A[I, :]) / nA)
    e_ref = float(torch.linalg.norm(A - A[:, J] @ torch.linalg.solve(A[I][:, J], A[I, :])) / nA)
    # the recurrence's rounding (eps cond^2) stays far below the error an FP32
    # core or FP32 entries would leave (0.90 against 0.29 at 20000^2, k = 100)
    assert abs(e_cur - e_ref) <= 5e-3 + 5e-2 * e_ref, (e_cur, e_ref)
