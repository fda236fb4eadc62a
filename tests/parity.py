"""Comparison rules shared by the GPU parity tests.

Pivots: identical to the oracle's for every step before the first step whose
row or column draw the oracle reports within `tie` (relative) of a CDF
boundary; a different summation order may legitimately pick the neighbour
there, and the sequences may differ afterwards.  With FP32 data the window is
the FP32 perturbation of the weights.

Factors: over the agreed prefix, the residual rows U(t,:) and the residual
columns C(:,t) = L(:,t) a_t (a_t = U(t, j_t), the pivot value) agree normwise:
||U_gpu - U_or||_F <= tol ||U_or||_F and ||C_gpu - C_or||_F <= tol ||C_or||_F.
L(:,t) = C(:,t) / a_t carries the same rounding amplified by 1/|a_t|, which for
late steps of a fast-decaying spectrum is far above 1/eps; comparing C keeps
the check independent of that conditioning while still fixing L (a_t is
checked through U).
"""
import os

import numpy as np

GPU_TOL = {"f64": 1e-12, "c128": 1e-12, "f32": 1e-5, "c64": 1e-5}
TIE = {"f64": 1e-12, "c128": 1e-12, "f32": 1e-5, "c64": 1e-5}


def to_np(a):
    if a is None:
        return None
    if hasattr(a, "detach"):
        return a.detach().cpu().numpy()
    return np.asarray(a)


def agreed_prefix(gpu, orc, tie, random_mode=True, residual_scaled=False, estimate_eps=None):
    """Number of leading steps with identical pivots, and the first step the
    oracle flags as a near-tie (steps after it are not required to agree).

    With residual_scaled, the window at step t is tie * sqrt(T_0 / T_t): the
    data's rounding is absolute (of the size of the input's entries), so its
    effect on the weights relative to the current total grows as the residual
    shrinks.  With estimate_eps (matrix-free form), the window also covers the
    row-norm estimate's absolute error, of order estimate_eps * T_0, relative
    to the current total T_t."""
    gI, gJ = to_np(gpu.I), to_np(gpu.J)
    oI, oJ = orc["I"], orc["J"]
    k = min(len(gI), len(oI))
    if random_mode:
        m = np.minimum(orc["row_margin"], orc["col_margin"])[:k]
        thr = np.full(k, tie)
        T = np.asarray(orc["T"][:k])
        if residual_scaled:
            thr = tie * np.sqrt(T[0] / np.maximum(T, 1e-300))
        if estimate_eps is not None:
            thr = np.maximum(thr, estimate_eps * T[0] / np.maximum(T, 1e-300))
        bad = np.nonzero(m < thr)[0]
        tie_step = int(bad[0]) if len(bad) else k
    else:
        tie_step = k
    same = 0
    while same < k and gI[same] == oI[same] and gJ[same] == oJ[same]:
        same += 1
    return same, tie_step


def assert_pivots(gpu, orc, tie, random_mode=True, min_steps=1, residual_scaled=False, estimate_eps=None):
    same, tie_step = agreed_prefix(gpu, orc, tie, random_mode, residual_scaled, estimate_eps)
    assert same >= min(tie_step, len(orc["I"])), (
        f"pivots differ at step {same} before the first near-tie step {tie_step}: "
        f"gpu {to_np(gpu.I)[:same + 1]} / {to_np(gpu.J)[:same + 1]} vs "
        f"oracle {orc['I'][:same + 1]} / {orc['J'][:same + 1]}")
    assert same >= min_steps, f"only {same} agreed steps"
    return same


def assert_factors(gpu, orc, upto, tol):
    if upto == 0:
        return
    Lg, Ug = to_np(gpu.L)[:, :upto], to_np(gpu.U)[:upto]
    Lo, Uo = orc["L"][:, :upto], orc["U"][:upto]
    piv = Uo[np.arange(upto), orc["J"][:upto]]
    Cg, Co = Lg * piv[None, :], Lo * piv[None, :]
    ec = np.linalg.norm(Cg - Co) / max(np.linalg.norm(Co), 1e-300)
    eu = np.linalg.norm(Ug - Uo) / max(np.linalg.norm(Uo), 1e-300)
    log = os.environ.get("RPLU_PARITY_LOG")
    if log:  # one line per comparison: the measured errors beside the tolerance they are held to
        with open(log, "a") as f:
            f.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]}\t{upto}\t{ec:.3e}\t{eu:.3e}\t"
                    f"{tol:.1e}\n")
    assert ec <= tol and eu <= tol, (f"normwise residual-column err {ec:.3e}, U err {eu:.3e} "
                                     f"(tol {tol:.1e}, {upto} steps)")
    return ec, eu


def rel_error(A, L, U):
    return np.linalg.norm(A - to_np(L) @ to_np(U)) / np.linalg.norm(A)
