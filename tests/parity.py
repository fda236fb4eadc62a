"""Comparison rules shared by the GPU parity tests.

Pivots: identical to the oracle's for every step before the first step whose
row or column draw the oracle reports within `tie` (relative) of a CDF
boundary; a different summation order may legitimately pick the neighbour
there, and the sequences may differ afterwards.  With FP32 data the window is
the FP32 perturbation of the weights.

Factors: over the agreed prefix, ||L_gpu - L_or||_F <= tol ||L_or||_F and
likewise for U (normwise; entrywise comparison is meaningless for late, small
rows and columns, whose rounding is amplified by 1/|pivot|).
"""
import numpy as np

GPU_TOL = {"f64": 1e-12, "c128": 1e-12, "f32": 1e-5, "c64": 1e-5}
TIE = {"f64": 1e-12, "c128": 1e-12, "f32": 1e-5, "c64": 1e-5}


def to_np(a):
    if a is None:
        return None
    if hasattr(a, "detach"):
        return a.detach().cpu().numpy()
    return np.asarray(a)


def agreed_prefix(gpu, orc, tie, random_mode=True, residual_scaled=False):
    """Number of leading steps with identical pivots, and the first step the
    oracle flags as a near-tie (steps after it are not required to agree).

    With residual_scaled, the window at step t is tie * sqrt(T_0 / T_t): the
    data's rounding is absolute (of the size of the input's entries), so its
    effect on the weights relative to the current total grows as the residual
    shrinks."""
    gI, gJ = to_np(gpu.I), to_np(gpu.J)
    oI, oJ = orc["I"], orc["J"]
    k = min(len(gI), len(oI))
    if random_mode:
        m = np.minimum(orc["row_margin"], orc["col_margin"])[:k]
        thr = np.full(k, tie)
        if residual_scaled:
            T = np.asarray(orc["T"][:k])
            thr = tie * np.sqrt(T[0] / np.maximum(T, 1e-300))
        bad = np.nonzero(m < thr)[0]
        tie_step = int(bad[0]) if len(bad) else k
    else:
        tie_step = k
    same = 0
    while same < k and gI[same] == oI[same] and gJ[same] == oJ[same]:
        same += 1
    return same, tie_step


def assert_pivots(gpu, orc, tie, random_mode=True, min_steps=1, residual_scaled=False):
    same, tie_step = agreed_prefix(gpu, orc, tie, random_mode, residual_scaled)
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
    el = np.linalg.norm(Lg - Lo) / max(np.linalg.norm(Lo), 1e-300)
    eu = np.linalg.norm(Ug - Uo) / max(np.linalg.norm(Uo), 1e-300)
    assert el <= tol and eu <= tol, f"normwise L err {el:.3e}, U err {eu:.3e} (tol {tol:.1e}, {upto} steps)"
    return el, eu


def rel_error(A, L, U):
    return np.linalg.norm(A - to_np(L) @ to_np(U)) / np.linalg.norm(A)
