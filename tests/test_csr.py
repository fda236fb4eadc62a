"""The host-side CSR checks and the stable CSR -> CSC transposition of the
sparse CUR form (csrc/csr.h), built with g++ into a small checker: valid
matrices transpose exactly as scipy's canonical CSC does, malformed ones are
rejected with their reason."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_22344_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("csr") / "csr_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "harness", "csr_check.cpp"), "-o", exe],
                   check=True)
    return exe


def _run(exe, n, m, rp, ci, v):
    text = f"{n} {m} {len(ci)}\n" + " ".join(map(str, rp)) + "\n" + " ".join(map(str, ci)) + "\n" + \
        " ".join(repr(float(x)) for x in v) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_transposition_matches_scipy(checker, seed):
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    S = sp.random(n, m, density=0.1, random_state=rng, data_rvs=lambda k: rng.standard_normal(k)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    out = _run(checker, n, m, S.indptr, S.indices, S.data)
    assert out[0] == "ok"
    C = S.tocsc()
    C.sort_indices()
    assert [int(x) for x in out[1].split()] == list(C.indptr)
    if C.nnz:
        assert [int(x) for x in out[2].split()] == list(C.indices)
        assert np.array_equal(np.array([float(x) for x in out[3].split()]), C.data)


def test_graph_with_empty_rows_and_columns(checker):
    import scipy.sparse as sp
    S = W.chung_lu_graph(300, avg_degree=2.0, exponent=2.5, seed=3)
    S = sp.csr_matrix(S)
    S.sort_indices()
    assert (np.diff(S.indptr) == 0).any()  # isolated vertices
    out = _run(checker, 300, 300, S.indptr, S.indices, S.data)
    assert out[0] == "ok"
    C = S.tocsc()
    C.sort_indices()
    assert [int(x) for x in out[1].split()] == list(C.indptr)


def _walk_cost(d, G, long_deg=8):
    """FP64 warp instructions of one walk with G lanes per row: per group of
    32 / G consecutive rows the longest short row's ceil(degree / G) plus
    log2(G)."""
    rpw = 32 // G
    cost = 0
    for g0 in range(0, len(d), rpw):
        grp = [x for x in d[g0:g0 + rpw] if x <= long_deg]
        cost += max([-(-x // G) for x in grp], default=0) + int(np.log2(G))
    return cost


def test_segment_lanes_of_a_power_law_graph(checker):
    """The kernels' walk of the rows: rows of degree above 8 (the harness's
    threshold) are listed for a CTA each, and the short rows share warps in
    segments of G lanes, G in {2, ..., 32} minimising the walk's FP64 warp
    instructions (ties to the larger G)."""
    import scipy.sparse as sp
    for seed, deg in ((1, 3.0), (2, 6.0), (4, 0.5)):
        S = sp.csr_matrix(W.chung_lu_graph(500, avg_degree=deg, exponent=2.2, seed=seed))
        S.sort_indices()
        out = _run(checker, 500, 500, S.indptr, S.indices, S.data)
        fields = [int(x) for x in out[4].split()]
        d = np.diff(S.indptr).tolist()
        assert fields[1:] == [p for p, x in enumerate(d) if x > 8]
        costs = {G: _walk_cost(d, G) for G in (32, 16, 8, 4, 2)}
        best = min(costs.values())
        assert fields[0] == max(G for G, c in costs.items() if c == best), costs


@pytest.mark.parametrize("rp,ci,v,why", [
    ([1, 2, 3, 4], [0, 2, 1, 0], [1, 2, 3, 4], "row_ptr[0] must be 0"),
    ([0, 3, 2, 4], [0, 2, 1, 0], [1, 2, 3, 4], "row_ptr must be nondecreasing"),
    ([0, 2, 3, 4], [0, 3, 1, 0], [1, 2, 3, 4], "column index out of range"),
    ([0, 2, 3, 4], [2, 0, 1, 0], [1, 2, 3, 4], "column indices must increase strictly within each row"),
    ([0, 2, 3, 4], [1, 1, 1, 0], [1, 2, 3, 4], "column indices must increase strictly within each row"),
    ([0, 2, 3, 4], [0, 2, 1, 0], [1, float("nan"), 3, 4], "input has a non-finite entry"),
])
def test_malformed_csr_is_rejected(checker, rp, ci, v, why):
    assert _run(checker, 3, 3, rp, ci, v)[0] == why
