"""The library's host-side quadtrees and interaction lists (csrc/bh_plan.h,
App. C, Algorithm C.1), built with g++ into a small checker: the trees are
permutations with boxes that hold their points and children that tile their
parent; every (target, source) pair is covered exactly once, by an aggregated
source node of its target leaf or by an exact source leaf; alpha is
1 / d_min^2(source node, leaf).  The bounds evaluated from these lists equal
the oracle's bounds (its own tree code, pinned against brute-force norms)."""
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
    exe = str(tmp_path_factory.mktemp("bh") / "bh_plan_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "harness", "bh_plan_check.cpp"),
                    "-o", exe], check=True)
    return exe


def _run(checker, tmp_path, x, y, G, B, nu, leaf):
    n, m, p = len(x), len(y), G.shape[1]
    f = tmp_path / "in.bin"
    with open(f, "wb") as fh:
        fh.write(np.array([n, m, p, leaf], dtype=np.int64).tobytes())
        fh.write(np.array([nu], dtype=np.float64).tobytes())
        for a in (x, y, G, B):
            fh.write(np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).tobytes())
    out = subprocess.run([checker, str(f)], capture_output=True, text=True, timeout=300)
    lines = out.stdout.split("\n")
    assert out.returncode == 0 and lines[0].startswith("ok"), out.stdout[:200] + out.stderr
    return np.array([float(v) for v in lines[1:1 + n]])


def _case(kind, seed, n=180, m=150):
    rng = np.random.default_rng(seed)
    if kind == "spirals":
        x, y = W.cauchy_spirals(n, m, seed=seed)
        return x, y, np.ones((n, 1), complex), np.ones((1, m), complex)
    if kind == "intervals":
        x, y = rng.uniform(-1, 1, n) + 0j, rng.uniform(3, 5, m) + 0j
        return x, y, rng.standard_normal((n, 2)) + 0j, rng.standard_normal((2, m)) + 0j
    if kind == "clouds":
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        y = 0.5 + rng.standard_normal(m) + 1j * rng.standard_normal(m)
        G = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
        B = rng.standard_normal((3, m)) + 1j * rng.standard_normal((3, m))
        return x, y, G, B
    if kind == "coincident":  # repeated points: zero-extent leaves larger than the leaf size
        x = np.repeat(rng.standard_normal(12) + 1j * rng.standard_normal(12), n // 12)
        y = 4 + np.repeat(rng.standard_normal(10) + 1j * rng.standard_normal(10), m // 10)
        return x, y, np.ones((len(x), 1), complex), np.ones((1, len(y)), complex)
    # disk, the Loewner points of the paper's Sec. 5.2 experiments, p = 2
    x = np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
    y = np.sqrt(rng.random(m)) * np.exp(2j * np.pi * rng.random(m))
    f = lambda z: np.tan(2 * z ** 4)  # noqa: E731
    G, B = W.loewner_generators(x, y, f(x), f(y))
    return x, y, G, B


@pytest.mark.parametrize("kind", ["spirals", "intervals", "clouds", "coincident", "disk"])
@pytest.mark.parametrize("nu,leaf", [(1.0, 8), (2.0, 16), (5.0, 32), (5.0, 4), (5.0, 1000)])
def test_lists_partition_the_pairs_and_match_the_oracle(checker, tmp_path, orc, kind, nu, leaf):
    x, y, G, B = _case(kind, 3)
    u = _run(checker, tmp_path, x, y, G, B, nu, leaf)
    uo = orc.bh_bounds(x, y, G, B, nu=nu, leaf=leaf)
    np.testing.assert_allclose(u, uo, rtol=1e-11, atol=0)


@pytest.mark.parametrize("n,m", [(1, 1), (1, 40), (40, 1), (3, 2)])
def test_tiny_problems(checker, tmp_path, orc, n, m):
    rng = np.random.default_rng(n * 100 + m)
    x = rng.standard_normal(n) + 0j
    y = 5 + rng.standard_normal(m) + 0j
    G, B = np.ones((n, 1), complex), np.ones((1, m), complex)
    u = _run(checker, tmp_path, x, y, G, B, 5.0, 4)
    np.testing.assert_allclose(u, orc.bh_bounds(x, y, G, B, nu=5.0, leaf=4), rtol=1e-12)
    rho = (np.abs(W.cauchy_like_dense(x, y, G, B)) ** 2).sum(axis=1)
    assert np.all(u >= rho * (1 - 1e-12))
