"""The double-double arithmetic of the CUR forms' core (csrc/dd.cuh), compiled
as host C++ with g++ (no FMA contraction; the FMA it calls is exact by
definition), against exact rational arithmetic: TwoProduct is exact, and sums,
products and reciprocals are accurate to a few units of 2^-104."""
import os
import random
import shutil
import subprocess
from fractions import Fraction as F

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_22344_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("dd") / "dd_check")
    subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "harness", "dd_check.cpp"), "-o", exe], check=True)
    return exe


def _rdd(rng):
    hi = rng.uniform(-1, 1) * 10.0 ** rng.randint(-12, 12)
    lo = hi * rng.uniform(-1, 1) * 2.0 ** -54
    s = hi + lo  # normalise: |lo| <= ulp(hi) / 2
    return s, lo - (s - hi)


def test_operations_against_exact_rationals(checker):
    rng = random.Random(7)
    cases = []
    for _ in range(2000):
        a, b = _rdd(rng), _rdd(rng)
        cases += [("add", a, b), ("mul", a, b), ("mul_d", a, (b[0], 0.0)), ("recip", a, (1.0, 0.0)),
                  ("two_prod", (a[0], 0.0), (b[0], 0.0))]
    text = "".join(f"{op} {a[0]!r} {a[1]!r} {b[0]!r} {b[1]!r}\n" for op, a, b in cases)
    out = subprocess.run([checker], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    worst = {}
    for (op, a, b), line in zip(cases, out):
        hi, lo = (float(x) for x in line.split())
        got = F(hi) + F(lo)
        A, B = F(a[0]) + F(a[1]), F(b[0]) + F(b[1])
        exact = {"add": A + B, "mul": A * B, "mul_d": A * B, "recip": 1 / A, "two_prod": A * B}[op]
        if op == "two_prod":
            assert got == exact
            continue
        scale = abs(A) + abs(B) if op == "add" else abs(exact)
        if scale:
            worst[op] = max(worst.get(op, 0.0), float(abs(got - exact) / scale))
        assert abs(lo) <= abs(hi) * 2.0 ** -52  # normalised result
    for op, w in worst.items():
        assert w <= 16 * 2.0 ** -104, (op, w)
