"""The fixed-point weight arithmetic of the CUDA sampler (csrc/fixedpoint.h),
compiled as host C++ with g++, against exact rational arithmetic."""
import os
import random
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2601_22344_gb300", "csrc")

HARNESS = r"""
#include <stdio.h>
#include <stdlib.h>
#include "fixedpoint.h"
using namespace rplu;
static void put(u128 v) { printf("%016llx%016llx\n", (unsigned long long)(v >> 64), (unsigned long long)v); }
int main() {
  char op[16];
  while (scanf("%15s", op) == 1) {
    if (op[0] == 'f') {            /* f <double bits> E */
      unsigned long long b; int E; scanf("%llx %d", &b, &E);
      double w; memcpy(&w, &b, 8); put(fx_f64(w, E));
    } else if (op[0] == 's') {     /* s <float bits> E */
      unsigned b; int E; scanf("%x %d", &b, &E);
      float v; memcpy(&v, &b, 4); put(fx_sq(v, E));
    } else if (op[0] == 'q') {     /* q <double bits> E */
      unsigned long long b; int E; scanf("%llx %d", &b, &E);
      double v; memcpy(&v, &b, 8); put(fx_sq(v, E));
    } else if (op[0] == 't') {     /* t U Thi Tlo */
      unsigned long long U, th, tl; scanf("%llx %llx %llx", &U, &th, &tl);
      put(fx_target(U, ((u128)th << 64) | tl));
    } else if (op[0] == 'd') {     /* d Thi Tlo E */
      unsigned long long th, tl; int E; scanf("%llx %llx %d", &th, &tl, &E);
      double r = fx_to_double(((u128)th << 64) | tl, E); unsigned long long rb; memcpy(&rb, &r, 8);
      printf("%016llx\n", rb);
    } else if (op[0] == 'e') {     /* e kind maxbits count terms */
      int kind, terms; unsigned long long mb; long long cnt; scanf("%d %llx %lld %d", &kind, &mb, &cnt, &terms);
      int E = kind == 0 ? fx_scale_f64(mb, cnt) : kind == 1 ? fx_scale_sq32((unsigned)mb, cnt, terms)
                                                              : fx_scale_sq64(mb, cnt, terms);
      printf("%d\n", E);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    d = tmp_path_factory.mktemp("fx")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split()
    return run


def _b64(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _b32(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _floor_pow2(fr, E):
    v = fr * (Fraction(2) ** E)
    return v.numerator // v.denominator


def test_f64_weights_exact(fx):
    rng = random.Random(1)
    vals = [0.0, 5e-324, 2.2250738585072014e-308, 1.0, 0.75, 3.0e300]
    vals += [rng.random() * 10 ** rng.randint(-300, 300) for _ in range(300)]
    lines, want = [], []
    for v in vals:
        E = rng.randint(-1200, 1200) if v else 0
        # keep the result inside 128 bits
        if v:
            e2 = Fraction(v).numerator.bit_length() - Fraction(v).denominator.bit_length()
            E = min(E, 120 - e2)
        lines.append(f"f {_b64(v):x} {E}")
        want.append(_floor_pow2(Fraction(v), E))
    got = [int(g, 16) for g in fx(lines)]
    assert got == want


def test_squares_exact(fx):
    rng = random.Random(2)
    lines, want = [], []
    for _ in range(300):
        v32 = struct.unpack("<f", struct.pack("<f", rng.uniform(-1, 1) * 10 ** rng.randint(-40, 38)))[0]
        E = 100 - 2 * (Fraction(abs(v32)).numerator.bit_length() - Fraction(abs(v32)).denominator.bit_length()) if v32 else 0
        lines.append(f"s {_b32(v32):x} {E}")
        want.append(_floor_pow2(Fraction(v32) ** 2, E))
        v64 = rng.uniform(-1, 1) * 10 ** rng.randint(-300, 300)
        E = 100 - 2 * (Fraction(abs(v64)).numerator.bit_length() - Fraction(abs(v64)).denominator.bit_length())
        lines.append(f"q {_b64(v64):x} {E}")
        want.append(_floor_pow2(Fraction(v64) ** 2, E))
    got = [int(g, 16) for g in fx(lines)]
    assert got == want


def test_target_exact(fx):
    rng = random.Random(3)
    lines, want = [], []
    for _ in range(300):
        U = rng.getrandbits(53)
        T = rng.getrandbits(rng.randint(1, 127))
        lines.append(f"t {U:x} {T >> 64:x} {T & (2**64 - 1):x}")
        want.append((U * T) >> 53)
    got = [int(g, 16) for g in fx(lines)]
    assert got == want
    assert all(g < max(1, (T_ := 0)) or True for g in got)


def test_to_double_rounds_to_nearest_ulp(fx):
    rng = random.Random(4)
    lines, exact = [], []
    for _ in range(200):
        T = rng.getrandbits(rng.randint(1, 127))
        E = rng.randint(-200, 900)
        lines.append(f"d {T >> 64:x} {T & (2**64 - 1):x} {E}")
        exact.append(Fraction(T) / Fraction(2) ** E)
    got = [struct.unpack("<d", struct.pack("<Q", int(g, 16)))[0] for g in fx(lines)]
    for g, e in zip(got, exact):
        assert abs(Fraction(g) - e) <= e * Fraction(1, 2 ** 51)


@pytest.mark.parametrize("kind,terms", [(0, 1), (1, 1), (1, 2), (2, 1), (2, 2)])
def test_scale_keeps_totals_below_2_127_with_fine_resolution(fx, kind, terms):
    rng = random.Random(5 + kind)
    lines, cases = [], []
    for _ in range(60):
        cnt = rng.choice([1, 2, 3, 1000, 32768, 20000, 1 << 20, (1 << 31) - 1])
        if kind == 0:
            mx = rng.random() * 10 ** rng.randint(-300, 300)
            mb = _b64(mx)
        elif kind == 1:
            mx = struct.unpack("<f", struct.pack("<f", rng.random() * 10 ** rng.randint(-37, 37)))[0]
            mb = _b32(mx)
        else:
            mx = rng.random() * 10 ** rng.randint(-150, 150)
            mb = _b64(mx)
        lines.append(f"e {kind} {mb:x} {cnt} {terms}")
        cases.append((mx, cnt))
    Es = [int(v) for v in fx(lines)]
    for (mx, cnt), E in zip(cases, Es):
        w = Fraction(mx) if kind == 0 else Fraction(mx) ** 2 * terms
        tot = w * cnt * Fraction(2) ** E
        assert tot < 2 ** 127
        # resolution: the largest weight spans at least 2^(124 - bits(count)) steps
        assert w * Fraction(2) ** E >= Fraction(2) ** (124 - cnt.bit_length() - (4 if kind else 1))
