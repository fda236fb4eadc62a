// Exact 128-bit fixed-point weights for the inverse-CDF draws.
//
// A non-negative weight w (an FP64 squared row norm, or the exact square of an
// FP32/FP64 entry) is represented as floor(w * 2^E) in an unsigned 128-bit
// integer.  E is chosen from the largest weight and the number of weights so
// that the total of all weights stays below 2^127; the smallest representable
// step is then at most 2^-(126 - bits(count)) of the largest weight.  Sums of
// these integers are exact and independent of the order of summation, so a
// prefix sum can be split over threads, warps and blocks in any way and still
// give the same draw.
//
// Compiles as CUDA device code and as plain host C++ (gcc), so the arithmetic
// is tested on the CPU.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define RPLU_HD __host__ __device__ __forceinline__
#else
#define RPLU_HD inline
#endif

namespace rplu {

typedef unsigned __int128 u128;

RPLU_HD uint64_t fx_bits64(double v) {
  uint64_t b;
  memcpy(&b, &v, 8);
  return b;
}
RPLU_HD uint32_t fx_bits32(float v) {
  uint32_t b;
  memcpy(&b, &v, 4);
  return b;
}

// bit length of a non-negative count (0 for 0)
RPLU_HD int fx_bitlen(uint64_t c) {
  int b = 0;
  while (c) {
    ++b;
    c >>= 1;
  }
  return b;
}

// (mant, X): w = mant * 2^X for the FP64 value with bits b (sign ignored)
RPLU_HD void fx_split64(uint64_t b, uint64_t& mant, int& X) {
  const int ex = (int)((b >> 52) & 0x7FF);
  const uint64_t f = b & ((1ull << 52) - 1);
  if (ex == 0) { mant = f; X = -1074; }
  else { mant = f | (1ull << 52); X = ex - 1075; }
}
RPLU_HD void fx_split32(uint32_t b, uint32_t& mant, int& X) {
  const int ex = (int)((b >> 23) & 0xFF);
  const uint32_t f = b & 0x7FFFFFu;
  if (ex == 0) { mant = f; X = -149; }
  else { mant = f | 0x800000u; X = ex - 150; }
}

// v * 2^sh for a 128-bit v, truncated (sh may be negative)
RPLU_HD u128 fx_shift(u128 v, int sh) {
  if (v == 0) return 0;
  if (sh >= 0) return sh >= 128 ? (u128)0 : (v << sh);
  const int r = -sh;
  return r >= 128 ? (u128)0 : (v >> r);
}

// Scale exponent for weights that are FP64 values <= the value with bits maxb.
RPLU_HD int fx_scale_f64(uint64_t maxb, int64_t count) {
  int ex = (int)((maxb >> 52) & 0x7FF);
  if (ex == 0) ex = 1;  // subnormal or zero maximum
  // every weight < 2^(ex - 1022); count * that * 2^E <= 2^127
  return 1149 - ex - fx_bitlen((uint64_t)count);
}

// Scale exponent for squares of FP32 entries with |v| <= the value with bits
// maxb; `terms` = 2 for complex entries (|re|^2 + |im|^2), else 1.
RPLU_HD int fx_scale_sq32(uint32_t maxb, int64_t count, int terms) {
  int ex = (int)((maxb >> 23) & 0xFF);
  if (ex == 0) ex = 1;
  // every |v| < 2^(ex - 126); square < 2^(2 ex - 252)
  return 127 - fx_bitlen((uint64_t)count) - (terms == 2 ? 1 : 0) - 2 * (ex - 126);
}
RPLU_HD int fx_scale_sq64(uint64_t maxb, int64_t count, int terms) {
  int ex = (int)((maxb >> 52) & 0x7FF);
  if (ex == 0) ex = 1;
  return 127 - fx_bitlen((uint64_t)count) - (terms == 2 ? 1 : 0) - 2 * (ex - 1022);
}

// floor(w * 2^E) for a non-negative FP64 w
RPLU_HD u128 fx_f64(double w, int E) {
  uint64_t mant;
  int X;
  fx_split64(fx_bits64(w) & ~(1ull << 63), mant, X);
  return fx_shift((u128)mant, X + E);
}

// floor(v^2 * 2^E), exact square of an FP32 / FP64 value
RPLU_HD u128 fx_sq(float v, int E) {
  uint32_t mant;
  int X;
  fx_split32(fx_bits32(v) & 0x7FFFFFFFu, mant, X);
  return fx_shift((u128)((uint64_t)mant * mant), 2 * X + E);
}
RPLU_HD u128 fx_sq(double v, int E) {
  uint64_t mant;
  int X;
  fx_split64(fx_bits64(v) & ~(1ull << 63), mant, X);
  return fx_shift((u128)mant * mant, 2 * X + E);
}

// floor(U * T / 2^53) for U < 2^53, T < 2^127: the draw target for the
// uniform U * 2^-53.
RPLU_HD u128 fx_target(uint64_t U, u128 T) {
  const uint64_t tl = (uint64_t)T, th = (uint64_t)(T >> 64);
  const u128 p0 = (u128)U * tl;  // < 2^117
  const u128 p1 = (u128)U * th;  // < 2^116
  return (p1 << 11) + (p0 >> 53);
}

// v * 2^-E as FP64 (the exact integer rounded to FP64, then scaled exactly
// unless the result underflows)
RPLU_HD double fx_to_double(u128 v, int E) {
  const double hi = (double)(uint64_t)(v >> 64);
  const double lo = (double)(uint64_t)v;
  return ldexp(hi * 18446744073709551616.0 + lo, -E);
}

}  // namespace rplu
