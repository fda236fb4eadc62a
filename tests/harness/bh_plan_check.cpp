// Host-side check of the quadtree / interaction-list builder (bh_plan.h).
// Reads a problem from the binary file argv[1]:
//   int64 n, m, p, leaf; double nu; then x (n complex), y (m complex),
//   G (n x p complex, row-major), B (p x m complex, row-major), as re/im pairs.
// Verifies:
//   * every target point lies in exactly one target leaf, every tree node's
//     box holds its points and the permutations are permutations;
//   * every (target, source) pair is covered exactly once, by one aggregated
//     source node of its target leaf or by one exact source leaf;
//   * aggregated entries keep the source node apart from the leaf
//     (d_min^2(s, leaf) > 0) and carry alpha = 1 / d_min^2(s, leaf);
// then prints "ok" and the n bounds of Algorithm C.2 evaluated from the lists
// in FP64 (one per line), for comparison with the oracle's bounds.
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "bh_plan.h"

using cplx = std::complex<double>;
using namespace rplu;

static int fail(const char* what) {
  std::printf("FAIL %s\n", what);
  return 1;
}

int main(int argc, char** argv) {
  if (argc < 2) return fail("usage");
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return fail("open");
  int64_t hdr[4];
  double nu;
  if (std::fread(hdr, 8, 4, f) != 4 || std::fread(&nu, 8, 1, f) != 1) return fail("header");
  const int64_t n = hdr[0], m = hdr[1], P = hdr[2], leaf = hdr[3];
  std::vector<cplx> x(n), y(m), G(n * P), B(P * m);
  if (std::fread(x.data(), 16, n, f) != (size_t)n || std::fread(y.data(), 16, m, f) != (size_t)m ||
      std::fread(G.data(), 16, n * P, f) != (size_t)(n * P) || std::fread(B.data(), 16, P * m, f) != (size_t)(P * m))
    return fail("body");
  std::fclose(f);
  std::vector<double> xr(n), xi(n), yr(m), yi(m);
  for (int64_t q = 0; q < n; ++q) { xr[q] = x[q].real(); xi[q] = x[q].imag(); }
  for (int64_t q = 0; q < m; ++q) { yr[q] = y[q].real(); yi[q] = y[q].imag(); }
  BhPlan pl;
  bh_make_plan(pl, xr.data(), xi.data(), n, yr.data(), yi.data(), m, nu, leaf);

  // trees: permutations and boxes
  for (int side = 0; side < 2; ++side) {
    const BhTree& t = side ? pl.src : pl.tgt;
    const std::vector<double>& re = side ? yr : xr;
    const std::vector<double>& im = side ? yi : xi;
    const int64_t cnt = side ? m : n;
    std::vector<int> seen(cnt, 0);
    for (int64_t q : t.perm) {
      if (q < 0 || q >= cnt || seen[q]++) return fail("perm");
    }
    for (const BhNode& nd : t.nodes) {
      for (int64_t q = nd.lo; q < nd.hi; ++q) {
        const int64_t i = t.perm[q];
        if (re[i] < nd.x0 || re[i] > nd.x1 || im[i] < nd.y0 || im[i] > nd.y1) return fail("box");
      }
      if (!nd.leaf) {
        int64_t at = nd.lo;
        for (int c = 0; c < 4; ++c) {
          if (nd.child[c] < 0) continue;
          const BhNode& ch = t.nodes[nd.child[c]];
          if (ch.lo != at) return fail("children not contiguous");
          at = ch.hi;
        }
        if (at != nd.hi) return fail("children do not cover the node");
      }
    }
  }
  // coverage of every (target, source) pair
  std::vector<int> cover(n * m, 0);
  int64_t covered_leaves = 0;
  for (size_t l = 0; l < pl.tleaf.size(); ++l) {
    const BhNode& tl = pl.tgt.nodes[pl.tleaf[l]];
    covered_leaves += tl.hi - tl.lo;
    for (int64_t e = pl.a_off[l]; e < pl.a_off[l + 1]; ++e) {
      const BhNode& s = pl.src.nodes[pl.a_node[e]];
      const double dn = bh_detail::dmin2(s, tl);
      if (!(dn > 0.0)) return fail("aggregated pair touches its leaf");
      if (pl.a_alpha[e] != 1.0 / dn) return fail("alpha");
      for (int64_t a = tl.lo; a < tl.hi; ++a)
        for (int64_t b = s.lo; b < s.hi; ++b) ++cover[pl.tgt.perm[a] * m + pl.src.perm[b]];
    }
    for (int64_t e = pl.e_off[l]; e < pl.e_off[l + 1]; ++e) {
      const BhNode& s = pl.src.nodes[pl.e_node[e]];
      if (!s.leaf) return fail("exact entry is not a source leaf");
      for (int64_t a = tl.lo; a < tl.hi; ++a)
        for (int64_t b = s.lo; b < s.hi; ++b) ++cover[pl.tgt.perm[a] * m + pl.src.perm[b]];
    }
  }
  if (covered_leaves != n) return fail("target leaves do not partition the points");
  for (int64_t q = 0; q < n * m; ++q)
    if (cover[q] != 1) return fail("pair covered other than once");

  // bounds from the lists (Algorithm C.2), FP64
  std::vector<double> u(n, 0.0);
  for (size_t l = 0; l < pl.tleaf.size(); ++l) {
    const BhNode& tl = pl.tgt.nodes[pl.tleaf[l]];
    for (int64_t e = pl.a_off[l]; e < pl.a_off[l + 1]; ++e) {
      const BhNode& s = pl.src.nodes[pl.a_node[e]];
      std::vector<cplx> H(P * P, 0.0);
      for (int64_t b = s.lo; b < s.hi; ++b) {
        const int64_t j = pl.src.perm[b];
        for (int64_t r = 0; r < P; ++r)
          for (int64_t c = 0; c < P; ++c) H[r * P + c] += B[r * m + j] * std::conj(B[c * m + j]);
      }
      for (int64_t a = tl.lo; a < tl.hi; ++a) {
        const int64_t i = pl.tgt.perm[a];
        cplx acc = 0.0;
        for (int64_t r = 0; r < P; ++r)
          for (int64_t c = 0; c < P; ++c) acc += G[i * P + r] * H[r * P + c] * std::conj(G[i * P + c]);
        u[i] += pl.a_alpha[e] * acc.real();
      }
    }
    for (int64_t e = pl.e_off[l]; e < pl.e_off[l + 1]; ++e) {
      const BhNode& s = pl.src.nodes[pl.e_node[e]];
      for (int64_t a = tl.lo; a < tl.hi; ++a) {
        const int64_t i = pl.tgt.perm[a];
        for (int64_t b = s.lo; b < s.hi; ++b) {
          const int64_t j = pl.src.perm[b];
          cplx sv = 0.0;
          for (int64_t r = 0; r < P; ++r) sv += G[i * P + r] * B[r * m + j];
          u[i] += std::norm(sv / (x[i] - y[j]));
        }
      }
    }
  }
  std::printf("ok %zu %zu %zu\n", pl.tleaf.size(), pl.src.nodes.size(), pl.a_node.size());
  for (int64_t i = 0; i < n; ++i) std::printf("%.17g\n", u[i]);
  return 0;
}
