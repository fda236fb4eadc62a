// Quadtrees and interaction lists for the row-norm upper bounds of
// Cauchy-like matrices (App. C, Algorithm C.1), built once per factorization
// on the host.  Plain C++ (no CUDA), tested on the CPU (tests/test_bh_plan.py).
//
// Tree rules: a node holds the contiguous range [lo, hi) of its points in
// tree order and the tight bounding box of those points (real part x,
// imaginary part y); it is a leaf when it holds at most `leaf` points, when
// its box has no extent, or at depth 60.  A node splits its box at the centre
// into four quadrants taken in the order (low x, low y), (high x, low y),
// (low x, high y), (high x, high y), a point on a split line going to the
// high side, points keeping their relative order.
//
// Lists (Algorithm C.1): starting from the pair of roots, a (source, target)
// pair with d_max^2 <= nu d_min^2 (box distances, d_min > 0) is aggregated:
// every target leaf under the target node records (source node, alpha =
// 1 / d_min^2(source node, leaf)); a pair of two leaves is recorded as exact;
// otherwise the node with more points (the target on a tie) is split, a leaf
// never.
#pragma once

#include <stdint.h>

#include <vector>

namespace rplu {

struct BhNode {
  int64_t lo = 0, hi = 0;
  double x0 = 0, x1 = 0, y0 = 0, y1 = 0;
  int64_t child[4] = {-1, -1, -1, -1};
  bool leaf = true;
};

struct BhTree {
  std::vector<BhNode> nodes;  // nodes[0] is the root
  std::vector<int64_t> perm;  // tree order -> original index
};

namespace bh_detail {

inline int64_t build(BhTree& t, const double* re, const double* im, int64_t lo, int64_t hi, int64_t leaf,
                     int depth, std::vector<int64_t>& tmp) {
  const int64_t id = (int64_t)t.nodes.size();
  t.nodes.emplace_back();
  BhNode nd;
  nd.lo = lo;
  nd.hi = hi;
  nd.x0 = nd.y0 = 1e308;
  nd.x1 = nd.y1 = -1e308;
  for (int64_t q = lo; q < hi; ++q) {
    const double a = re[t.perm[q]], b = im[t.perm[q]];
    nd.x0 = a < nd.x0 ? a : nd.x0;
    nd.x1 = a > nd.x1 ? a : nd.x1;
    nd.y0 = b < nd.y0 ? b : nd.y0;
    nd.y1 = b > nd.y1 ? b : nd.y1;
  }
  nd.leaf = (hi - lo <= leaf) || (nd.x1 <= nd.x0 && nd.y1 <= nd.y0) || depth >= 60;
  if (!nd.leaf) {
    const double cx = 0.5 * (nd.x0 + nd.x1), cy = 0.5 * (nd.y0 + nd.y1);
    int64_t bounds[5];
    int64_t w = 0;
    tmp.resize((size_t)(hi - lo));
    for (int c = 0; c < 4; ++c) {
      bounds[c] = lo + w;
      for (int64_t q = lo; q < hi; ++q) {
        const int64_t i = t.perm[q];
        const int qc = (re[i] >= cx ? 1 : 0) + (im[i] >= cy ? 2 : 0);
        if (qc == c) tmp[(size_t)w++] = i;
      }
    }
    bounds[4] = hi;
    for (int64_t q = lo; q < hi; ++q) t.perm[q] = tmp[(size_t)(q - lo)];
    for (int c = 0; c < 4; ++c)
      if (bounds[c + 1] > bounds[c]) nd.child[c] = build(t, re, im, bounds[c], bounds[c + 1], leaf, depth + 1, tmp);
  }
  t.nodes[(size_t)id] = nd;
  return id;
}

inline double dmin2(const BhNode& a, const BhNode& b) {
  double dx = 0.0, dy = 0.0;
  if (a.x1 < b.x0) dx = b.x0 - a.x1;
  else if (b.x1 < a.x0) dx = a.x0 - b.x1;
  if (a.y1 < b.y0) dy = b.y0 - a.y1;
  else if (b.y1 < a.y0) dy = a.y0 - b.y1;
  return dx * dx + dy * dy;
}

inline double dmax2(const BhNode& a, const BhNode& b) {
  const double ax = a.x1 - b.x0 < 0 ? b.x0 - a.x1 : a.x1 - b.x0;
  const double bx = b.x1 - a.x0 < 0 ? a.x0 - b.x1 : b.x1 - a.x0;
  const double ay = a.y1 - b.y0 < 0 ? b.y0 - a.y1 : a.y1 - b.y0;
  const double by = b.y1 - a.y0 < 0 ? a.y0 - b.y1 : b.y1 - a.y0;
  const double dx = ax > bx ? ax : bx, dy = ay > by ? ay : by;
  return dx * dx + dy * dy;
}

inline void leaves_under(const BhTree& t, int64_t node, std::vector<int64_t>& out) {
  const BhNode& nd = t.nodes[(size_t)node];
  if (nd.leaf) {
    out.push_back(node);
    return;
  }
  for (int c = 0; c < 4; ++c)
    if (nd.child[c] >= 0) leaves_under(t, nd.child[c], out);
}

}  // namespace bh_detail

inline void bh_build_tree(BhTree& t, const double* re, const double* im, int64_t n, int64_t leaf) {
  t.nodes.clear();
  t.perm.resize((size_t)n);
  for (int64_t q = 0; q < n; ++q) t.perm[(size_t)q] = q;
  std::vector<int64_t> tmp;
  if (n > 0) bh_detail::build(t, re, im, 0, n, leaf, 0, tmp);
}

// Interaction lists per target leaf, in CSR form over the target leaves.
struct BhPlan {
  BhTree tgt, src;
  std::vector<int64_t> tleaf;   // target leaf node ids
  std::vector<int64_t> a_off;   // aggregated entries of leaf l: [a_off[l], a_off[l+1])
  std::vector<int32_t> a_node;  // source node
  std::vector<double> a_alpha;  // 1 / d_min^2(source node, leaf)
  std::vector<int64_t> e_off;   // exact source leaves of leaf l: [e_off[l], e_off[l+1])
  std::vector<int32_t> e_node;
};

inline void bh_make_plan(BhPlan& p, const double* xre, const double* xim, int64_t n, const double* yre,
                         const double* yim, int64_t m, double nu, int64_t leaf) {
  using namespace bh_detail;
  bh_build_tree(p.tgt, xre, xim, n, leaf);
  bh_build_tree(p.src, yre, yim, m, leaf);
  p.tleaf.clear();
  if (n > 0) leaves_under(p.tgt, 0, p.tleaf);
  std::vector<int64_t> slot(p.tgt.nodes.size(), -1);
  for (size_t l = 0; l < p.tleaf.size(); ++l) slot[(size_t)p.tleaf[l]] = (int64_t)l;
  std::vector<std::vector<std::pair<int32_t, double>>> agg(p.tleaf.size());
  std::vector<std::vector<int32_t>> ex(p.tleaf.size());
  std::vector<std::pair<int64_t, int64_t>> stack;  // (source, target)
  if (n > 0 && m > 0) stack.push_back({0, 0});
  std::vector<int64_t> under;
  while (!stack.empty()) {
    const auto pr = stack.back();
    stack.pop_back();
    const BhNode& s = p.src.nodes[(size_t)pr.first];
    const BhNode& t = p.tgt.nodes[(size_t)pr.second];
    const double dn = dmin2(s, t), dx = dmax2(s, t);
    if (dn > 0.0 && dx <= nu * dn) {
      under.clear();
      leaves_under(p.tgt, pr.second, under);
      for (int64_t lf : under)
        agg[(size_t)slot[(size_t)lf]].push_back({(int32_t)pr.first, 1.0 / dmin2(s, p.tgt.nodes[(size_t)lf])});
      continue;
    }
    if (s.leaf && t.leaf) {
      ex[(size_t)slot[(size_t)pr.second]].push_back((int32_t)pr.first);
      continue;
    }
    const bool split_t = !t.leaf && (s.leaf || (t.hi - t.lo) >= (s.hi - s.lo));
    if (split_t) {
      for (int c = 0; c < 4; ++c)
        if (t.child[c] >= 0) stack.push_back({pr.first, t.child[c]});
    } else {
      for (int c = 0; c < 4; ++c)
        if (s.child[c] >= 0) stack.push_back({s.child[c], pr.second});
    }
  }
  p.a_off.assign(p.tleaf.size() + 1, 0);
  p.e_off.assign(p.tleaf.size() + 1, 0);
  p.a_node.clear();
  p.a_alpha.clear();
  p.e_node.clear();
  for (size_t l = 0; l < p.tleaf.size(); ++l) {
    for (const auto& e : agg[l]) {
      p.a_node.push_back(e.first);
      p.a_alpha.push_back(e.second);
    }
    for (int32_t e : ex[l]) p.e_node.push_back(e);
    p.a_off[l + 1] = (int64_t)p.a_node.size();
    p.e_off[l + 1] = (int64_t)p.e_node.size();
  }
}

}  // namespace rplu
