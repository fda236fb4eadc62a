// Host-side checks and transposition of a CSR matrix for the sparse CUR form
// (rplu_sparse_cur): plain C++, no CUDA, so it is also built and tested on the
// CPU (tests/harness/csr_check.cpp).
#pragma once

#include <cmath>
#include <cstdint>
#include <vector>

namespace rplu {

// Empty string when row_ptr (n + 1 entries), col_idx and val (row_ptr[n]
// entries each) form a valid CSR matrix with m columns: row_ptr[0] = 0 and
// nondecreasing, every column index in [0, m) and strictly increasing within its
// row (so entries are unique), every value finite.  Otherwise the reason.
inline const char* csr_check(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col_idx,
                             const double* val) {
  if (row_ptr[0] != 0) return "row_ptr[0] must be 0";
  for (int64_t p = 0; p < n; ++p)
    if (row_ptr[p + 1] < row_ptr[p]) return "row_ptr must be nondecreasing";
  for (int64_t p = 0; p < n; ++p) {
    for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
      const int32_t q = col_idx[e];
      if (q < 0 || q >= m) return "column index out of range";
      if (e > row_ptr[p] && q <= col_idx[e - 1]) return "column indices must increase strictly within each row";
      if (!std::isfinite(val[e])) return "input has a non-finite entry";
    }
  }
  return "";
}

// CSC of a valid CSR matrix by a stable counting sort: col_ptr (m + 1), and
// for each column its row indices in increasing order with their values.
inline void csr_to_csc(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                       std::vector<int64_t>& col_ptr, std::vector<int32_t>& row_idx, std::vector<double>& cval) {
  const int64_t nnz = row_ptr[n];
  col_ptr.assign((size_t)m + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) ++col_ptr[(size_t)col_idx[e] + 1];
  for (int64_t q = 0; q < m; ++q) col_ptr[(size_t)q + 1] += col_ptr[(size_t)q];
  std::vector<int64_t> next(col_ptr.begin(), col_ptr.end() - 1);
  row_idx.assign((size_t)(nnz > 0 ? nnz : 1), 0);
  cval.assign((size_t)(nnz > 0 ? nnz : 1), 0.0);
  for (int64_t p = 0; p < n; ++p) {
    for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
      const int64_t pos = next[(size_t)col_idx[e]]++;
      row_idx[(size_t)pos] = (int32_t)p;
      cval[(size_t)pos] = val[e];
    }
  }
}

// How the sparse kernels walk a compressed index (row pointers of the CSR, or
// column pointers of the CSC): rows of degree at most long_deg are walked by a
// segment of G lanes of a warp (32 / G consecutive rows per warp at a time),
// the longer rows are listed in *long_rows and each gets a whole CTA.  The
// walks' sums are FP64, a slow pipe on this GPU, so G (a power of two in
// [2, 32]) minimises the FP64 warp instructions of one walk over this matrix:
// per group of 32 / G rows, the longest row's ceil(degree / G) fused
// multiply-adds plus log2(G) butterfly additions; ties go to the larger G.
// Returns G.
inline int segment_lanes(int64_t n, const int64_t* ptr, int64_t long_deg, std::vector<int32_t>& long_rows) {
  long_rows.clear();
  for (int64_t p = 0; p < n; ++p)
    if (ptr[p + 1] - ptr[p] > long_deg) long_rows.push_back((int32_t)p);
  int best = 32, lg = 5;
  int64_t best_cost = -1;
  for (int G = 32; G >= 2; G /= 2, --lg) {
    const int64_t rpw = 32 / G;
    int64_t cost = 0;
    for (int64_t g0 = 0; g0 < n; g0 += rpw) {
      int64_t it = 0;
      for (int64_t p = g0; p < n && p < g0 + rpw; ++p) {
        const int64_t deg = ptr[p + 1] - ptr[p];
        if (deg > long_deg) continue;
        const int64_t c = (deg + G - 1) / G;
        it = c > it ? c : it;
      }
      cost += it + lg;
    }
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = G;
    }
  }
  return best;
}
}  // namespace rplu
