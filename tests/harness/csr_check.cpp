// Reads a CSR matrix from stdin ("n m nnz", then row_ptr, col_idx, val) and
// prints csr_check's verdict ("ok" or the reason) and, when valid, the CSC
// arrays from csr_to_csc (col_ptr, row_idx, values with 17 significant digits),
// then segment_lanes of the rows with long_deg = 8 (G, then the long rows).
#include <cstdio>
#include <vector>

#include "csr.h"

int main() {
  long long n, m, nnz;
  if (std::scanf("%lld %lld %lld", &n, &m, &nnz) != 3) return 2;
  std::vector<int64_t> rp((size_t)n + 1);
  std::vector<int32_t> ci((size_t)(nnz > 0 ? nnz : 1));
  std::vector<double> v((size_t)(nnz > 0 ? nnz : 1));
  for (auto& x : rp) {
    long long t;
    if (std::scanf("%lld", &t) != 1) return 2;
    x = t;
  }
  for (long long e = 0; e < nnz; ++e) {
    int t;
    if (std::scanf("%d", &t) != 1) return 2;
    ci[(size_t)e] = t;
  }
  for (long long e = 0; e < nnz; ++e)
    if (std::scanf("%lf", &v[(size_t)e]) != 1) return 2;
  const char* why = rplu::csr_check(n, m, rp.data(), ci.data(), v.data());
  if (why[0]) {
    std::printf("%s\n", why);
    return 0;
  }
  std::printf("ok\n");
  std::vector<int64_t> cp;
  std::vector<int32_t> ri;
  std::vector<double> cv;
  rplu::csr_to_csc(n, m, rp.data(), ci.data(), v.data(), cp, ri, cv);
  for (auto x : cp) std::printf("%lld ", (long long)x);
  std::printf("\n");
  for (long long e = 0; e < nnz; ++e) std::printf("%d ", ri[(size_t)e]);
  std::printf("\n");
  for (long long e = 0; e < nnz; ++e) std::printf("%.17g ", cv[(size_t)e]);
  std::printf("\n");
  // the kernels' walk of the rows with long rows above degree 8: lanes per short row, then the long rows
  std::vector<int32_t> lr;
  const int G = rplu::segment_lanes(n, rp.data(), 8, lr);
  std::printf("%d", G);
  for (auto p : lr) std::printf(" %d", p);
  std::printf("\n");
  return 0;
}
