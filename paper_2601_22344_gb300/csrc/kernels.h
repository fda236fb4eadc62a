// Host-side launch descriptors of the RPLU kernels (shared by dense.cu,
// cauchy.cu, batch.cu and the C-ABI layer).  All pointers are device memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rplu {

struct JobState;

// Optional timing of the per-step hot kernel: CUDA events recorded around each
// launch on the launching stream; read after the call's final synchronisation.
struct HotTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  int64_t launches = 0;       // hot-kernel launches
  int64_t all_launches = 0;   // every kernel launch of the call
  void* impl = nullptr;       // event list (abi.cu)
  void begin();
  void end();
  double elapsed_ms();        // after synchronisation
  void release();
};

// Dense form (Algorithm 1, two-stage draw of Sec. 4.1).
struct DenseLaunch {
  const void* A;      // input, row stride lda; may equal S (in-place init)
  int64_t lda;
  void* S;            // residual, row stride lds (multiple of the 16-byte vector), 16-byte aligned
  int64_t lds;
  int64_t n, m, k;
  double* d;          // n squared row norms
  double* rowmax;     // n, COMPLETE mode only (else null)
  int64_t* rowarg;    // n, COMPLETE mode only
  uint8_t* row_used;  // n, zeroed
  uint8_t* col_used;  // m, zeroed
  void* ublk;         // pivot rows of the current block: blk x lds elements, 16-byte aligned rows
  int32_t blk;        // steps between write-backs of S (1 = every step)
  void* L;            // n x k column-major, zeroed
  void* U;            // k x m row-major
  int64_t* I;         // k
  int64_t* J;         // k
  double* T_hist;     // k + 1
  JobState* st;       // zeroed
  uint64_t seed;
  int32_t mode;       // rplu_pivot
  double tol;
  const int64_t* gI;  // GIVEN mode
  const int64_t* gJ;
  int32_t num_sms;
};

cudaError_t dense_run(int32_t dtype, const DenseLaunch& a, cudaStream_t s, HotTimer* tm);
// The RPLU_PIVOT_RANDOM draw of one step on a cluster of 8 CTAs (sample_cluster.cu).
cudaError_t dense_sample_cluster(int32_t dtype, const DenseLaunch& a, cudaStream_t s);

// Matrix-free Cauchy form (Sec. 5.1 with p = 1; LU-form Algorithm 2 and the
// row-norm update of Sec. 4.1).
struct CauchyLaunch {
  const void* x;      // n points
  const void* y;      // m points
  int64_t n, m, k;
  double* d;          // n
  uint8_t* row_used;  // n, zeroed
  uint8_t* col_used;  // m, zeroed
  void* rhat;         // m residual row (working precision)
  void* urow;         // m masked pivot row (working precision), U(t,:)
  void* chat;         // unused by the current kernels (reserved)
  void* L;            // n x k column-major, zeroed
  void* U;            // k x m row-major, zeroed
  int64_t* I;
  int64_t* J;
  double* T_hist;     // k + 1
  void* vproj;        // k complex FP64: U(s,:) conj(u)
  void* part;         // matvec partial sums: nchunk x n complex FP64
  int32_t nchunk;     // column chunks of the matvec
  JobState* st;
  uint64_t seed;
  int32_t mode;
  double tol;
  const int64_t* gI;
  const int64_t* gJ;
  int32_t num_sms;
  // CUR form (Algorithm 2 as printed; L and U above are null): rows A(I,:) and
  // columns A(:,J) are generated again each step and the core inverse
  // Uc = A(I,J)^{-1} is kept, updated by Eq. block-inverse-update
  cf64* core;         // k x k, leading dimension k: Uc(p, s), p over J positions, s over I positions
  void* lcol;         // n multipliers of the step (working precision)
  cf64* vb;           // k: b^T = A(i,J) Uc
  cf64* ve;           // k: e = Uc A(I,j)
  cf64* vg;           // k: g(I) of the step's matvec
  cf64* vh;           // k: h = Uc g(I)
};

// Cauchy-like form through generators (Sec. 5.1, Algorithm 3 with exact row norms):
// A_pq = sum_l G[p,l] B[l,q] / (x_p - y_q); the residual is carried by G, B.
struct CauchyLikeLaunch {
  const void* x;      // n points
  const void* y;      // m points
  void* G;            // n x p row-major, updated in place
  void* B;            // p x m row-major, updated in place
  int64_t n, m, p, k;
  double* d;          // n exact squared row norms of the residual
  uint8_t* row_used;  // n, zeroed
  uint8_t* col_used;  // m, zeroed
  void* r;            // m: pivot row of the step
  void* gi;           // p: G(i,:) before the update
  void* bj;           // p: B(:,j) before the update
  void* L;            // n x k column-major
  void* U;            // k x m row-major
  int64_t* I;
  int64_t* J;
  double* T_hist;     // k + 1
  double* part;       // nchunk x n row-norm partial sums
  int32_t nchunk;
  JobState* st;
  uint64_t seed;
  int32_t mode;
  double tol;
  const int64_t* gI;
  const int64_t* gJ;
  int32_t num_sms;
  int32_t gate;       // row-norm passes: kGateNone every step, kGateFallback only for a
                      // step whose bound-based proposals were all rejected, kGateForced always
};

enum : int32_t { kGateNone = 0, kGateFallback = 1, kGateForced = 2 };

int32_t cauchy_like_chunks(int64_t n, int64_t m, int32_t dtype, int64_t p, int32_t num_sms);
cudaError_t cauchy_like_run(int32_t dtype, const CauchyLikeLaunch& a, cudaStream_t s, HotTimer* tm);
// Single launches of the exact-norm form's kernels, for the bound-based draw:
// the row-norm pass (norms + reduction, honouring a.gate), the generator
// update of the step drawn, and the final exact total into T_hist[k_done].
cudaError_t cauchy_like_norms(int32_t dtype, const CauchyLikeLaunch& a, cudaStream_t s);
cudaError_t cauchy_like_update(int32_t dtype, const CauchyLikeLaunch& a, cudaStream_t s);
cudaError_t cauchy_like_finish(const CauchyLikeLaunch& a, cudaStream_t s);

// Device copy of the quadtrees and interaction lists of App. C (Algorithm
// C.1) for one factorization, and the per-step buffers of Algorithm C.2.
// Tree positions index the points sorted into tree order (tperm / sperm map
// a position to the original index).  All pointers are device memory.
struct BhLaunch {
  int32_t n_tleaf;          // target leaves
  int32_t n_snode;          // source nodes (node 0 is the root)
  int32_t n_sleaf;          // source leaves
  int32_t tleaf_max;        // most points in one target leaf
  const int32_t* tperm;     // n
  const int32_t* sperm;     // m
  const int2* tleaf;        // n_tleaf: [lo, hi) tree positions of each target leaf
  const int2* snode;        // n_snode: [lo, hi) tree positions of each source node
  const int32_t* sparent;   // n_snode: parent node (-1 for the root)
  const int32_t* sleaf;     // n_sleaf: node ids of the source leaves, in tree order
  int32_t n_sinner;         // internal (non-leaf) source nodes
  const int32_t* sinner;    // n_sinner: their node ids
  const int2* sleafrange;   // n_snode: [lo, hi) range of sleaf under each node
  const int32_t* a_off;     // n_tleaf + 1: aggregated entries of target leaf l
  const int32_t* a_node;    //   source node of each entry
  const double* a_alpha;    //   1 / d_min^2(source node, target leaf)
  const int32_t* e_off;     // n_tleaf + 1: source leaves summed exactly for leaf l
  const int32_t* e_node;
  double* H;                // n_snode x p x p complex FP64 Gram matrices (re, im interleaved)
  int32_t nslice;           // CTAs per target leaf, each summing a share of its exact leaves
  double* u;                // nslice x n partial upper bounds, original row order; the bound
                            // of row p is their sum in slice order
  int32_t* attempts;        // k proposals per step (kMaxAttempts + 1: exact fallback), or null
  int32_t stop_max;         // 1: stop when max(u) <= tol^2 max(u at step 0); 0: sum(u) <= tol^2 T0
  int32_t exact_ends;       // 1: exact row-norm passes before the loop (T0) and after it (T_hist[k_done]);
                            // 0 (CUR-AAA, max rule): neither, T0 and T_hist[k_done] stay 0
  double* umax0;            // max(u) at step 0 (device)
  // graph mode: the step loop is a conditional WHILE node of one CUDA graph and
  // the exact fallback an IF node inside it; the draw kernel sets h_fb, the
  // loop-control kernel h_loop
  int32_t use_graph;
  int64_t* iter;            // loop iterations run (device, zeroed)
  cudaGraphConditionalHandle h_loop;
  cudaGraphConditionalHandle h_fb;
};

// Algorithm 3 with the row draw by rejection against the bounds of App. C.
cudaError_t cauchy_like_bh_run(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s,
                               HotTimer* tm);
// The bounds u of Algorithm C.2 for the current generators, once (no factorization).
cudaError_t cauchy_like_bh_bounds(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s);

int32_t cauchy_chunks(int64_t n, int64_t m, int32_t dtype, int32_t num_sms);
cudaError_t cauchy_run(int32_t dtype, const CauchyLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm);
cudaError_t cauchy_init(int32_t dtype, const CauchyLaunch& a, cudaStream_t s, HotTimer* tm);
cudaError_t cauchy_finish(const CauchyLaunch& a, cudaStream_t s, HotTimer* tm);
// Steps of the CUR form (a.core set, a.L and a.U null).
cudaError_t cauchy_cur_run(int32_t dtype, const CauchyLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm);
// The FP64 core (leading dimension k) into the caller's k x k array (float64 for real
// dtypes, complex128 for complex ones), zero past kd.
cudaError_t cauchy_core_out(int32_t dtype, const cf64* core, int64_t k, int64_t kd, void* out, int num_sms,
                            cudaStream_t s);

// CUR-AAA (Sec. 5.3): the split of the samples and the Loewner generators.
struct AaaLaunch {
  const void* z;            // m complex128 samples
  const void* f;            // m complex128 values
  int64_t m;
  uint64_t seed;
  int32_t num_sms;
  uint8_t* flag;            // m scratch flags
  int32_t* cnt;             // compaction block counts (aaa_compact_blocks(m))
  int64_t* total;           // 1
  int32_t* bad;             // 1, zeroed: set when the split's permutation failed
  int64_t* xidx;            // ceil(m/2): indices of X in z
  int64_t* yidx;            // floor(m/2): indices of Y
  void* x;                  // X points, values
  void* fx;
  void* y;                  // Y points, values
  void* fy;
  void* G;                  // ceil(m/2) x 2 generators
  void* B;                  // 2 x floor(m/2)
  unsigned long long* fmax_bits;  // max |f| as FP64 bits
};

// Buffers of one barycentric fit with k support points.
struct AaaFit {
  int64_t* sup;             // k indices into z
  int64_t* rows;            // m - k non-support sample indices
  void* A;                  // (m - k) x k complex128, column-major (then Householder vectors and R)
  double* part;             // column-norm partial sums (4 x SMs)
  double* s;                // k reflector scales
  void* rdiag;              // k diagonal of R
  double* part2;            // k x row-chunks x 2 partial dot products
  void* sw;                 // k scaled dot products
  void* w;                  // k weights (unit 2-norm)
  void* y;                  // k scratch
  int32_t* iters;           // inverse-iteration count
  unsigned long long* err_bits;  // max |f - r| as FP64 bits
};

// Workspace of a grid-wide exact draw (grid_draw.cuh) over a long weight
// vector: the keys' running maximum (zero between draws), and one exact
// fixed-point total (16 bytes) per chunk of `len` weights.
struct GridDraw {
  unsigned long long* maxb;
  void* part;
  int64_t chunks;
  int64_t len;
};
// chunks of at least 8192 weights, at most 4 per SM
inline void grid_draw_shape(int64_t n, int num_sms, int64_t* chunks, int64_t* len) {
  int64_t c = (n + 8191) / 8192;
  const int64_t cap = (int64_t)num_sms * 4;
  if (c > cap) c = cap;
  if (c < 1) c = 1;
  *len = (n + c - 1) / c;
  if (*len < 1) *len = 1;
  *chunks = (n + *len - 1) / *len;
  if (*chunks < 1) *chunks = 1;
}

// RPLU in CUR form (Algorithm 2) on the multi-level Toeplitz matrix of Sec. 4.2:
// the drifted Gaussian kernel of Eq. kernel on the grid {0, h, ..., (N-1) h}^3,
// A_pq = K(x_p - x_q) = T1 (x) T0 (x) T0 (N x N Toeplitz factors, n = N^3,
// p = (a N + b) N + c).  Real FP64 throughout.
struct Toeplitz3Launch {
  int32_t N;
  int64_t n, k;
  const double* t1;   // 2N - 1 taps: T1[a, a'] = t1[a - a' + N - 1] (the shifted axis)
  const double* t0;   // 2N - 1 taps of the two unshifted axes
  double* r1d;        // 2N: squared row sums of T1, then of T0
  double* d;          // n row norms
  uint8_t* row_used;  // n, zeroed
  uint8_t* col_used;  // n, zeroed
  double* rhat;       // n residual row
  double* urow;       // n masked pivot row u
  double* lcol;       // n multipliers l
  double* g;          // n: A u (uncorrected; k_t3_dupdate subtracts sum_s h_s A(p,J_s) as it generates them)
  double* tmp;        // n: mode-product scratch
  int64_t* I;
  int64_t* J;
  double* T_hist;     // k + 1
  double* core;       // k x k (leading dimension k): A(I,J)^{-1}, double-double high parts
  double* core_lo;    // k x k: its low parts
  double* vb;         // k: b^T = A(i,J) Uc (double-double: vb + vb_lo)
  double* vb_lo;
  double* ve;         // k: e = Uc A(I,j) (double-double: ve + ve_lo)
  double* ve_lo;
  double* vg;         // k: g(I)
  double* vh;         // k: h = Uc g(I)
  JobState* st;       // a_re + a_im: the pivot sigma = A(i,j) - A(i,J) Uc A(I,j) in double-double
  uint64_t seed;
  int32_t mode;
  double tol;
  const int64_t* gI;
  const int64_t* gJ;
  int32_t num_sms;
  GridDraw rdraw;     // the row draw over d (n)
  GridDraw cdraw;     // the column draw over |u|^2 (n)
};
cudaError_t toeplitz3_init(const Toeplitz3Launch& a, cudaStream_t s, HotTimer* tm);
cudaError_t toeplitz3_cur_run(const Toeplitz3Launch& a, cudaStream_t s, int64_t steps, HotTimer* tm);
cudaError_t toeplitz3_finish(const Toeplitz3Launch& a, cudaStream_t s, HotTimer* tm);
// out (k x k) = the leading kd x kd block of the core, zeros elsewhere
cudaError_t toeplitz3_core_out(const double* core, int64_t k, int64_t kd, double* out, int num_sms, cudaStream_t s);
constexpr int32_t kToeplitzMaxN = 640;

// RPLU in CUR form (Algorithm 2) on a sparse matrix (Sec. 4.3) given in CSR,
// with its CSC copy for the columns; real FP64.
struct SparseCurLaunch {
  int64_t n, m, k;
  const int64_t* rp;  // n + 1 row pointers
  const int32_t* ci;  // nnz column indices
  const double* rv;   // nnz values (row order)
  const int64_t* cp;  // m + 1 column pointers
  const int32_t* ri;  // nnz row indices
  const double* cv;   // nnz values (column order)
  double* d;          // n row norms
  uint8_t* row_used;  // n, zeroed
  uint8_t* col_used;  // m, zeroed
  double* rhat;       // m residual row
  double* urow;       // m masked pivot row u
  double* ccol;       // n pivot column A(:,j) (the raw entries; the correction is gathered)
  int32_t* row_piv;   // n: the step at which the row was pivoted, -1 if never
  int32_t* col_piv;   // m: likewise for the columns
  double* lcol;       // n multipliers l
  double* g;          // n: A u (uncorrected; k_sp_dupdate subtracts sum_s h_s A(p,J_s) on the fly)
  int64_t* I;
  int64_t* J;
  double* T_hist;     // k + 1
  double* core;       // k x k (leading dimension k): A(I,J)^{-1}, double-double high parts
  double* core_lo;    // k x k: its low parts
  double* vb;         // k: b^T = A(i,J) Uc (double-double: vb + vb_lo)
  double* vb_lo;
  double* ve;         // k: e = Uc A(I,j) (double-double: ve + ve_lo)
  double* ve_lo;
  double* vg;         // k: g(I)
  double* vh;         // k: h = Uc g(I)
  JobState* st;       // a_re + a_im: the pivot sigma = A(i,j) - A(i,J) Uc A(I,j) in double-double
  uint64_t seed;
  int32_t mode;
  double tol;
  const int64_t* gI;
  const int64_t* gJ;
  int32_t num_sms;
  GridDraw rdraw;     // the row draw over d (n)
  GridDraw cdraw;     // the column draw over |u|^2 (m)
  int32_t row_lanes;          // lanes per short CSR row (segment_lanes in csr.h)
  int32_t col_lanes;          // lanes per short CSC column
  const int32_t* long_rows;   // CSR rows with more than kSpLongDeg entries: a CTA each
  int64_t n_long_rows;
  const int32_t* long_cols;   // likewise for the CSC columns
  int64_t n_long_cols;
};
constexpr int64_t kSpLongDeg = 1024;  // rows and columns longer than this get a whole CTA
cudaError_t sparse_cur_init(const SparseCurLaunch& a, cudaStream_t s, HotTimer* tm);
cudaError_t sparse_cur_run(const SparseCurLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm);
cudaError_t sparse_cur_finish(const SparseCurLaunch& a, cudaStream_t s, HotTimer* tm);

int64_t aaa_compact_blocks(int64_t m);
cudaError_t aaa_split(const AaaLaunch& a, cudaStream_t s);
// Support points z[set[piv[0..k)]], weights by Householder QR of the Loewner
// matrix and inverse iteration on R, and the largest error over the samples.
cudaError_t aaa_fit(const AaaLaunch& a, const int64_t* piv, const int64_t* set, int64_t k, AaaFit& o, cudaStream_t s);
constexpr int64_t kAaaRowChunk = 2048;
// r(zq) of Eq. aaa-barycentric at nq query points.
cudaError_t aaa_query(const void* t, const void* ft, const void* w, int64_t k, const void* zq, int64_t nq, void* rq,
                      int num_sms, cudaStream_t s);

}  // namespace rplu
