// Dense-form RPLU on the device (paper: Algorithm 1, Sec. 1; two-stage pivot
// draw of Sec. 4.1).  The residual S stays in HBM.  Per step t:
//   k_dense_sample  (1 CTA)  T = sum d, stop test, row draw by d, pivot row
//                            S^(t)(i,:), column draw by its squared entries
//                            (pivoted columns masked), U(t,:) = S^(t)(i,:)
//   k_dense_pass_tma (grid)  per row p: l_p = S^(t)(p,j)/a (FP64 division),
//                            L(p,t) = l_p, S^(t+1)(p,:) = S^(t)(p,:) - l_p U(t,:)
//                            (FMA), S^(t+1)(p,j) = 0, d_p = sum_q |S^(t+1)(p,q)|^2
// The pass reads S once per step.  It writes S back only every `blk` steps:
// in between, S in memory is S^(t0) of the block start t0 and each pass
// applies the pending updates of steps t0..t to the values in registers, in
// the same order and with the same fused multiply-adds as a write-back every
// step, so the numbers are identical for every blk.  Rows already pivoted are
// exactly zero and are skipped.
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "sampler.cuh"
#include "tma.cuh"

namespace rplu {
namespace {

constexpr int kUpdThreads = 256;   // init pass
constexpr int kUpdMinBlocks = 4;
constexpr int kMaxBlk = 8;         // largest number of steps between write-backs
constexpr int kSampleThreads = 1024;

template <typename T> struct alignas(16) Vec { T v[Traits<T>::kVec]; };
static_assert(sizeof(Vec<float>) == 16 && sizeof(Vec<cf32>) == 16 && sizeof(Vec<cf64>) == 16, "16-byte vectors");

template <typename T> __device__ __forceinline__ Vec<T> as_vec(float4 r) {
  Vec<T> o;
  memcpy(&o, &r, 16);
  return o;
}
template <typename T> __device__ __forceinline__ float4 as_f4(const Vec<T>& v) {
  float4 r;
  memcpy(&r, &v, 16);
  return r;
}
// S is streamed once per step: evict-first loads and stores keep L1/L2 for the pivot row.
template <typename T> __device__ __forceinline__ Vec<T> ld_stream(const Vec<T>* p) {
  return as_vec<T>(__ldcs(reinterpret_cast<const float4*>(p)));
}
template <typename T> __device__ __forceinline__ void st_stream(Vec<T>* p, const Vec<T>& v) {
  __stcs(reinterpret_cast<float4*>(p), as_f4(v));
}
template <typename T> __device__ __forceinline__ Vec<T> ld_cached(const Vec<T>* p) {
  return as_vec<T>(__ldg(reinterpret_cast<const float4*>(p)));
}

// squared magnitude accumulated in the working precision
__device__ __forceinline__ float sq_acc(float x, float acc) { return fmaf(x, x, acc); }
__device__ __forceinline__ double sq_acc(double x, double acc) { return fma(x, x, acc); }
__device__ __forceinline__ float sq_acc(cf32 x, float acc) { return fmaf(x.im, x.im, fmaf(x.re, x.re, acc)); }
__device__ __forceinline__ double sq_acc(cf64 x, double acc) { return fma(x.im, x.im, fma(x.re, x.re, acc)); }


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void warp_argmax(double& v, int64_t& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double uv = __shfl_xor_sync(0xffffffffu, v, o);
    int64_t ui = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(uv, ui, v, i)) { v = uv; i = ui; }
  }
}

// Rows of this CTA: a contiguous range, so every SM gets the same share.
__device__ __forceinline__ void cta_rows(int64_t n, int64_t& r0, int64_t& r1) {
  const int64_t rpc = (n + gridDim.x - 1) / gridDim.x;
  r0 = (int64_t)blockIdx.x * rpc;
  r1 = min(n, r0 + rpc);
}

// ------------------------------------------------------------------ init
// S = A (unless in place), d_p = sum_q |A_pq|^2, non-finite check, row maxima.
template <typename T, bool kVecA, bool kComplete>
__global__ void __launch_bounds__(kUpdThreads, kUpdMinBlocks) k_dense_init(DenseLaunch a) {
  using real = typename Traits<T>::real;
  constexpr int V = Traits<T>::kVec;
  constexpr int UNR = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t r0, r1;
  cta_rows(a.n, r0, r1);
  const T* A = (const T*)a.A;
  T* S = (T*)a.S;
  const bool copy = (const void*)A != (const void*)S;
  bool bad = false;
  for (int64_t p = r0 + warp; p < r1; p += nw) {
    const T* arow = A + p * a.lda;
    T* srow = S + p * a.lds;
    double dsum = 0.0, rmax = -1.0;
    int64_t rarg = -1;
    int64_t q0 = 0;
    if (kVecA) {
      const int nvec = (int)(a.m / V);
      const Vec<T>* av = (const Vec<T>*)arow;
      Vec<T>* sv = (Vec<T>*)srow;
      for (int v0 = 0; v0 < nvec; v0 += 32 * UNR) {
        Vec<T> x[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int idx = v0 + u * 32 + lane;
          if (idx < nvec) x[u] = ld_stream(av + idx);
        }
        real acc = 0;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int idx = v0 + u * 32 + lane;
          if (idx < nvec) {
#pragma unroll
            for (int e = 0; e < V; ++e) {
              bad |= !finite_v(x[u].v[e]);
              acc = sq_acc(x[u].v[e], acc);
              if (kComplete) {
                const double w = abs2_d(x[u].v[e]);
                if (better(w, (int64_t)idx * V + e, rmax, rarg)) { rmax = w; rarg = (int64_t)idx * V + e; }
              }
            }
            if (copy) st_stream(sv + idx, x[u]);
          }
        }
        dsum += (double)acc;
      }
      q0 = nvec * V;
    }
    for (int64_t q = q0 + lane; q < a.m; q += 32) {
      const T x = arow[q];
      bad |= !finite_v(x);
      dsum += abs2_d(x);
      if (kComplete) {
        const double w = abs2_d(x);
        if (better(w, q, rmax, rarg)) { rmax = w; rarg = q; }
      }
      if (copy) srow[q] = x;
    }
    dsum = warp_sum(dsum);
    if (kComplete) warp_argmax(rmax, rarg);
    if (lane == 0) {
      a.d[p] = dsum;
      if (kComplete) { a.rowmax[p] = rmax; a.rowarg[p] = rarg; }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) {
    atomicOr(&a.st->err, kErrNonFinite);
    a.st->done = 1;
  }
}

// ----------------------------------------------------------------- sample
// One CTA: exact fixed-point draws (sampler.cuh).  Row weights are d; the
// pivot row S^(t)(i,:) is S(i,:) minus the pending updates of the block, with
// pivoted columns masked; it is staged in ublk[r] (r = t - t0) and written to
// U(t,:); column weights are its squared entries.
template <typename T>
__global__ void __launch_bounds__(kSampleThreads) k_dense_sample(DenseLaunch a) {
  __shared__ FxScratch sh;
  __shared__ T Li[kMaxBlk];
  JobState* st = a.st;
  if (st->done) return;
  const int64_t t = st->t;
  const int r = (int)(t % a.blk);
  const int64_t t0 = t - r;
  const T* S = (const T*)a.S;
  const T* Lout = (const T*)a.L;
  const double* d = a.d;
  const uint8_t* col_used = a.col_used;
  uint64_t mb = max_bits_f64(d, a.n);
  mb = block_max_u64(mb, sh);
  const int Er = fx_scale_f64(mb, a.n);
  auto dw = [d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); };
  T* urow = (T*)a.U + t * a.m;
  T* ub = (T*)a.ublk;
  T* rh = ub + (int64_t)r * a.lds;
  int64_t i = -1, j = -1;
  bool ok = false;
  int32_t err = 0;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    u128 Tfx;
    if (a.mode == RPLU_PIVOT_RANDOM) {
      i = fx_block_draw(dw, a.n, draw_u53(a.seed, t, 0, attempt), true, &Tfx, sh);
    } else {
      (void)fx_block_draw(dw, a.n, 0, false, &Tfx, sh);
      if (a.mode == RPLU_PIVOT_C2) {
        i = fx_block_argmax([d](int64_t p) -> uint64_t { return fx_bits64(d[p]); }, a.n, sh);
      } else if (a.mode == RPLU_PIVOT_COMPLETE) {
        const double* rm = a.rowmax;
        i = fx_block_argmax([rm](int64_t p) -> uint64_t { return fx_bits64(rm[p]); }, a.n, sh);
      } else {
        i = a.gI[t];
      }
    }
    const double T_ = fx_to_double(Tfx, Er);
    if (attempt == 0) {
      const double T0 = (t == 0) ? T_ : st->T0;
      if (threadIdx.x == 0) {
        a.T_hist[t] = T_;
        if (t == 0) st->T0 = T_;
      }
      if (!(T_ > 0.0) || (a.tol > 0.0 && T_ <= a.tol * a.tol * T0)) break;
    } else if (!(T_ > 0.0)) {
      break;
    }
    if (a.mode == RPLU_PIVOT_GIVEN && (i < 0 || i >= a.n || a.row_used[i])) {
      err = kErrBadGiven;
      break;
    }
    if (i < 0) break;
    // S^(t)(i,:): the stored row minus the pending updates of steps t0..t-1
    if (threadIdx.x < r) Li[threadIdx.x] = Lout[(t0 + threadIdx.x) * a.n + i];
    __syncthreads();
    const T* srow = S + i * a.lds;
    uint64_t cb = 0;
    // four columns per thread and round, their loads issued before the chains
    constexpr int kU = 4;
    const int64_t st = blockDim.x;
    for (int64_t q0 = threadIdx.x; q0 < a.lds; q0 += kU * st) {
      T x[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t q = q0 + u * st;
        x[u] = q < a.m ? srow[q] : zero_v<T>();
      }
      for (int s = 0; s < r; ++s) {
        T uv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int64_t q = q0 + u * st;
          uv[u] = q < a.lds ? ub[(int64_t)s * a.lds + q] : zero_v<T>();
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) x[u] = fms(x[u], Li[s], uv[u]);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t q = q0 + u * st;
        if (q >= a.lds) break;
        const T v = (q < a.m && !col_used[q]) ? x[u] : zero_v<T>();
        rh[q] = v;
        if (q < a.m) urow[q] = v;
        const uint64_t b = entry_max_bits(v);
        cb = b > cb ? b : cb;
      }
    }
    cb = block_max_u64(cb, sh);  // also orders the staged-row writes before the reads below
    const int Ec = fx_entry_scale<T>(cb, a.m);
    const T* rr = rh;
    auto cw = [rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); };
    u128 Rfx = 1;
    if (a.mode == RPLU_PIVOT_RANDOM) {
      j = fx_block_draw(cw, a.m, draw_u53(a.seed, t, 1, attempt), true, &Rfx, sh);
    } else if (a.mode == RPLU_PIVOT_C2) {
      (void)fx_block_draw(cw, a.m, 0, false, &Rfx, sh);
      j = fx_block_argmax(cw, a.m, sh);
    } else if (a.mode == RPLU_PIVOT_COMPLETE) {
      j = a.rowarg[i];
    } else {
      j = a.gJ[t];
      if (j < 0 || j >= a.m || col_used[j]) {
        err = kErrBadGiven;
        break;
      }
    }
    if (Rfx == 0 || j < 0) {
      if (threadIdx.x == 0) a.d[i] = 0.0;
      __syncthreads();
      continue;
    }
    ok = true;
    break;
  }
  double ar = 0.0, ai = 0.0;
  if (ok) {
    to_d(rh[j], ar, ai);
    if (ar == 0.0 && ai == 0.0) {
      ok = false;
      err = kErrZeroPivot;
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      st->done = 1;
      st->k_done = t;
      if (err) atomicOr(&st->err, err);
    }
    return;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.col_used[j] = 1;
    a.row_used[i] = 1;
    a.I[t] = i;
    a.J[t] = j;
    st->i = i;
    st->j = j;
    st->a_re = ar;
    st->a_im = ai;
    st->cur = t;
    st->t = t + 1;
  }
}

// d = a * b + c on two FP32 lanes at once (one instruction; each lane rounded
// exactly like a scalar fmaf)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// -------------------------------------------------------------- TMA pass
// The same per-step pass, fed by bulk asynchronous copies.  A producer warp
// streams tiles of kTRows rows x kTVec 16-byte vectors of S, each with the
// same columns of the block's pending pivot rows, into a ring of shared-memory
// stages (full/empty mbarriers); kTConsumers warps apply the pending updates:
// thread (cv, half) owns column vectors cv and cv + kTVec/2 of rows
// 4*half .. 4*half+3 of a tile, so each pivot-row vector it loads serves four
// rows.  Tiles go column chunk by column chunk within a row block, row block
// after row block; the pivot-row columns come with every tile (from L2).
// Tiles of 16 rows x 2 KB (half the pivot-row bytes per stage, one stage more
// in the ring) were measured slower at 32768^2: 0.92 against 0.81 ms per
// launch.  Row-norm partials are summed per thread in the working precision
// and across tiles and threads in FP64, in a fixed order.  Every wait is
// bounded (tma.cuh).
// Eight consumer warps, two 16-byte vectors of four rows per thread and tile.
// Sixteen warps with one vector each were measured slower on the FP32 pass
// (0.96 against 0.83 ms per 32768^2 step): a 17-warp CTA caps a thread at 96
// registers (five warps share one scheduler's register file) and the
// deep-block specialisations spill.
constexpr int kTConsumers = 8;
constexpr int kTThreads = (kTConsumers + 1) * 32;
constexpr int kTRows = 8;
constexpr int kTVec = 256;       // 16-byte vectors per row per stage
constexpr int kTPer = 2;         // vectors per consumer thread per row and stage
template <typename T> constexpr int tma_stages() { return sizeof(T) <= 4 ? 3 : 2; }
constexpr int kTMaxRows = 256;  // rows per CTA

// every layout fits the 227 KB of dynamic shared memory a CTA may opt in to
constexpr size_t kMaxDynSmem = 232448;

// One stage: kTRows rows of S, then the pivot rows (kMaxBlk, or exactly kR1 for
// a kernel specialised on kR1 pending updates), kTVec vectors each.  A kernel
// specialised on kR1 sizes its ring to what is left of the shared memory: the
// ring's depth (the S bytes in flight) sets the copy rate of the read-only
// steps (measured at 32768²: two stages instead of three made every step 17 %
// slower), so the steps with few pending updates, whose stages are smaller,
// get deeper rings.
template <typename T, bool kComplete, int kR1 = 0>
struct TmaLayout {
  static constexpr int srows = kTRows + (kR1 > 0 ? kR1 : kMaxBlk);
  static constexpr size_t stage_bytes = (size_t)srows * kTVec * 16;
  static constexpr size_t rest = 6 * 16 + (size_t)kTMaxRows * 4 * 8 * (kComplete ? 3 : 1) +
                                 (size_t)kTMaxRows * kMaxBlk * sizeof(T) + 2 * kMaxBlk * 4 + kTMaxRows + 256 + 16;
  static constexpr int fit = (int)((kMaxDynSmem - rest) / stage_bytes);
  static constexpr size_t buf = 0;
  static constexpr int stages = kR1 > 0 ? (fit < 6 ? fit : 6) : tma_stages<T>();
  static constexpr size_t full = buf + (size_t)stages * stage_bytes;
  static constexpr size_t empty = full + stages * 8;
  static constexpr size_t part = empty + stages * 8;
  static constexpr size_t rmx = part + (size_t)kTMaxRows * 4 * 8;
  static constexpr size_t rag = rmx + (kComplete ? (size_t)kTMaxRows * 4 * 8 : 0);
  static constexpr size_t lsh = rag + (kComplete ? (size_t)kTMaxRows * 4 * 8 : 0);
  static constexpr size_t jvo = lsh + (size_t)kTMaxRows * kMaxBlk * sizeof(T);
  static constexpr size_t act = jvo + 2 * kMaxBlk * 4;
  static constexpr size_t jchk = act + kTMaxRows;  // bit per column chunk holding a pivot column of the block
  static constexpr size_t misc = jchk + 256;
  static constexpr size_t bytes = misc + 16;
};

static_assert(TmaLayout<float, false, 1>::bytes <= kMaxDynSmem && TmaLayout<float, false, 8>::bytes <= kMaxDynSmem &&
                  TmaLayout<float, false, 8>::stages >= 3 &&
              TmaLayout<float, false>::bytes <= kMaxDynSmem && TmaLayout<float, true>::bytes <= kMaxDynSmem &&
                  TmaLayout<double, false>::bytes <= kMaxDynSmem && TmaLayout<double, true>::bytes <= kMaxDynSmem &&
                  TmaLayout<cf32, false>::bytes <= kMaxDynSmem && TmaLayout<cf32, true>::bytes <= kMaxDynSmem &&
                  TmaLayout<cf64, false>::bytes <= kMaxDynSmem && TmaLayout<cf64, true>::bytes <= kMaxDynSmem,
              "pass layout exceeds the shared-memory limit");

// kR1 > 0: the number of updates applied per element (r + 1 = t - t0 + 1) is
// the compile-time constant kR1 (the host picks the instantiation per step, so
// unrolled loops carry no predicated-off iterations); kR1 == 0: read at run time.
template <typename T, bool kComplete, int kR1>
__global__ void __launch_bounds__(kTThreads, 1) k_dense_pass_tma(DenseLaunch a) {
  using real = typename Traits<T>::real;
  using Lay = TmaLayout<T, kComplete, kR1>;
  constexpr int V = Traits<T>::kVec;
  constexpr int kStg = Lay::stages;
  extern __shared__ __align__(128) uint8_t smem[];
  Vec<T>* buf = (Vec<T>*)(smem + Lay::buf);
  uint64_t* full = (uint64_t*)(smem + Lay::full);
  uint64_t* empty = (uint64_t*)(smem + Lay::empty);
  double* part = (double*)(smem + Lay::part);
  double* rmx = (double*)(smem + Lay::rmx);
  int64_t* rag = (int64_t*)(smem + Lay::rag);
  T (*Lsh)[kMaxBlk] = (T (*)[kMaxBlk])(smem + Lay::lsh);
  int* jv = (int*)(smem + Lay::jvo);
  int* je = jv + kMaxBlk;
  uint8_t* act = smem + Lay::act;
  uint32_t* jchk = (uint32_t*)(smem + Lay::jchk);
  volatile int* abort = (volatile int*)(smem + Lay::misc);

  JobState* st = a.st;
  if (st->done) return;
  const int64_t t = st->cur, i = st->i, jt = st->j;
  const int r = kR1 > 0 ? kR1 - 1 : (int)(t % a.blk);
  if (kR1 > 0 && (int)(t % a.blk) != r) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
      atomicOr(&st->err, kErrInternal);
      st->done = 1;
    }
    return;
  }
  const int64_t t0 = t - r;
  const bool write = (r == a.blk - 1) && (t + 1 < a.k);
  const double ar = st->a_re, ai = st->a_im;
  const int64_t r0 = (int64_t)blockIdx.x * a.n / gridDim.x;
  const int64_t r1 = (int64_t)(blockIdx.x + 1) * a.n / gridDim.x;
  const int nrows = (int)(r1 - r0);
  const int nrb = (nrows + kTRows - 1) / kTRows;
  const int nvec = (int)(a.m / V);
  const int nch = (nvec + kTVec - 1) / kTVec;
  const int total = nrb * nch;
  T* S = (T*)a.S;
  T* Lout = (T*)a.L;
  const T* ubs = (const T*)a.ublk;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- prologue: barriers, row flags, multipliers, pivot columns of the block
  if (tid == 0) {
    for (int q = 0; q < kStg; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kTConsumers);
    }
    *abort = 0;
    mbar_fence_init();
  }
  if (tid < 64) jchk[tid] = 0;
  if (tid < kMaxBlk) {
    const int64_t js = tid <= r ? a.J[t0 + tid] : -1;
    jv[tid] = js >= 0 ? (int)(js / V) : -1;
    je[tid] = js >= 0 ? (int)(js % V) : 0;
  }
  __syncthreads();
  if (tid < kMaxBlk && jv[tid] >= 0) {
    const int chk = jv[tid] / kTVec;
    if (chk < 64 * 32) atomicOr(&jchk[chk >> 5], 1u << (chk & 31));
  }
  for (int rl = tid; rl < nrows; rl += kTThreads) {
    const int64_t p = r0 + rl;
    const bool on = !a.row_used[p];
    act[rl] = on;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      part[rl * 4 + w] = 0.0;
      if (kComplete) { rmx[rl * 4 + w] = -1.0; rag[rl * 4 + w] = -1; }
    }
    if (p == i) {
      Lout[t * a.n + i] = one_v<T>();
      a.d[i] = 0.0;
      if (kComplete) { a.rowmax[i] = 0.0; a.rowarg[i] = -1; }
    }
    if (on) {
      T x = S[p * a.lds + jt];
      for (int s = 0; s < r; ++s) {
        const T ls = Lout[(t0 + s) * a.n + p];
        Lsh[rl][s] = ls;
        x = fms(x, ls, ubs[(int64_t)s * a.lds + jt]);
      }
      double xr, xi, lr, li;
      to_d(x, xr, xi);
      cdiv_d(xr, xi, ar, ai, lr, li);
      const T l = from_d<T>(lr, li);
      Lout[t * a.n + p] = l;
      Lsh[rl][r] = l;
    }
  }
  __syncthreads();

  if (warp == kTConsumers) {
    // ---- producer: lane q < kTRows copies row q of the tile, lane kTRows + s2
    // copies pivot row s2; lane 0 first announces the tile's byte count
    int g = 0;
    for (; g < total; ++g) {
      const int sidx = g % kStg;
      bool ok = true;
      if (lane == 0 && g >= kStg) ok = mbar_wait_bounded(&empty[sidx], ((g / kStg) - 1) & 1, abort);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      const int rb = g / nch, ch = g % nch;
      const int vb = ch * kTVec;
      const int nv = min(kTVec, nvec - vb);
      const uint32_t bytes = (uint32_t)nv * 16u;
      const int rl = rb * kTRows + lane;
      const bool srow = lane < kTRows && rl < nrows && act[rl];
      const bool urow = lane >= kTRows && lane - kTRows <= r;
      const unsigned mask = __ballot_sync(0xffffffffu, srow || urow);
      if (lane == 0) mbar_arrive_expect_tx(&full[sidx], (uint32_t)__popc(mask) * bytes);
      __syncwarp();
      Vec<T>* stg = buf + (size_t)sidx * Lay::srows * kTVec;
      if (srow)
        bulk_g2s(stg + (size_t)lane * kTVec, S + (r0 + rl) * a.lds + (int64_t)vb * V, bytes, &full[sidx]);
      if (urow)
        bulk_g2s(stg + (size_t)lane * kTVec, ubs + (int64_t)(lane - kTRows) * a.lds + (int64_t)vb * V, bytes,
                 &full[sidx]);
    }
    if (lane == 0 && *abort) {
      // let every issued copy land before the block exits
      for (int gg = (g > kStg ? g - kStg : 0); gg < g; ++gg) {
        const int sidx = gg % kStg;
        const long long c0 = clock64();
        while (!mbar_try_wait(&full[sidx], (gg / kStg) & 1) && clock64() - c0 < kWaitCycles) {
        }
      }
    }
  } else {
    // ---- consumers: thread (cv, half) owns vectors cv + kTVec/kTPer * e2, e2 < kTPer,
    // of rows 4*half .. 4*half+3 of every tile
    constexpr int kCols = kTVec / kTPer;  // 128 column slots per half
    static_assert(kCols * (kTRows / 4) == kTConsumers * 32 && kTRows + kMaxBlk <= 32, "pass tile geometry");
    const int cv = tid & (kCols - 1);
    const int half = tid / kCols;
    const int w4 = warp & 3;
    int sidx = 0;
    uint32_t ph = 0;
    bool alive = true;
    for (int rb = 0; rb < nrb && alive; ++rb) {
      const int rl0 = rb * kTRows + half * 4;
      unsigned on = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (rl0 + q < nrows && act[rl0 + q]) on |= 1u << q;
      // multipliers of this thread's rows, in registers for the whole row block
      T Lq[4][kMaxBlk];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int s2 = 0; s2 < kMaxBlk; ++s2)
          Lq[q][s2] = (s2 <= r && ((on >> q) & 1u)) ? Lsh[rl0 + q][s2] : zero_v<T>();
      real acc[4];
      float2 acc2[4];     // FP32 fast path: two partial sums per row over 4 tiles
      float mid[4];       // FP32 fast path: sum of those over 8 groups, then FP64
      float2 nL2[4][kMaxBlk];  // FP32 fast path: negated multipliers, duplicated per lane pair
      double dsum[4], bmx[4];
      int64_t bag[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = 0;
        acc2[q] = make_float2(0.f, 0.f);
        mid[q] = 0.f;
        dsum[q] = 0.0;
        bmx[q] = -1.0;
        bag[q] = -1;
        if constexpr (std::is_same<T, float>::value && !kComplete) {
#pragma unroll
          for (int s2 = 0; s2 < kMaxBlk; ++s2) {
            const float nl = -(float)Lq[q][s2];
            nL2[q][s2] = make_float2(nl, nl);
          }
        }
      }
      for (int ch = 0; ch < nch; ++ch) {
        if (!mbar_wait_bounded(&full[sidx], ph, abort)) { alive = false; break; }
        const Vec<T>* stg = buf + (size_t)sidx * Lay::srows * kTVec;
        // chunks past the bitmask's 2048 are always checked for pivot columns
        const bool jtile = ch >= 64 * 32 || ((jchk[ch >> 5] >> (ch & 31)) & 1u);
        if constexpr (std::is_same<T, float>::value && !kComplete) {
          // FP32: float4 tiles, two lanes per instruction (fma.rn.f32x2)
          if (on) {
            const float4* st4 = reinterpret_cast<const float4*>(stg);
#pragma unroll
            for (int e2 = 0; e2 < kTPer; ++e2) {
              const int c = cv + e2 * kCols;
              const int v = ch * kTVec + c;
              if (v < nvec) {
                float4 x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) x[q] = st4[(half * 4 + q) * kTVec + c];
#pragma unroll
                for (int s2 = 0; s2 < kMaxBlk; ++s2) {
                  if (s2 <= r) {
                    const float4 u = st4[(kTRows + s2) * kTVec + c];
                    const float2 ulo = make_float2(u.x, u.y), uhi = make_float2(u.z, u.w);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                      const float2 nl = nL2[q][s2];
                      float2 lo = ffma2(nl, ulo, make_float2(x[q].x, x[q].y));
                      float2 hi = ffma2(nl, uhi, make_float2(x[q].z, x[q].w));
                      x[q] = make_float4(lo.x, lo.y, hi.x, hi.y);
                    }
                  }
                }
                if (jtile) {
                  unsigned zm = 0;
#pragma unroll
                  for (int s2 = 0; s2 < kMaxBlk; ++s2)
                    if (s2 <= r && v == jv[s2]) zm |= 1u << je[s2];
                  if (zm) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                      if (zm & 1u) x[q].x = 0.f;
                      if (zm & 2u) x[q].y = 0.f;
                      if (zm & 4u) x[q].z = 0.f;
                      if (zm & 8u) x[q].w = 0.f;
                    }
                  }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  acc2[q] = ffma2(make_float2(x[q].x, x[q].y), make_float2(x[q].x, x[q].y), acc2[q]);
                  acc2[q] = ffma2(make_float2(x[q].z, x[q].w), make_float2(x[q].z, x[q].w), acc2[q]);
                  if (write && ((on >> q) & 1u))
                    __stcs(reinterpret_cast<float4*>(S + (r0 + rl0 + q) * a.lds) + v, x[q]);
                }
              }
            }
          }
        } else if (on) {
#pragma unroll
          for (int e2 = 0; e2 < kTPer; ++e2) {
            const int c = cv + e2 * kCols;
            const int v = ch * kTVec + c;
            if (v < nvec) {
              Vec<T> x[4];
#pragma unroll
              for (int q = 0; q < 4; ++q)
                x[q] = ((on >> q) & 1u) ? stg[(size_t)(half * 4 + q) * kTVec + c] : Vec<T>{};
#pragma unroll
              for (int s2 = 0; s2 < kMaxBlk; ++s2) {
                if (s2 <= r) {
                  const Vec<T> u = stg[(size_t)(kTRows + s2) * kTVec + c];
#pragma unroll
                  for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < V; ++e) x[q].v[e] = fms(x[q].v[e], Lq[q][s2], u.v[e]);
                }
              }
              if (jtile) {
                unsigned zm = 0;
#pragma unroll
                for (int s2 = 0; s2 < kMaxBlk; ++s2)
                  if (s2 <= r && v == jv[s2]) zm |= 1u << je[s2];
                if (zm) {
#pragma unroll
                  for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < V; ++e)
                      if ((zm >> e) & 1u) x[q].v[e] = zero_v<T>();
                }
              }
#pragma unroll
              for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int e = 0; e < V; ++e) {
                  acc[q] = sq_acc(x[q].v[e], acc[q]);
                  if (kComplete) {
                    const double w = abs2_d(x[q].v[e]);
                    const int64_t col = (int64_t)v * V + e;
                    if (better(w, col, bmx[q], bag[q])) { bmx[q] = w; bag[q] = col; }
                  }
                }
                if (write && ((on >> q) & 1u)) st_stream((Vec<T>*)(S + (r0 + rl0 + q) * a.lds) + v, x[q]);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sidx]);
        if ((ch & 3) == 3) {
          if constexpr (std::is_same<T, float>::value && !kComplete) {
            // FP32 path: FP64 (slow on this GPU) only once per 32 tiles
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              mid[q] += acc2[q].x + acc2[q].y;
              acc2[q] = make_float2(0.f, 0.f);
            }
            if ((ch & 31) == 31) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                dsum[q] += (double)mid[q];
                mid[q] = 0.f;
              }
            }
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              dsum[q] += (double)acc[q];
              acc[q] = 0;
            }
          }
        }
        if (++sidx == kStg) { sidx = 0; ph ^= 1u; }
      }
      if (!alive) break;
      // row partials of this warp: FP64 tree over the lanes
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double ds = dsum[q] + (double)acc[q] + (double)(mid[q] + (acc2[q].x + acc2[q].y));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
        if (kComplete) warp_argmax(bmx[q], bag[q]);
        if (lane == 0 && ((on >> q) & 1u)) {
          part[(rl0 + q) * 4 + w4] = ds;
          if (kComplete) { rmx[(rl0 + q) * 4 + w4] = bmx[q]; rag[(rl0 + q) * 4 + w4] = bag[q]; }
        }
      }
    }
    named_sync(1, kTConsumers * 32);
    // ---- epilogue: ragged tail (m not a multiple of the vector width), row norms
    for (int rl = tid; rl < nrows; rl += kTConsumers * 32) {
      if (!act[rl]) continue;
      const int64_t p = r0 + rl;
      double ds = ((part[rl * 4] + part[rl * 4 + 1]) + part[rl * 4 + 2]) + part[rl * 4 + 3];
      double mx = -1.0;
      int64_t mg = -1;
      if (kComplete) {
        for (int w = 0; w < 4; ++w)
          if (better(rmx[rl * 4 + w], rag[rl * 4 + w], mx, mg)) { mx = rmx[rl * 4 + w]; mg = rag[rl * 4 + w]; }
      }
      for (int64_t c = (int64_t)nvec * V; c < a.m; ++c) {
        T xv = S[p * a.lds + c];
        for (int s = 0; s <= r; ++s) xv = fms(xv, Lsh[rl][s], ubs[(int64_t)s * a.lds + c]);
        for (int s = 0; s <= r; ++s)
          if (c == (int64_t)jv[s] * V + je[s]) xv = zero_v<T>();
        ds += abs2_d(xv);
        if (kComplete && better(abs2_d(xv), c, mx, mg)) { mx = abs2_d(xv); mg = c; }
        if (write) S[p * a.lds + c] = xv;
      }
      a.d[p] = ds;
      if (kComplete) { a.rowmax[p] = mx; a.rowarg[p] = mg; }
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) {
    atomicOr(&st->err, kErrTimeout);
    st->done = 1;
    st->k_done = t;
  }
}

// ----------------------------------------------------------------- finish
__global__ void __launch_bounds__(kSampleThreads) k_dense_finish(const double* d, int64_t n, double* T_hist,
                                                               JobState* st) {
  __shared__ FxScratch sh;
  const double T = fx_total_f64(d, n, sh);
  if (threadIdx.x == 0) {
    if (!st->done) {
      st->done = 1;
      st->k_done = st->t;
    }
    T_hist[st->k_done] = T;
    if (st->k_done == 0 && st->t == 0) st->T0 = T;
  }
}

// The pass kernels need more than 48 KB of dynamic shared memory, an opt-in
// that cudaFuncSetAttribute records for the current device only.  Each
// device gets it once (a flag per device and element type); the mutex keeps
// concurrent callers (a session's worker threads, user threads on several
// GPUs) from racing on the table.
template <typename T>
cudaError_t set_pass_attrs() {
  static std::mutex mu;
  static std::vector<char> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)done.size() <= dev) done.resize(dev + 1, 0);
  if (done[dev]) return cudaSuccess;
  const int nb = (int)TmaLayout<T, false>::bytes, cb = (int)TmaLayout<T, true>::bytes;
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 0>, at, nb)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, true, 0>, at, cb)) != cudaSuccess) return e;
  if (std::is_same<T, float>::value) {
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 1>, at, (int)TmaLayout<T, false, 1>::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 2>, at, (int)TmaLayout<T, false, 2>::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 3>, at, (int)TmaLayout<T, false, 3>::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 4>, at, (int)TmaLayout<T, false, 4>::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 5>, at, (int)TmaLayout<T, false, 5>::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 6>, at, (int)TmaLayout<T, false, 6>::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 7>, at, (int)TmaLayout<T, false, 7>::bytes)) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_dense_pass_tma<T, false, 8>, at, (int)TmaLayout<T, false, 8>::bytes)) != cudaSuccess)
      return e;
  }
  done[dev] = 1;
  return cudaSuccess;
}

template <typename T>
cudaError_t dense_run_t(const DenseLaunch& a, cudaStream_t s, HotTimer* tm) {
  constexpr int V = Traits<T>::kVec;
  const bool complete = a.mode == RPLU_PIVOT_COMPLETE;
  const int64_t warps = kUpdThreads / 32;
  int64_t grid = (a.n + warps - 1) / warps;
  const int64_t cap = (int64_t)a.num_sms * kUpdMinBlocks;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  const bool vecA = ((uintptr_t)a.A % 16 == 0) && ((a.lda * (int64_t)sizeof(T)) % 16 == 0) && a.m >= V;
  if (a.n > 0 && a.m > 0) {
    if (vecA) {
      if (complete) k_dense_init<T, true, true><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
      else k_dense_init<T, true, false><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
    } else {
      if (complete) k_dense_init<T, false, true><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
      else k_dense_init<T, false, false><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
    }
    tm->all_launches += 1;
  }
  // per-step pass: TMA-fed, contiguous row ranges of at most kTMaxRows rows
  const size_t smem = complete ? TmaLayout<T, true>::bytes : TmaLayout<T, false>::bytes;
  // FP32 without complete pivoting runs a kernel specialised on r + 1
  constexpr bool kSpec = std::is_same<T, float>::value;
  {
    cudaError_t e = set_pass_attrs<T>();
    if (e != cudaSuccess) return e;
  }
  int per_sm = 1;
  if (complete) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_pass_tma<T, true, 0>, kTThreads, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_pass_tma<T, false, 0>, kTThreads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t pgrid = (int64_t)a.num_sms * per_sm;
  const int64_t need = (a.n + kTMaxRows - 1) / kTMaxRows;
  if (pgrid < need) pgrid = need;
  if (pgrid > a.n) pgrid = a.n > 0 ? a.n : 1;
  const dim3 g((unsigned)pgrid);
  for (int64_t t = 0; t < a.k; ++t) {
    if (a.mode == RPLU_PIVOT_RANDOM) {
      const int32_t dt = std::is_same<T, float>::value ? RPLU_F32 : std::is_same<T, double>::value ? RPLU_F64
                         : std::is_same<T, cf32>::value ? RPLU_C64 : RPLU_C128;
      cudaError_t e = dense_sample_cluster(dt, a, s);
      if (e != cudaSuccess) return e;
    } else {
      k_dense_sample<T><<<1, kSampleThreads, 0, s>>>(a);
    }
    tm->begin();
    if (complete) {
      k_dense_pass_tma<T, true, 0><<<g, kTThreads, smem, s>>>(a);
    } else if (kSpec) {
      // the host knows r = t mod blk: the device draws every step, so t is the step index
      switch ((int)(t % a.blk) + 1) {
        case 1: k_dense_pass_tma<T, false, 1><<<g, kTThreads, TmaLayout<T, false, 1>::bytes, s>>>(a); break;
        case 2: k_dense_pass_tma<T, false, 2><<<g, kTThreads, TmaLayout<T, false, 2>::bytes, s>>>(a); break;
        case 3: k_dense_pass_tma<T, false, 3><<<g, kTThreads, TmaLayout<T, false, 3>::bytes, s>>>(a); break;
        case 4: k_dense_pass_tma<T, false, 4><<<g, kTThreads, TmaLayout<T, false, 4>::bytes, s>>>(a); break;
        case 5: k_dense_pass_tma<T, false, 5><<<g, kTThreads, TmaLayout<T, false, 5>::bytes, s>>>(a); break;
        case 6: k_dense_pass_tma<T, false, 6><<<g, kTThreads, TmaLayout<T, false, 6>::bytes, s>>>(a); break;
        case 7: k_dense_pass_tma<T, false, 7><<<g, kTThreads, TmaLayout<T, false, 7>::bytes, s>>>(a); break;
        default: k_dense_pass_tma<T, false, 8><<<g, kTThreads, TmaLayout<T, false, 8>::bytes, s>>>(a); break;
      }
    } else {
      k_dense_pass_tma<T, false, 0><<<g, kTThreads, smem, s>>>(a);
    }
    tm->end();
    tm->all_launches += 2;
  }
  k_dense_finish<<<1, kSampleThreads, 0, s>>>(a.d, a.n, a.T_hist, a.st);
  tm->all_launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t dense_run(int32_t dtype, const DenseLaunch& a, cudaStream_t s, HotTimer* tm) {
  switch (dtype) {
    case RPLU_F32: return dense_run_t<float>(a, s, tm);
    case RPLU_F64: return dense_run_t<double>(a, s, tm);
    case RPLU_C64: return dense_run_t<cf32>(a, s, tm);
    case RPLU_C128: return dense_run_t<cf64>(a, s, tm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rplu
