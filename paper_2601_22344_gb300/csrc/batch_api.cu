// Host side of rplu_batch and of the batch plan (include/rplu.h): argument
// checks, staging of host buffers, job ordering, workspace, launch-shape
// choice (fixed default or measured autotuning), CUDA-graph capture of the
// persistent launch, and per-job results.  All arithmetic runs in k_batch
// (batch.cu) or, for jobs too large for it, in the single-job kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "rplu.h"

namespace rplu {
namespace {

// Jobs with n or m above this run through rplu_dense one at a time (rplu_batch)
// or are rejected (plans): the per-job shared-memory state grows with n + m.
constexpr int64_t kBatchMaxDim = 4096;
constexpr int kDefaultThreads = 256, kDefaultRows = 8, kDefaultBlk = 6;

int64_t elem_bytes(int32_t dt) { return dt == RPLU_F32 ? 4 : dt == RPLU_F64 ? 8 : dt == RPLU_C64 ? 8 : -1; }
int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

__device__ __forceinline__ float cauchy_entry(float x, float y) { return 1.0f / (x - y); }
__device__ __forceinline__ double cauchy_entry(double x, double y) { return 1.0 / (x - y); }
// complex64: conj(z) / |z|^2 with the correctly rounded reciprocal of |z|^2, as the kernels generate it
__device__ __forceinline__ cf32 cauchy_entry(cf32 x, cf32 y) {
  const float zr = __fsub_rn(x.re, y.re), zi = __fsub_rn(x.im, y.im);
  const float inv = __frcp_rn(fmaf(zr, zr, zi * zi));
  return cf32{zr * inv, -zi * inv};
}

template <typename T>
__global__ void k_materialise_cauchy(const T* x, const T* y, int64_t n, int64_t m, T* A) {
  const int64_t total = n * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / m, q = e - p * m;
    A[e] = cauchy_entry(x[p], y[q]);
  }
}

// Basic validity of one job (pointers, sizes, type); message on failure.
const char* job_invalid(const rplu_job& jb) {
  if (jb.kind != 0 && jb.kind != 1) return "job kind must be 0 (dense) or 1 (Cauchy)";
  if (jb.dtype != RPLU_F32 && jb.dtype != RPLU_F64 && jb.dtype != RPLU_C64)
    return "batch jobs must be RPLU_F32, RPLU_F64 or RPLU_C64";
  if (jb.n < 0 || jb.m < 0 || jb.k_max < 0) return "negative size";
  if (jb.k_max > std::min(jb.n, jb.m)) return "k_max exceeds min(n, m)";
  if (!(jb.rel_tol >= 0.0) || !std::isfinite(jb.rel_tol)) return "rel_tol must be finite and >= 0";
  if (jb.kind == 0 && jb.n * jb.m > 0 && !jb.A) return "dense job without A";
  if (jb.kind == 0 && jb.lda != 0 && jb.lda < jb.m) return "lda < m";
  if (jb.kind == 1 && ((jb.n > 0 && !jb.x) || (jb.m > 0 && !jb.y))) return "Cauchy job without points";
  if (jb.k_max > 0 && (!jb.I || !jb.J || !jb.L || !jb.U)) return "NULL output with k_max > 0";
  if (jb.memory < 0 || jb.memory > 3)
    return "memory must be 0 (query), 1 (host), 2 (device) or 3 (host, accessed in place)";
  return nullptr;
}

int64_t lda_of(const rplu_job& jb) { return jb.kind == 0 ? (jb.lda ? jb.lda : jb.m) : jb.m; }
bool rows_aligned(const void* A, int64_t lda, int64_t w) { return (uintptr_t)A % 16 == 0 && (lda * w) % 16 == 0; }

bool fits_kernel(const rplu_job& jb) { return jb.n <= kBatchMaxDim && jb.m <= kBatchMaxDim; }

void finish_job(rplu_job& jb, const BatchDesc& d) {
  jb.k_done = d.k_done;
  jb.rel_res = d.T0 > 0.0 ? std::sqrt(std::max(d.T_final, 0.0) / d.T0) : 0.0;
  if (d.err) {
    jb.status = RPLU_ERR_INVALID;
    jb.rel_res = NAN;
  } else if (jb.rel_tol > 0.0 && d.k_done == jb.k_max && jb.k_max > 0 &&
             d.T_final > jb.rel_tol * jb.rel_tol * d.T0) {
    jb.status = RPLU_NOT_CONVERGED;
  } else {
    jb.status = RPLU_OK;
  }
}

// Jobs of one type in one persistent launch.
struct Group {
  int32_t dtype = RPLU_F32;
  std::vector<int32_t> idx;     // caller's job indices
  std::vector<BatchDesc> desc;  // as sent to the device
  std::vector<int32_t> order;   // visiting order, largest first
  int64_t n_max = 0, lds_max = 0;  // dense jobs
  int64_t gn_max = 0, gm_max = 0;  // Cauchy jobs (generator form)
  int64_t s_bytes = 0;          // workspace for jobs that may outlive one block
  BatchDesc* d_desc = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_counter = nullptr;
  char* d_S = nullptr;
  BatchArgs args{};
  BatchShape shape{kDefaultThreads, kDefaultRows, 1};
  double tuned_ms = 0.0;
};

int max_dyn_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Layout of a group once its descriptors (inputs/outputs) are filled: order,
// sizes, and the workspace each job needs for write-back interval blk_min.
void plan_group(Group& g, int blk_min) {
  const int64_t w = elem_bytes(g.dtype), V = 16 / w;
  g.n_max = g.gn_max = 1;
  g.lds_max = g.gm_max = V;
  g.s_bytes = 0;
  for (auto& d : g.desc) {
    d.lds = std::max<int64_t>(align_up(d.m, V), V);
    if (d.kind == 0) {
      g.n_max = std::max(g.n_max, d.n);
      g.lds_max = std::max(g.lds_max, d.lds);
    } else {
      g.gn_max = std::max(g.gn_max, d.n);
      g.gm_max = std::max(g.gm_max, d.lds);
    }
    d.S = nullptr;
    if (d.kind == 0 && d.k_max > blk_min) {  // Cauchy jobs (generator form) keep no residual
      d.S = (void*)(intptr_t)(g.s_bytes + 1);  // offset + 1, resolved when the arena exists
      g.s_bytes += align_up(d.n * d.lds * w, 256);
    }
  }
  g.order.resize(g.desc.size());
  std::iota(g.order.begin(), g.order.end(), 0);
  std::stable_sort(g.order.begin(), g.order.end(), [&](int32_t a, int32_t b) {
    return g.desc[a].n * g.desc[a].m > g.desc[b].n * g.desc[b].m;
  });
}

void resolve_workspace(Group& g) {
  for (auto& d : g.desc)
    if (d.S) d.S = g.d_S + ((intptr_t)d.S - 1);
}

// Largest write-back interval <= want whose shared memory fits one CTA.
int32_t group_kinds(const Group& g) {
  int32_t k = 0;
  for (const auto& d : g.desc) k |= d.kind == 1 ? kKindCauchy : kKindDense;
  return k;
}

// The group's layout sizes with write-back interval blk, as the kernel sees them.
BatchArgs dims_of(const Group& g, int blk) {
  BatchArgs a{};
  a.n_max = g.n_max;
  a.lds_max = g.lds_max;
  a.gn_max = g.gn_max;
  a.gm_max = g.gm_max;
  a.blk = blk;
  a.kinds = group_kinds(g);
  return a;
}

int fit_blk(const Group& g, int want) {
  const int lim = max_dyn_smem();
  for (int b = want; b >= 1; --b)
    if (batch_smem_bytes(g.dtype, dims_of(g, b)) <= lim) return b;
  return 0;
}

cudaError_t set_shape(Group& g, int threads, int rows, int blk, int ctas_per_sm, int sms, int* occ_out) {
  const int64_t smem = batch_smem_bytes(g.dtype, dims_of(g, blk));
  int occ = 0;
  cudaError_t e = batch_occupancy(g.dtype, threads, rows, smem, &occ);
  if (e != cudaSuccess) return e;
  if (occ_out) *occ_out = occ;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int cps = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  g.shape.threads = threads;
  g.shape.rows = rows;
  g.shape.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * cps, (int64_t)g.desc.size()));
  g.args.blk = blk;
  return cudaSuccess;
}

cudaError_t enqueue_group(Group& g, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(g.d_counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  return batch_launch(g.dtype, g.args, g.shape, s);
}

void fill_args(Group& g, int32_t mode) {
  g.args.jobs = g.d_desc;
  g.args.order = g.d_order;
  g.args.njobs = (int32_t)g.desc.size();
  g.args.counter = g.d_counter;
  g.args.mode = mode;
  g.args.n_max = g.n_max;
  g.args.lds_max = g.lds_max;
  g.args.gn_max = g.gn_max;
  g.args.gm_max = g.gm_max;
  g.args.kinds = group_kinds(g);
}

// Measured autotuning: every candidate shape runs the whole group once (the
// results do not depend on the shape); the fastest is kept.
cudaError_t tune_group(Group& g, int sms, cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  int best_t = kDefaultThreads, best_r = kDefaultRows, best_b = 0, best_c = 0;
  float best = 1e30f;
  const int threads_c[2] = {128, 256};
  const int rows_c[2] = {4, 8};
  const int blk_c[3] = {4, 6, 8};
  for (int bi = 0; bi < 3 && e == cudaSuccess; ++bi) {
    const int blk = fit_blk(g, blk_c[bi]);
    if (blk != blk_c[bi]) continue;
    for (int ti = 0; ti < 2 && e == cudaSuccess; ++ti)
      for (int ri = 0; ri < 2 && e == cudaSuccess; ++ri) {
        int occ = 0;
        e = set_shape(g, threads_c[ti], rows_c[ri], blk, 0, sms, &occ);
        // shapes without a compiled kernel for this type, or that do not fit, are skipped
        if (e == cudaErrorInvalidConfiguration || e == cudaErrorInvalidValue) {
          (void)cudaGetLastError();
          e = cudaSuccess;
          continue;
        }
        for (int cps = 1; cps <= std::min(occ, 4) && e == cudaSuccess; ++cps) {
          e = set_shape(g, threads_c[ti], rows_c[ri], blk, cps, sms, nullptr);
          if (e != cudaSuccess) break;
          e = enqueue_group(g, s);  // warm
          if (e == cudaSuccess) e = cudaEventRecord(e0, s);
          if (e == cudaSuccess) e = enqueue_group(g, s);
          if (e == cudaSuccess) e = cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e == cudaSuccess && ms < best) {
            best = ms;
            best_t = threads_c[ti]; best_r = rows_c[ri]; best_b = blk; best_c = cps;
          }
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  if (best_b == 0) return cudaErrorInvalidConfiguration;
  g.tuned_ms = best;
  return set_shape(g, best_t, best_r, best_b, best_c, sms, nullptr);
}

// ------------------------------------------------------------ one-shot path

// Stream-ordered device memory of the one-shot path comes from one pool per
// device that keeps up to kPoolKeep bytes reserved after they are freed, so
// that calls in a row do not map the staging of a large batch again.
constexpr uint64_t kPoolKeep = (uint64_t)8 << 30;

cudaError_t staging_pool(cudaMemPool_t* out) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeep;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    pools[dev] = pool;
  }
  *out = pools[dev];
  return cudaSuccess;
}

struct Arena {
  cudaStream_t s;
  cudaMemPool_t pool = nullptr;
  std::vector<void*> ptrs;
  explicit Arena(cudaStream_t st) : s(st) {}
  ~Arena() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  cudaError_t alloc(void** p, int64_t bytes) {
    *p = nullptr;
    if (bytes <= 0) return cudaSuccess;
    if (!pool) {
      cudaError_t e = staging_pool(&pool);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, (size_t)bytes, pool, s);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

// Host-to-host copies of many pieces; large totals are split over a few
// threads by bytes (a piece is never split).
struct HostCopy {
  void* dst;
  const void* src;
  int64_t bytes;
};
void host_copies(const std::vector<HostCopy>& v) {
  int64_t total = 0;
  for (const HostCopy& c : v) total += c.bytes;
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t by_size = 1 + total / ((int64_t)8 << 20);
  const int nt = (int)std::min<int64_t>(std::min<int64_t>(8, hw > 0 ? hw : 1), by_size);
  auto run = [&v](size_t a, size_t b) {
    for (size_t q = a; q < b; ++q) std::memcpy(v[q].dst, v[q].src, (size_t)v[q].bytes);
  };
  if (nt <= 1) {
    run(0, v.size());
    return;
  }
  std::vector<size_t> cut(nt + 1, v.size());
  cut[0] = 0;
  int64_t acc = 0;
  int k = 1;
  for (size_t q = 0; q < v.size() && k < nt; ++q) {
    acc += v[q].bytes;
    if (acc >= total * k / nt) cut[k++] = q + 1;
  }
  std::vector<std::thread> th;
  for (int q = 1; q < nt; ++q) th.emplace_back(run, cut[q], cut[q + 1]);
  run(cut[0], cut[1]);
  for (std::thread& t : th) t.join();
}

// Staged copies of a job's host buffers.
struct Staged {
  bool in_host = false, out_host = false, in_stage = false;
  bool direct = false;  // host buffers read and written in place by the device (no pinned staging)
  int64_t off_in = 0, off_out = 0;
};

// Pinned host memory for the bulk copies of host-resident jobs, kept across
// calls (grow-only).  A call holds `mu` while it uses the buffers, so calls
// that stage host buffers run one at a time.
struct PinnedStage {
  std::mutex mu;
  void* in = nullptr;
  void* out = nullptr;
  size_t in_cap = 0, out_cap = 0;
  static cudaError_t grow(void** p, size_t* cap, size_t bytes) {
    if (bytes <= *cap) return cudaSuccess;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaHostAlloc(p, want, cudaHostAllocPortable);
    if (e == cudaSuccess) *cap = want;
    return e;
  }
};
PinnedStage g_pinned;

// One contiguous piece to copy: `bytes` from src to dst.  Either end is device
// memory or, on a device that accesses pageable host memory in place, host
// memory.
struct CopySeg {
  unsigned char* dst;
  const unsigned char* src;
  int64_t bytes;
};

// Copies the pieces (one CTA per piece at a time; 16-byte copies where source
// and destination allow, 4-byte ones for the rest: every piece is a whole
// number of 4-byte elements).  Gathers the results into one packed buffer,
// and moves host jobs' points in and factors out where the device reaches
// their host memory.
__global__ void k_copy_segs(const CopySeg* segs, int64_t nseg) {
  for (int64_t k = blockIdx.x; k < nseg; k += gridDim.x) {
    const CopySeg g = segs[k];
    unsigned char* d = g.dst;
    int64_t head = 0;
    if ((((uintptr_t)g.src | (uintptr_t)d) & 15) == 0) {
      head = g.bytes / 16 * 16;
      const float4* s4 = reinterpret_cast<const float4*>(g.src);
      float4* d4 = reinterpret_cast<float4*>(d);
      for (int64_t e = threadIdx.x; e < head / 16; e += blockDim.x) d4[e] = s4[e];
    }
    const uint32_t* s1 = reinterpret_cast<const uint32_t*>(g.src + head);
    uint32_t* d1 = reinterpret_cast<uint32_t*>(d + head);
    for (int64_t e = threadIdx.x; e < (g.bytes - head) / 4; e += blockDim.x) d1[e] = s1[e];
  }
}

// Enqueues k_copy_segs over `segs` (the list itself copied to workspace from `ar`).
cudaError_t copy_segs(Arena& ar, const std::vector<CopySeg>& segs, int sms, cudaStream_t s) {
  if (segs.empty()) return cudaSuccess;
  CopySeg* d = nullptr;
  if (ar.alloc((void**)&d, (int64_t)(segs.size() * sizeof(CopySeg))) != cudaSuccess) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemcpyAsync(d, segs.data(), segs.size() * sizeof(CopySeg), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)std::min<size_t>(segs.size(), (size_t)sms * 8);
  k_copy_segs<<<g, 256, 0, s>>>(d, (int64_t)segs.size());
  return cudaGetLastError();
}

// Jobs too large for the persistent kernel: one rplu_dense call each.
rplu_status run_single(rplu_job& jb, const rplu_opts& o, cudaStream_t s) {
  const int64_t w = elem_bytes(jb.dtype);
  void* A = nullptr;
  rplu_status st = RPLU_OK;
  if (jb.kind == 1) {
    const bool dev = host_on_device(jb.x);
    const void* xd = jb.x;
    const void* yd = jb.y;
    void* xs = nullptr;
    void* ys = nullptr;
    if (cudaMallocAsync(&A, (size_t)(jb.n * jb.m * w + 16), s) != cudaSuccess) return RPLU_ERR_NOMEM;
    if (!dev) {
      if (cudaMallocAsync(&xs, (size_t)(jb.n * w + 16), s) != cudaSuccess ||
          cudaMallocAsync(&ys, (size_t)(jb.m * w + 16), s) != cudaSuccess) {
        if (xs) cudaFreeAsync(xs, s);
        cudaFreeAsync(A, s);
        return RPLU_ERR_NOMEM;
      }
      cudaMemcpyAsync(xs, jb.x, jb.n * w, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(ys, jb.y, jb.m * w, cudaMemcpyHostToDevice, s);
      xd = xs;
      yd = ys;
    }
    const int64_t blocks = (jb.n * jb.m + 255) / 256;
    const unsigned gsz = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, 4096));
    if (jb.dtype == RPLU_F32)
      k_materialise_cauchy<float><<<gsz, 256, 0, s>>>((const float*)xd, (const float*)yd, jb.n, jb.m, (float*)A);
    else if (jb.dtype == RPLU_C64)
      k_materialise_cauchy<cf32><<<gsz, 256, 0, s>>>((const cf32*)xd, (const cf32*)yd, jb.n, jb.m, (cf32*)A);
    else
      k_materialise_cauchy<double><<<gsz, 256, 0, s>>>((const double*)xd, (const double*)yd, jb.n, jb.m, (double*)A);
    if (xs) cudaFreeAsync(xs, s);
    if (ys) cudaFreeAsync(ys, s);
  }
  rplu_opts jo = o;
  jo.dtype = jb.dtype;
  jo.rel_tol = jb.rel_tol;
  jo.lda = jb.kind == 1 ? jb.m : jb.lda;
  jo.overwrite_input = jb.kind == 1;
  std::vector<double> T(jb.k_max + 1, 0.0);
  jo.T_hist = T.data();
  jo.prof = nullptr;
  int64_t kd = 0;
  st = rplu_dense(jb.kind == 1 ? A : jb.A, jb.n, jb.m, jb.k_max, jb.seed, &jo, jb.I, jb.J, jb.L, jb.U, &kd);
  jb.k_done = kd;
  if (st == RPLU_OK || st == RPLU_NOT_CONVERGED) jb.rel_res = T[0] > 0 ? std::sqrt(T[kd] / T[0]) : 0.0;
  if (A) cudaFreeAsync(A, s);
  return st;
}

}  // namespace
}  // namespace rplu

using namespace rplu;

struct PlanCopy {
  void* dst;
  int64_t dpitch;
  const void* src;
  int64_t spitch, width, height;
};

struct rplu_batch_plan {
  rplu_job* jobs = nullptr;
  std::vector<PlanCopy> copies;  // misaligned dense inputs -> aligned plan buffers
  int32_t njobs = 0;
  std::vector<Group> groups;
  std::vector<void*> dev_allocs;
  BatchDesc* h_mirror = nullptr;  // pinned; the descriptors after each run, group after group
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t last = nullptr;
  bool ran = false;
};

namespace {

void plan_free(rplu_batch_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) {
    cudaStreamSynchronize(p->cap);
    cudaStreamDestroy(p->cap);
  }
  for (void* q : p->dev_allocs) cudaFree(q);
  if (p->h_mirror) cudaFreeHost(p->h_mirror);
  delete p;
}

// The group holding the most jobs (the one the shape query reports).
const Group* main_group(const rplu_batch_plan* p) {
  const Group* best = nullptr;
  for (const auto& g : p->groups)
    if (!best || g.desc.size() > best->desc.size()) best = &g;
  return best;
}

}  // namespace

extern "C" {

rplu_status rplu_batch(rplu_job* jobs, int32_t njobs, const rplu_opts* opts) {
  rplu_opts o;
  if (opts) o = *opts;
  else rplu_opts_init(&o);
  if (njobs < 0 || (njobs > 0 && !jobs)) return host_fail(RPLU_ERR_INVALID, "bad job array");
  if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2)
    return host_fail(RPLU_ERR_INVALID, "rplu_batch supports RPLU_PIVOT_RANDOM and RPLU_PIVOT_C2");
  if (njobs == 0) return RPLU_OK;
  cudaStream_t s = (cudaStream_t)o.stream;
  int sms = 0;
  cudaError_t ce = host_num_sms(&sms);
  bool pageable = false;
  if (ce == cudaSuccess) ce = host_pageable_access(&pageable);
  if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));

  Group groups[3];
  groups[0].dtype = RPLU_F32;
  groups[1].dtype = RPLU_F64;
  groups[2].dtype = RPLU_C64;
  std::vector<int32_t> single;
  std::vector<Staged> stg(njobs);
  int64_t stage_bytes = 0, out_bytes = 0;  // the input region first, the output region after it
  bool any_host_in = false, any_host_out = false;
  for (int32_t b = 0; b < njobs; ++b) {
    rplu_job& jb = jobs[b];
    jb.k_done = 0;
    jb.rel_res = NAN;
    jb.status = RPLU_OK;
    if (const char* why = job_invalid(jb)) {
      jb.status = RPLU_ERR_INVALID;
      host_fail(RPLU_ERR_INVALID, why);
      continue;
    }
    if (!fits_kernel(jb)) {
      single.push_back(b);
      continue;
    }
    const int64_t w = elem_bytes(jb.dtype);
    Staged& sg = stg[b];
    const void* in0 = jb.kind == 0 ? jb.A : jb.x;
    const bool host = jb.memory == 1 || jb.memory == 3;
    sg.in_host = jb.n * jb.m > 0 && (host || (jb.memory == 0 && !host_on_device(in0)));
    sg.out_host = jb.k_max > 0 && (host || (jb.memory == 0 && !host_on_device(jb.L)));
    sg.direct = jb.memory == 3 && pageable;
    // dense inputs are read with 16-byte vector loads: host or misaligned rows are staged
    sg.in_stage = sg.in_host || (jb.kind == 0 && jb.n * jb.m > 0 && !rows_aligned(jb.A, lda_of(jb), w));
    if (sg.in_stage) {
      sg.off_in = stage_bytes;
      stage_bytes += jb.kind == 0 ? align_up(jb.n * align_up(jb.m, 16 / w) * w, 256)
                                  : align_up(jb.n * w, 256) + align_up(jb.m * w, 256);
      any_host_in |= sg.in_host && !sg.direct;
    }
    if (sg.out_host) {
      sg.off_out = out_bytes;
      out_bytes += 2 * align_up(jb.k_max * 8, 256) + align_up(jb.n * jb.k_max * w, 256) +
                   align_up(jb.k_max * jb.m * w, 256);
      any_host_out |= !sg.direct;
    }
    groups[jb.dtype == RPLU_F32 ? 0 : jb.dtype == RPLU_F64 ? 1 : 2].idx.push_back(b);
  }

  rplu_status worst = RPLU_OK;
  auto note = [&worst](rplu_status st) {
    if (st != RPLU_OK && (worst == RPLU_OK || worst == RPLU_NOT_CONVERGED)) worst = st;
  };
  // host-resident jobs use the pinned buffers: one copy in, one copy out
  std::unique_lock<std::mutex> pin_lock(g_pinned.mu, std::defer_lock);
  if (any_host_in || any_host_out) {
    pin_lock.lock();
    if (PinnedStage::grow(&g_pinned.in, &g_pinned.in_cap, (size_t)stage_bytes) != cudaSuccess)
      return host_fail(RPLU_ERR_NOMEM, "pinned staging buffer");
  }
  for (Group& g : groups) g.desc.reserve(g.idx.size());
  {
    Arena ar(s);
    char* stage = nullptr;
    if (stage_bytes + out_bytes > 0 && ar.alloc((void**)&stage, stage_bytes + out_bytes) != cudaSuccess)
      return host_fail(RPLU_ERR_NOMEM, "staging buffers");
    char* hin = (char*)g_pinned.in;
    // host inputs in place: gathered into the device staging by one kernel (the
    // piece list outlives the call's final synchronisation)
    std::vector<CopySeg> in_segs;
    {
      for (Group& g : groups) {
        const int64_t w = elem_bytes(g.dtype);
        for (int32_t b : g.idx) {
          const rplu_job& jb = jobs[b];
          const Staged& sg = stg[b];
          if (!sg.in_host || !sg.direct) continue;
          unsigned char* p = (unsigned char*)stage + sg.off_in;
          if (jb.kind == 0) {
            const int64_t ldp = align_up(jb.m, 16 / w), lda = jb.lda ? jb.lda : jb.m;
            for (int64_t r = 0; r < jb.n; ++r)
              in_segs.push_back(CopySeg{p + r * ldp * w, (const unsigned char*)jb.A + r * lda * w, jb.m * w});
          } else {
            in_segs.push_back(CopySeg{p, (const unsigned char*)jb.x, jb.n * w});
            in_segs.push_back(CopySeg{p + align_up(jb.n * w, 256), (const unsigned char*)jb.y, jb.m * w});
          }
        }
      }
      ce = copy_segs(ar, in_segs, sms, s);
      if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
    }
    // other host inputs packed into pinned memory and sent in one copy
    if (any_host_in) {
      std::vector<HostCopy> pieces;
      for (Group& g : groups) {
        const int64_t w = elem_bytes(g.dtype);
        for (int32_t b : g.idx) {
          const rplu_job& jb = jobs[b];
          const Staged& sg = stg[b];
          if (!sg.in_host || sg.direct) continue;
          char* p = hin + sg.off_in;
          if (jb.kind == 0) {
            const int64_t ldp = align_up(jb.m, 16 / w), lda = jb.lda ? jb.lda : jb.m;
            for (int64_t r = 0; r < jb.n; ++r)
              pieces.push_back(HostCopy{p + r * ldp * w, (const char*)jb.A + r * lda * w, jb.m * w});
          } else {
            pieces.push_back(HostCopy{p, jb.x, jb.n * w});
            pieces.push_back(HostCopy{p + align_up(jb.n * w, 256), jb.y, jb.m * w});
          }
        }
      }
      host_copies(pieces);
      ce = cudaMemcpyAsync(stage, hin, (size_t)stage_bytes, cudaMemcpyHostToDevice, s);
      if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
    }
    for (Group& g : groups) {
      if (g.idx.empty()) continue;
      const int64_t w = elem_bytes(g.dtype);
      for (int32_t b : g.idx) {
        const rplu_job& jb = jobs[b];
        const Staged& sg = stg[b];
        BatchDesc d;
        std::memset(&d, 0, sizeof(d));
        d.n = jb.n; d.m = jb.m; d.k_max = jb.k_max; d.tol = jb.rel_tol; d.seed = jb.seed; d.kind = jb.kind;
        d.lda = jb.kind == 0 ? (jb.lda ? jb.lda : jb.m) : jb.m;
        d.A = jb.A; d.x = jb.x; d.y = jb.y;
        if (sg.in_stage) {
          char* p = stage + sg.off_in;
          if (jb.kind == 0) {
            const int64_t ldp = align_up(jb.m, 16 / w);
            // device rows that are not 16-byte aligned: realigned on the device (host rows came in the bulk copy)
            if (!sg.in_host) cudaMemcpy2DAsync(p, ldp * w, jb.A, d.lda * w, jb.m * w, jb.n, cudaMemcpyDeviceToDevice, s);
            d.A = p;
            d.lda = ldp;
          } else {
            d.x = p;
            d.y = p + align_up(jb.n * w, 256);
          }
        }
        d.I = jb.I; d.J = jb.J; d.L = jb.L; d.U = jb.U;
        if (sg.out_host) {
          char* p = stage + stage_bytes + sg.off_out;
          d.I = (int64_t*)p;
          p += align_up(jb.k_max * 8, 256);
          d.J = (int64_t*)p;
          p += align_up(jb.k_max * 8, 256);
          d.L = p;
          p += align_up(jb.n * jb.k_max * w, 256);
          d.U = p;
        }
        g.desc.push_back(d);
      }
      plan_group(g, kDefaultBlk);
      const int blk = fit_blk(g, kDefaultBlk);
      if (blk < kDefaultBlk) plan_group(g, blk);
      if (blk == 0) return host_fail(RPLU_ERR_INVALID, "batch jobs too large for one CTA's shared memory");
      if (ar.alloc((void**)&g.d_desc, (int64_t)(g.desc.size() * sizeof(BatchDesc))) != cudaSuccess ||
          ar.alloc((void**)&g.d_order, (int64_t)(g.order.size() * sizeof(int32_t))) != cudaSuccess ||
          ar.alloc((void**)&g.d_counter, 16) != cudaSuccess ||
          ar.alloc((void**)&g.d_S, g.s_bytes) != cudaSuccess)
        return host_fail(RPLU_ERR_NOMEM, "batch workspace");
      resolve_workspace(g);
      fill_args(g, o.pivot);
      ce = set_shape(g, kDefaultThreads, kDefaultRows, blk, 0, sms, nullptr);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(g.d_desc, g.desc.data(), g.desc.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice, s);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(g.d_order, g.order.data(), g.order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
      if (ce == cudaSuccess) ce = enqueue_group(g, s);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(g.desc.data(), g.d_desc, g.desc.size() * sizeof(BatchDesc), cudaMemcpyDeviceToHost, s);
      if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
    }
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
    // host outputs: I, J in full and the first k_done columns of L and rows of U,
    // written in place by one kernel, or gathered on the device into one packed
    // buffer (offsets in `segs` until it exists) and sent back in one copy
    std::vector<CopySeg> segs, out_segs;
    struct HostPiece {
      void* dst;
      int64_t off, bytes;
    };
    std::vector<HostPiece> pieces;
    int64_t packed = 0;
    auto piece = [&](bool direct, void* dst, const void* src, int64_t bytes) {
      if (bytes <= 0) return;
      if (direct) {
        out_segs.push_back(CopySeg{(unsigned char*)dst, (const unsigned char*)src, bytes});
        return;
      }
      segs.push_back(CopySeg{(unsigned char*)(uintptr_t)packed, (const unsigned char*)src, bytes});
      pieces.push_back(HostPiece{dst, packed, bytes});
      packed += align_up(bytes, 16);
    };
    for (Group& g : groups) {
      const int64_t w = elem_bytes(g.dtype);
      for (size_t q = 0; q < g.idx.size(); ++q) {
        rplu_job& jb = jobs[g.idx[q]];
        const BatchDesc& d = g.desc[q];
        finish_job(jb, d);
        const Staged& sg = stg[g.idx[q]];
        if (sg.out_host && jb.k_max > 0) {
          piece(sg.direct, jb.I, d.I, jb.k_max * 8);
          piece(sg.direct, jb.J, d.J, jb.k_max * 8);
          piece(sg.direct, jb.L, d.L, jb.n * d.k_done * w);
          piece(sg.direct, jb.U, d.U, d.k_done * jb.m * w);
        }
        note((rplu_status)jb.status);
      }
    }
    ce = copy_segs(ar, out_segs, sms, s);
    if (ce == cudaSuccess && out_segs.size() > 0 && segs.empty()) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
    if (!segs.empty()) {
      unsigned char* dpack = nullptr;
      if (ar.alloc((void**)&dpack, packed) != cudaSuccess) return host_fail(RPLU_ERR_NOMEM, "packed results");
      if (PinnedStage::grow(&g_pinned.out, &g_pinned.out_cap, (size_t)packed) != cudaSuccess)
        return host_fail(RPLU_ERR_NOMEM, "pinned result buffer");
      for (CopySeg& c : segs) c.dst = dpack + (uintptr_t)c.dst;
      ce = copy_segs(ar, segs, sms, s);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(g_pinned.out, dpack, (size_t)packed, cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
      const char* hout = (const char*)g_pinned.out;
      std::vector<HostCopy> copies;
      copies.reserve(pieces.size());
      for (const HostPiece& hp : pieces) copies.push_back(HostCopy{hp.dst, hout + hp.off, hp.bytes});
      host_copies(copies);
    }
  }
  for (int32_t b : single) {
    rplu_status st = run_single(jobs[b], o, s);
    jobs[b].status = st;
    note(st);
  }
  for (int32_t b = 0; b < njobs; ++b)
    if (jobs[b].status == RPLU_ERR_INVALID) note(RPLU_ERR_INVALID);
  cudaStreamSynchronize(s);
  return worst;
}

rplu_status rplu_batch_plan_create(rplu_job* jobs, int32_t njobs, const rplu_opts* opts, int32_t tune,
                                   rplu_batch_plan** plan) {
  if (!plan) return host_fail(RPLU_ERR_INVALID, "plan is NULL");
  *plan = nullptr;
  rplu_opts o;
  if (opts) o = *opts;
  else rplu_opts_init(&o);
  if (njobs <= 0 || !jobs) return host_fail(RPLU_ERR_INVALID, "a plan needs at least one job");
  if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2)
    return host_fail(RPLU_ERR_INVALID, "plans support RPLU_PIVOT_RANDOM and RPLU_PIVOT_C2");
  for (int32_t b = 0; b < njobs; ++b) {
    const rplu_job& jb = jobs[b];
    if (const char* why = job_invalid(jb)) return host_fail(RPLU_ERR_INVALID, why);
    if (!fits_kernel(jb)) return host_fail(RPLU_ERR_INVALID, "plan jobs must have n, m <= 4096");
    const bool in_dev = jb.n * jb.m == 0 ||
                        (jb.kind == 0 ? host_on_device(jb.A) : host_on_device(jb.x) && host_on_device(jb.y));
    const bool out_dev = jb.k_max == 0 || (host_on_device(jb.I) && host_on_device(jb.J) && host_on_device(jb.L) &&
                                           host_on_device(jb.U));
    if (!in_dev || !out_dev) return host_fail(RPLU_ERR_INVALID, "plan jobs must use device memory only");
  }
  int sms = 0;
  cudaError_t ce = host_num_sms(&sms);
  if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  rplu_batch_plan* p = new rplu_batch_plan;
  p->jobs = jobs;
  p->njobs = njobs;
  auto bail = [p](rplu_status st, const char* msg) {
    plan_free(p);
    return host_fail(st, msg);
  };
  ce = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return bail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  for (int dt : {RPLU_F32, RPLU_F64, RPLU_C64}) {
    Group g;
    g.dtype = dt;
    const int64_t w = elem_bytes(dt);
    for (int32_t b = 0; b < njobs; ++b) {
      const rplu_job& jb = jobs[b];
      if (jb.dtype != dt) continue;
      BatchDesc d;
      std::memset(&d, 0, sizeof(d));
      d.n = jb.n; d.m = jb.m; d.k_max = jb.k_max; d.tol = jb.rel_tol; d.seed = jb.seed; d.kind = jb.kind;
      d.lda = jb.kind == 0 ? (jb.lda ? jb.lda : jb.m) : jb.m;
      d.A = jb.A; d.x = jb.x; d.y = jb.y;
      d.I = jb.I; d.J = jb.J; d.L = jb.L; d.U = jb.U;
      if (jb.kind == 0 && jb.n * jb.m > 0 && !rows_aligned(jb.A, d.lda, w)) {
        // the graph copies the rows into an aligned buffer before each run
        const int64_t ldp = align_up(jb.m, 16 / w);
        void* q = nullptr;
        if (cudaMalloc(&q, (size_t)(jb.n * ldp * w)) != cudaSuccess) return bail(RPLU_ERR_NOMEM, "plan staging");
        p->dev_allocs.push_back(q);
        p->copies.push_back({q, ldp * w, jb.A, d.lda * w, jb.m * w, jb.n});
        d.A = q;
        d.lda = ldp;
      }
      g.idx.push_back(b);
      g.desc.push_back(d);
    }
    if (g.idx.empty()) continue;
    plan_group(g, 4);  // workspace for the smallest candidate interval
    if (fit_blk(g, 1) == 0) return bail(RPLU_ERR_INVALID, "batch jobs too large for one CTA's shared memory");
    void* q = nullptr;
    const size_t need[4] = {g.desc.size() * sizeof(BatchDesc), g.order.size() * sizeof(int32_t), 16,
                            (size_t)g.s_bytes};
    void** dst[4] = {(void**)&g.d_desc, (void**)&g.d_order, (void**)&g.d_counter, (void**)&g.d_S};
    for (int a = 0; a < 4; ++a) {
      if (need[a] == 0) continue;
      if (cudaMalloc(&q, need[a]) != cudaSuccess) return bail(RPLU_ERR_NOMEM, "plan workspace");
      p->dev_allocs.push_back(q);
      *dst[a] = q;
    }
    resolve_workspace(g);
    fill_args(g, o.pivot);
    ce = cudaMemcpyAsync(g.d_desc, g.desc.data(), need[0], cudaMemcpyHostToDevice, p->cap);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(g.d_order, g.order.data(), need[1], cudaMemcpyHostToDevice, p->cap);
    if (ce == cudaSuccess) {
      if (tune) ce = tune_group(g, sms, p->cap);
      else ce = set_shape(g, kDefaultThreads, kDefaultRows, fit_blk(g, kDefaultBlk), 0, sms, nullptr);
    }
    if (ce != cudaSuccess) return bail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
    p->groups.push_back(std::move(g));
  }
  ce = cudaStreamSynchronize(p->cap);
  if (ce == cudaSuccess) ce = cudaMallocHost((void**)&p->h_mirror, (size_t)njobs * sizeof(BatchDesc));
  if (ce != cudaSuccess) return bail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  // one graph: per group, reset the counter, the persistent launch, results to the pinned mirror
  ce = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) return bail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  size_t off = 0;
  cudaError_t ce2 = cudaSuccess;
  for (const PlanCopy& c : p->copies)
    if (ce2 == cudaSuccess)
      ce2 = cudaMemcpy2DAsync(c.dst, c.dpitch, c.src, c.spitch, c.width, c.height, cudaMemcpyDeviceToDevice, p->cap);
  for (Group& g : p->groups) {
    if (ce2 == cudaSuccess) ce2 = enqueue_group(g, p->cap);
    if (ce2 == cudaSuccess)
      ce2 = cudaMemcpyAsync(p->h_mirror + off, g.d_desc, g.desc.size() * sizeof(BatchDesc), cudaMemcpyDeviceToHost,
                            p->cap);
    off += g.desc.size();
  }
  ce = cudaStreamEndCapture(p->cap, &p->graph);
  if (ce2 != cudaSuccess) return bail(RPLU_ERR_CUDA, cudaGetErrorString(ce2));
  if (ce != cudaSuccess) return bail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (ce != cudaSuccess) return bail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  *plan = p;
  return RPLU_OK;
}

rplu_status rplu_batch_plan_run(rplu_batch_plan* plan, void* stream) {
  if (!plan) return host_fail(RPLU_ERR_INVALID, "plan is NULL");
  cudaError_t ce = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
  if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  plan->last = (cudaStream_t)stream;
  plan->ran = true;
  return RPLU_OK;
}

rplu_status rplu_batch_plan_wait(rplu_batch_plan* plan) {
  if (!plan) return host_fail(RPLU_ERR_INVALID, "plan is NULL");
  if (!plan->ran) return host_fail(RPLU_ERR_INVALID, "plan has not run");
  cudaError_t ce = cudaStreamSynchronize(plan->last);
  if (ce != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(ce));
  rplu_status worst = RPLU_OK;
  size_t off = 0;
  for (const Group& g : plan->groups) {
    for (size_t q = 0; q < g.idx.size(); ++q) {
      rplu_job& jb = plan->jobs[g.idx[q]];
      finish_job(jb, plan->h_mirror[off + q]);
      const rplu_status st = (rplu_status)jb.status;
      if (st != RPLU_OK && (worst == RPLU_OK || worst == RPLU_NOT_CONVERGED)) worst = st;
    }
    off += g.idx.size();
  }
  return worst;
}

rplu_status rplu_batch_plan_shape(const rplu_batch_plan* plan, int32_t shape[4], double* tuned_ms) {
  if (!plan || !shape) return host_fail(RPLU_ERR_INVALID, "NULL argument");
  const Group* g = main_group(plan);
  if (!g) return host_fail(RPLU_ERR_INVALID, "empty plan");
  int sms = 1;
  host_num_sms(&sms);
  shape[0] = g->shape.threads;
  shape[1] = g->shape.rows;
  shape[2] = g->args.blk;
  shape[3] = (g->shape.grid + sms - 1) / sms;
  if (tuned_ms) *tuned_ms = g->tuned_ms;
  return RPLU_OK;
}

void rplu_batch_plan_destroy(rplu_batch_plan* plan) { plan_free(plan); }

}  // extern "C"
