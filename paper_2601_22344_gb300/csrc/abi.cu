// C-ABI entry points of librplu (declared in include/rplu.h): argument
// checks, host/device pointer classification, stream-ordered workspace,
// staging of host data, and status mapping.  All arithmetic runs in the
// kernels of dense.cu, cauchy.cu and batch.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "batch.h"
#include "bh_plan.h"
#include "csr.h"
#include "kernels.h"
#include "rplu.h"

namespace rplu {
namespace {

thread_local std::string g_last_error;

rplu_status fail(rplu_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

rplu_status cuda_fail(cudaError_t e, const char* where) {
  return fail(RPLU_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int64_t dtype_bytes(int32_t dt) {
  switch (dt) {
    case RPLU_F32: return 4;
    case RPLU_F64: return 8;
    case RPLU_C64: return 8;
    case RPLU_C128: return 16;
    default: return -1;
  }
}

int64_t dtype_vec(int32_t dt) { return 16 / dtype_bytes(dt); }

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The device address of page-locked (pinned, mapped) host memory, or null for
// pageable host memory and device memory.
const void* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

struct DeviceInfo {
  int num_sms = 0;
  int pageable = 0;  // the device reads and writes pageable host memory in place (coherent host link)
};

std::mutex g_dev_mu;
std::vector<DeviceInfo> g_devs;

// Per-device set-up: SM count; the default memory pool keeps freed workspace
// for reuse instead of returning it to the driver at every synchronisation.
cudaError_t device_info(DeviceInfo* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if ((int)g_devs.size() <= dev) g_devs.resize(dev + 1);
  if (g_devs[dev].num_sms == 0) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool;
    e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e != cudaSuccess) return e;
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) return e;
    int pageable = 0;
    e = cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev);
    if (e != cudaSuccess) return e;
    g_devs[dev].pageable = pageable;
    g_devs[dev].num_sms = sms;
  }
  *out = g_devs[dev];
  return cudaSuccess;
}

// Stream-ordered allocations released (stream-ordered) when the call returns.
struct Workspace {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Workspace(cudaStream_t st) : s(st) {}
  ~Workspace() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename P>
  cudaError_t alloc(P** p, int64_t bytes) {
    *p = nullptr;
    if (bytes <= 0) return cudaSuccess;
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, (size_t)bytes, s);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    *p = (P*)q;
    return cudaSuccess;
  }
};

// A caller buffer seen from the device: the caller's own pointer when it is
// device memory, else a staging buffer copied in and/or out.
struct Buf {
  void* user = nullptr;
  void* dev = nullptr;
  int64_t bytes = 0;
  bool staged = false;
};

cudaError_t bind(Workspace& ws, Buf& b, const void* user, int64_t bytes, bool copy_in) {
  b.user = const_cast<void*>(user);
  b.bytes = bytes;
  if (bytes <= 0 || user == nullptr) {
    b.dev = nullptr;
    return cudaSuccess;
  }
  if (on_device(user)) {
    b.dev = b.user;
    return cudaSuccess;
  }
  b.staged = true;
  cudaError_t e = ws.alloc(&b.dev, bytes);
  if (e != cudaSuccess) return e;
  if (copy_in) return cudaMemcpyAsync(b.dev, user, (size_t)bytes, cudaMemcpyHostToDevice, ws.s);
  return cudaSuccess;
}

cudaError_t copy_out(const Buf& b, cudaStream_t s) {
  if (!b.staged || b.bytes <= 0) return cudaSuccess;
  return cudaMemcpyAsync(b.user, b.dev, (size_t)b.bytes, cudaMemcpyDeviceToHost, s);
}

rplu_status check_common(const rplu_opts& o, int64_t n, int64_t m, int64_t k, const int64_t* I, const int64_t* J,
                         const void* L, const void* U, const int64_t* k_done) {
  if (dtype_bytes(o.dtype) < 0) return fail(RPLU_ERR_INVALID, "unknown dtype");
  if (o.pivot < RPLU_PIVOT_RANDOM || o.pivot > RPLU_PIVOT_GIVEN) return fail(RPLU_ERR_INVALID, "unknown pivot mode");
  if (n < 0 || m < 0 || k < 0) return fail(RPLU_ERR_INVALID, "negative size");
  if (k > (n < m ? n : m)) return fail(RPLU_ERR_INVALID, "k exceeds min(n, m)");
  if (!k_done) return fail(RPLU_ERR_INVALID, "k_done is NULL");
  if (k > 0 && (!I || !J || !L || !U)) return fail(RPLU_ERR_INVALID, "NULL output with k > 0");
  if (!(o.rel_tol >= 0.0) || !std::isfinite(o.rel_tol)) return fail(RPLU_ERR_INVALID, "rel_tol must be finite and >= 0");
  if (o.pivot == RPLU_PIVOT_GIVEN && k > 0 && (!o.given_I || !o.given_J))
    return fail(RPLU_ERR_INVALID, "RPLU_PIVOT_GIVEN needs given_I and given_J");
  if (n > (int64_t)1 << 40 || m > (int64_t)1 << 40) return fail(RPLU_ERR_INVALID, "size too large");
  return RPLU_OK;
}

rplu_status finish_status(const JobState& st, const rplu_opts& o, int64_t k, double T_final) {
  const char* why = "";
  const rplu_status r = job_status(st, o.rel_tol, k, T_final, &why);
  return r == RPLU_OK ? RPLU_OK : fail(r, why);
}

rplu_opts default_opts() {
  rplu_opts o;
  std::memset(&o, 0, sizeof(o));
  o.dtype = RPLU_F64;
  o.pivot = RPLU_PIVOT_RANDOM;
  return o;
}

// ------------------------------------------------------ hot-kernel timer
std::mutex g_ev_mu;
std::vector<std::vector<cudaEvent_t>> g_ev_pool;  // per device, created with timing enabled

struct EvList {
  int dev = 0;
  std::vector<cudaEvent_t> ev;
};

cudaEvent_t acquire_event(int dev) {
  {
    std::lock_guard<std::mutex> lk(g_ev_mu);
    if ((int)g_ev_pool.size() <= dev) g_ev_pool.resize(dev + 1);
    if (!g_ev_pool[dev].empty()) {
      cudaEvent_t e = g_ev_pool[dev].back();
      g_ev_pool[dev].pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

#define CK(expr, where)                         \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

}  // namespace

rplu_status host_fail(rplu_status s, const char* msg) { return fail(s, msg); }
bool host_on_device(const void* p) { return on_device(p); }
cudaError_t host_num_sms(int* sms) {
  DeviceInfo di;
  cudaError_t e = device_info(&di);
  if (e == cudaSuccess) *sms = di.num_sms;
  return e;
}
cudaError_t host_pageable_access(bool* yes) {
  DeviceInfo di;
  cudaError_t e = device_info(&di);
  if (e == cudaSuccess) *yes = di.pageable != 0;
  return e;
}

void HotTimer::begin() {
  if (!on) return;
  EvList* l = (EvList*)impl;
  cudaEvent_t e = acquire_event(l->dev);
  if (e) {
    cudaEventRecord(e, s);
    l->ev.push_back(e);
  }
}

void HotTimer::end() {
  ++launches;
  if (!on) return;
  EvList* l = (EvList*)impl;
  cudaEvent_t e = acquire_event(l->dev);
  if (e) {
    cudaEventRecord(e, s);
    l->ev.push_back(e);
  }
}

double HotTimer::elapsed_ms() {
  if (!on) return 0.0;
  EvList* l = (EvList*)impl;
  double tot = 0.0;
  for (size_t q = 0; q + 1 < l->ev.size(); q += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, l->ev[q], l->ev[q + 1]) == cudaSuccess) tot += ms;
  }
  return tot;
}

void HotTimer::release() {
  if (!impl) return;
  EvList* l = (EvList*)impl;
  {
    std::lock_guard<std::mutex> lk(g_ev_mu);
    if ((int)g_ev_pool.size() <= l->dev) g_ev_pool.resize(l->dev + 1);
    for (cudaEvent_t e : l->ev) g_ev_pool[l->dev].push_back(e);
  }
  delete l;
  impl = nullptr;
}

namespace {

// Points (dtype) in device memory to host FP64 real and imaginary parts.
cudaError_t points_host(const void* dev, int64_t n, int32_t dtype, cudaStream_t s, std::vector<double>& re,
                        std::vector<double>& im) {
  const int64_t w = dtype_bytes(dtype);
  re.assign((size_t)n, 0.0);
  im.assign((size_t)n, 0.0);
  if (n == 0) return cudaSuccess;
  std::vector<unsigned char> raw((size_t)(n * w));
  cudaError_t e = cudaMemcpyAsync(raw.data(), dev, (size_t)(n * w), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  for (int64_t q = 0; q < n; ++q) {
    const unsigned char* src = raw.data() + q * w;
    if (dtype == RPLU_F32 || dtype == RPLU_C64) {
      float v[2] = {0.f, 0.f};
      std::memcpy(v, src, (size_t)w);
      re[(size_t)q] = v[0];
      im[(size_t)q] = v[1];
    } else {
      double v[2] = {0.0, 0.0};
      std::memcpy(v, src, (size_t)w);
      re[(size_t)q] = v[0];
      im[(size_t)q] = v[1];
    }
  }
  return cudaSuccess;
}

// Host arrays of a bound plan, kept until the call's final synchronisation.
struct BhHost {
  std::vector<int32_t> tperm, sperm, sleaf, sinner, a_off, a_node, e_off, e_node;
  std::vector<int2> tleaf, snode, sleafrange;
  std::vector<double> a_alpha;
};

template <typename V>
cudaError_t upload(Workspace& ws, const std::vector<V>& h, const V** out) {
  V* d = nullptr;
  cudaError_t e = ws.alloc(&d, (int64_t)std::max<size_t>(h.size(), 1) * (int64_t)sizeof(V));
  if (e == cudaSuccess && !h.empty())
    e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, ws.s);
  *out = d;
  return e;
}

// Quadtrees and interaction lists of App. C (Algorithm C.1) for the points
// x (n) and y (m) in device memory, uploaded into the workspace with the
// per-step buffers of Algorithm C.2.
rplu_status make_bh(Workspace& ws, int32_t dtype, const void* xdev, const void* ydev, int64_t n, int64_t m,
                    int64_t p, double nu, int64_t leaf, int64_t k, BhHost& h, BhLaunch& b) {
  std::vector<double> xr, xi, yr, yi;
  cudaError_t e = points_host(xdev, n, dtype, ws.s, xr, xi);
  if (e == cudaSuccess) e = points_host(ydev, m, dtype, ws.s, yr, yi);
  if (e != cudaSuccess) return cuda_fail(e, "read points");
  for (int64_t q = 0; q < n; ++q)
    if (!std::isfinite(xr[(size_t)q]) || !std::isfinite(xi[(size_t)q]))
      return fail(RPLU_ERR_INVALID, "input has a non-finite entry (or x_i == y_j)");
  for (int64_t q = 0; q < m; ++q)
    if (!std::isfinite(yr[(size_t)q]) || !std::isfinite(yi[(size_t)q]))
      return fail(RPLU_ERR_INVALID, "input has a non-finite entry (or x_i == y_j)");
  BhPlan plan;
  bh_make_plan(plan, xr.data(), xi.data(), n, yr.data(), yi.data(), m, nu, leaf);
  std::memset(&b, 0, sizeof(b));
  h.tperm.assign(plan.tgt.perm.begin(), plan.tgt.perm.end());
  h.sperm.assign(plan.src.perm.begin(), plan.src.perm.end());
  h.tleaf.clear();
  int32_t tmax = 0;
  for (int64_t id : plan.tleaf) {
    const BhNode& nd = plan.tgt.nodes[(size_t)id];
    h.tleaf.push_back(make_int2((int)nd.lo, (int)nd.hi));
    tmax = std::max<int32_t>(tmax, (int32_t)(nd.hi - nd.lo));
  }
  const size_t ns = plan.src.nodes.size();
  h.snode.resize(ns);
  h.sleafrange.resize(ns);
  h.sleaf.clear();
  h.sinner.clear();
  // leaves in tree order (ordered by their first point); each node's leaves
  // are then the contiguous run of leaves whose points lie in its range
  std::vector<std::pair<int64_t, int32_t>> leaves;
  for (size_t q = 0; q < ns; ++q) {
    const BhNode& nd = plan.src.nodes[q];
    h.snode[q] = make_int2((int)nd.lo, (int)nd.hi);
    if (nd.leaf) leaves.push_back({nd.lo, (int32_t)q});
    else h.sinner.push_back((int32_t)q);
  }
  std::sort(leaves.begin(), leaves.end());
  std::vector<int64_t> leaf_lo;
  for (const auto& lv : leaves) {
    h.sleaf.push_back(lv.second);
    leaf_lo.push_back(lv.first);
  }
  for (size_t q = 0; q < ns; ++q) {
    const BhNode& nd = plan.src.nodes[q];
    const int a0 = (int)(std::lower_bound(leaf_lo.begin(), leaf_lo.end(), nd.lo) - leaf_lo.begin());
    const int a1 = (int)(std::lower_bound(leaf_lo.begin(), leaf_lo.end(), nd.hi) - leaf_lo.begin());
    h.sleafrange[q] = make_int2(a0, a1);
  }
  h.a_off.assign(plan.a_off.begin(), plan.a_off.end());
  h.e_off.assign(plan.e_off.begin(), plan.e_off.end());
  h.a_node = plan.a_node;
  h.a_alpha = plan.a_alpha;
  h.e_node = plan.e_node;
  if (plan.a_node.size() >= (size_t)INT32_MAX || plan.e_node.size() >= (size_t)INT32_MAX)
    return fail(RPLU_ERR_INVALID, "interaction lists too long");
  b.n_tleaf = (int32_t)h.tleaf.size();
  b.n_snode = (int32_t)ns;
  b.n_sleaf = (int32_t)h.sleaf.size();
  b.n_sinner = (int32_t)h.sinner.size();
  b.tleaf_max = tmax;
  e = upload(ws, h.tperm, &b.tperm);
  if (e == cudaSuccess) e = upload(ws, h.sperm, &b.sperm);
  if (e == cudaSuccess) e = upload(ws, h.tleaf, &b.tleaf);
  if (e == cudaSuccess) e = upload(ws, h.snode, &b.snode);
  if (e == cudaSuccess) e = upload(ws, h.sleaf, &b.sleaf);
  if (e == cudaSuccess) e = upload(ws, h.sinner, &b.sinner);
  if (e == cudaSuccess) e = upload(ws, h.sleafrange, &b.sleafrange);
  if (e == cudaSuccess) e = upload(ws, h.a_off, &b.a_off);
  if (e == cudaSuccess) e = upload(ws, h.a_node, &b.a_node);
  if (e == cudaSuccess) e = upload(ws, h.a_alpha, &b.a_alpha);
  if (e == cudaSuccess) e = upload(ws, h.e_off, &b.e_off);
  if (e == cudaSuccess) e = upload(ws, h.e_node, &b.e_node);
  if (e == cudaSuccess) e = ws.alloc(&b.H, (int64_t)std::max<size_t>(ns, 1) * 2 * p * p * 8);
  // CTAs per target leaf: about 8 CTAs per SM in all (2 waves at 4 resident),
  // so that uneven leaves balance out
  int sms = 0;
  if (e == cudaSuccess) e = host_num_sms(&sms);
  b.nslice = (int32_t)std::min<int64_t>(8, std::max<int64_t>(1, (8 * (int64_t)sms + b.n_tleaf - 1) / std::max(b.n_tleaf, 1)));
  if (e == cudaSuccess) e = ws.alloc(&b.u, std::max<int64_t>(n, 1) * 8 * b.nslice);
  if (e == cudaSuccess) e = ws.alloc(&b.iter, 8);
  if (e == cudaSuccess) e = ws.alloc(&b.umax0, 8);
  if (e == cudaSuccess && k > 0) e = ws.alloc(&b.attempts, k * 4);
  if (e == cudaSuccess && k > 0) e = cudaMemsetAsync(b.attempts, 0, (size_t)k * 4, ws.s);
  if (e != cudaSuccess) return cuda_fail(e, "bound plan upload");
  return RPLU_OK;
}

rplu_status check_bound_args(double nu, int64_t leaf, int64_t n, int64_t m) {
  if (!(nu >= 1.0) || !std::isfinite(nu)) return fail(RPLU_ERR_INVALID, "bound_nu must be finite and >= 1");
  if (leaf < 1 || leaf > (1 << 20)) return fail(RPLU_ERR_INVALID, "bound leaf size must be in 1..2^20");
  if (n >= INT32_MAX || m >= INT32_MAX) return fail(RPLU_ERR_INVALID, "bound-based draw needs n, m < 2^31");
  return RPLU_OK;
}

// Starts the optional timer of a call; released (events back to the pool) on scope exit.
struct TimerScope {
  HotTimer tm;
  double* prof;
  TimerScope(double* p, cudaStream_t s) : prof(p) {
    tm.s = s;
    if (prof) {
      EvList* l = new EvList;
      cudaGetDevice(&l->dev);
      tm.impl = l;
      tm.on = true;
    }
  }
  // after the final synchronisation
  void report() {
    if (!prof) return;
    prof[0] += tm.elapsed_ms();
    prof[1] += (double)tm.launches;
    prof[2] += (double)tm.all_launches;
    prof[3] += 1.0;
  }
  ~TimerScope() { tm.release(); }
};

}  // namespace
}  // namespace rplu

namespace rplu {
namespace {
rplu_status cauchy_like_call(const void* x, const void* y, const void* G, const void* B, int64_t n, int64_t m,
                             int64_t p, int64_t k, uint64_t seed, const rplu_opts* opts, int64_t* I, int64_t* J,
                             void* L, void* U, int64_t* k_done, bool exact_ends);
}  // namespace
}  // namespace rplu

using namespace rplu;

extern "C" {

void rplu_opts_init(rplu_opts* o) {
  if (o) *o = default_opts();
}

int32_t rplu_version(void) { return 100; }

const char* rplu_status_string(rplu_status s) {
  switch (s) {
    case RPLU_OK: return "ok";
    case RPLU_ERR_INVALID: return "invalid argument or input";
    case RPLU_ERR_NOMEM: return "out of device memory";
    case RPLU_ERR_CUDA: return "CUDA error";
    case RPLU_ERR_TIMEOUT: return "device wait timed out";
    case RPLU_NOT_CONVERGED: return "tolerance not reached";
    case RPLU_CANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

const char* rplu_last_error(void) { return g_last_error.c_str(); }

rplu_status rplu_dense(const void* A, int64_t n, int64_t m, int64_t k, uint64_t seed, const rplu_opts* opts,
                       int64_t* I, int64_t* J, void* L, void* U, int64_t* k_done) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  rplu_status st0 = check_common(o, n, m, k, I, J, L, U, k_done);
  if (st0 != RPLU_OK) return st0;
  const int64_t lda = o.lda ? o.lda : m;
  if (lda < m) return fail(RPLU_ERR_INVALID, "lda < m");
  if (n > 0 && m > 0 && !A) return fail(RPLU_ERR_INVALID, "A is NULL");
  if (o.pivot == RPLU_PIVOT_COMPLETE && o.rel_tol > 0.0)
    return fail(RPLU_ERR_INVALID, "RPLU_PIVOT_COMPLETE does not take rel_tol");
  *k_done = 0;
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  const int64_t w = dtype_bytes(o.dtype);
  const int64_t V = dtype_vec(o.dtype);

  DenseLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.m = m; a.k = k;
  a.seed = seed; a.mode = o.pivot; a.tol = o.rel_tol; a.num_sms = di.num_sms;

  const bool a_dev = on_device(A);
  const bool aligned = ((uintptr_t)A % 16 == 0) && ((lda * w) % 16 == 0);
  if (a_dev && o.overwrite_input && aligned) {
    a.S = const_cast<void*>(A);
    a.lds = lda;
    a.A = A;
    a.lda = lda;
  } else {
    a.lds = (m + V - 1) / V * V;
    if (a.lds == 0) a.lds = V;
    CK(ws.alloc(&a.S, n * a.lds * w), "workspace S");
    const void* a_mapped = a_dev ? nullptr : mapped_host(A);
    if (a_dev) {
      a.A = A;
      a.lda = lda;
    } else if (a_mapped && aligned) {
      // pinned host A: the init kernel reads it in place over the host link while it
      // writes S and the row norms (no separate copy of A into device memory first)
      a.A = a_mapped;
      a.lda = lda;
    } else if (n > 0 && m > 0) {
      CK(cudaMemcpy2DAsync(a.S, (size_t)(a.lds * w), A, (size_t)(lda * w), (size_t)(m * w), (size_t)n,
                           cudaMemcpyHostToDevice, s), "stage A");
      a.A = a.S;
      a.lda = a.lds;
    }
  }
  JobState* dst = nullptr;
  CK(ws.alloc(&a.d, n * 8), "workspace d");
  CK(ws.alloc(&a.row_used, n), "workspace");
  CK(ws.alloc(&a.col_used, m), "workspace");
  int32_t blk = o.pass_block;
  if (blk <= 0) blk = default_pass_block(o.dtype);
  if (blk > 8) return fail(RPLU_ERR_INVALID, "pass_block must be at most 8");
  if (o.pivot == RPLU_PIVOT_COMPLETE) blk = 1;  // the row maxima come from the stored residual
  a.blk = blk;
  CK(ws.alloc(&a.ublk, (int64_t)blk * a.lds * w), "workspace");
  CK(ws.alloc(&a.T_hist, (k + 1) * 8), "workspace");
  CK(ws.alloc(&dst, (int64_t)sizeof(JobState)), "workspace");
  a.st = dst;
  if (o.pivot == RPLU_PIVOT_COMPLETE) {
    CK(ws.alloc(&a.rowmax, n * 8), "workspace");
    CK(ws.alloc(&a.rowarg, n * 8), "workspace");
  }
  if (n > 0) CK(cudaMemsetAsync(a.row_used, 0, n, s), "memset");
  if (m > 0) CK(cudaMemsetAsync(a.col_used, 0, m, s), "memset");
  CK(cudaMemsetAsync(dst, 0, sizeof(JobState), s), "memset");
  Buf bI, bJ, bL, bU, bgI, bgJ;
  CK(bind(ws, bI, I, k * 8, false), "bind I");
  CK(bind(ws, bJ, J, k * 8, false), "bind J");
  CK(bind(ws, bL, L, n * k * w, false), "bind L");
  CK(bind(ws, bU, U, k * m * w, false), "bind U");
  if (o.pivot == RPLU_PIVOT_GIVEN) {
    CK(bind(ws, bgI, o.given_I, k * 8, true), "bind given_I");
    CK(bind(ws, bgJ, o.given_J, k * 8, true), "bind given_J");
  }
  if (k > 0) {
    CK(cudaMemsetAsync(bI.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bJ.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bL.dev, 0, n * k * w, s), "memset");
    CK(cudaMemsetAsync(bU.dev, 0, k * m * w, s), "memset");
  }
  a.I = (int64_t*)bI.dev; a.J = (int64_t*)bJ.dev; a.L = bL.dev; a.U = bU.dev;
  a.gI = (const int64_t*)bgI.dev; a.gJ = (const int64_t*)bgJ.dev;

  TimerScope ts(o.prof, s);
  CK(dense_run(o.dtype, a, s, &ts.tm), "dense kernels");

  CK(copy_out(bI, s), "copy I");
  CK(copy_out(bJ, s), "copy J");
  CK(copy_out(bL, s), "copy L");
  CK(copy_out(bU, s), "copy U");
  if (o.T_hist) CK(cudaMemcpyAsync(o.T_hist, a.T_hist, (k + 1) * 8, cudaMemcpyDefault, s), "copy T_hist");
  if (o.d_out && n > 0) CK(cudaMemcpyAsync(o.d_out, a.d, n * 8, cudaMemcpyDefault, s), "copy d");
  JobState hst;
  CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
  std::vector<double> th(k + 1, 0.0);
  CK(cudaMemcpyAsync(th.data(), a.T_hist, (k + 1) * 8, cudaMemcpyDeviceToHost, s), "read T");
  CK(cudaStreamSynchronize(s), "synchronize");
  ts.report();
  *k_done = hst.k_done;
  return finish_status(hst, o, k, th[hst.k_done]);
}

rplu_status rplu_cauchy(const void* x, const void* y, int64_t n, int64_t m, int64_t k, uint64_t seed,
                        const rplu_opts* opts, int64_t* I, int64_t* J, void* L, void* U, int64_t* k_done) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  rplu_status st0 = check_common(o, n, m, k, I, J, L, U, k_done);
  if (st0 != RPLU_OK) return st0;
  if (o.pivot == RPLU_PIVOT_COMPLETE) return fail(RPLU_ERR_INVALID, "RPLU_PIVOT_COMPLETE needs the dense form");
  if ((n > 0 && !x) || (m > 0 && !y)) return fail(RPLU_ERR_INVALID, "x or y is NULL");
  *k_done = 0;
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  const int64_t w = dtype_bytes(o.dtype);

  CauchyLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.m = m; a.k = k;
  a.seed = seed; a.mode = o.pivot; a.tol = o.rel_tol; a.num_sms = di.num_sms;
  a.nchunk = cauchy_chunks(n, m, o.dtype, di.num_sms);
  Buf bx, by;
  CK(bind(ws, bx, x, n * w, true), "bind x");
  CK(bind(ws, by, y, m * w, true), "bind y");
  a.x = bx.dev; a.y = by.dev;
  JobState* dst = nullptr;
  CK(ws.alloc(&a.d, n * 8), "workspace d");
  CK(ws.alloc(&a.row_used, n), "workspace");
  CK(ws.alloc(&a.col_used, m), "workspace");
  CK(ws.alloc(&a.rhat, m * w), "workspace");
  CK(ws.alloc(&a.urow, m * w), "workspace");
  CK(ws.alloc(&a.T_hist, (k + 1) * 8), "workspace");
  CK(ws.alloc(&a.vproj, (k > 0 ? k : 1) * 16), "workspace");
  CK(ws.alloc(&a.part, (int64_t)a.nchunk * n * 16), "workspace");
  CK(ws.alloc(&dst, (int64_t)sizeof(JobState)), "workspace");
  a.st = dst;
  if (n > 0) CK(cudaMemsetAsync(a.row_used, 0, n, s), "memset");
  if (m > 0) CK(cudaMemsetAsync(a.col_used, 0, m, s), "memset");
  CK(cudaMemsetAsync(dst, 0, sizeof(JobState), s), "memset");
  Buf bI, bJ, bL, bU, bgI, bgJ;
  CK(bind(ws, bI, I, k * 8, false), "bind I");
  CK(bind(ws, bJ, J, k * 8, false), "bind J");
  CK(bind(ws, bL, L, n * k * w, false), "bind L");
  CK(bind(ws, bU, U, k * m * w, false), "bind U");
  if (o.pivot == RPLU_PIVOT_GIVEN) {
    CK(bind(ws, bgI, o.given_I, k * 8, true), "bind given_I");
    CK(bind(ws, bgJ, o.given_J, k * 8, true), "bind given_J");
  }
  if (k > 0) {
    CK(cudaMemsetAsync(bI.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bJ.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bL.dev, 0, n * k * w, s), "memset");
    CK(cudaMemsetAsync(bU.dev, 0, k * m * w, s), "memset");
  }
  a.I = (int64_t*)bI.dev; a.J = (int64_t*)bJ.dev; a.L = bL.dev; a.U = bU.dev;
  a.gI = (const int64_t*)bgI.dev; a.gJ = (const int64_t*)bgJ.dev;

  TimerScope ts(o.prof, s);
  CK(cauchy_init(o.dtype, a, s, &ts.tm), "cauchy init");
  JobState hst;
  std::memset(&hst, 0, sizeof(hst));
  int64_t launched = 0;
  const int64_t max_seq = (int64_t)kMaxAttempts * (k + 1);
  while (k > 0) {
    const int64_t steps = k - hst.t;
    CK(cauchy_run(o.dtype, a, s, steps, &ts.tm), "cauchy kernels");
    launched += steps;
    CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (hst.done || hst.t >= k || launched >= max_seq) break;
  }
  CK(cauchy_finish(a, s, &ts.tm), "cauchy finish");
  CK(copy_out(bI, s), "copy I");
  CK(copy_out(bJ, s), "copy J");
  CK(copy_out(bL, s), "copy L");
  CK(copy_out(bU, s), "copy U");
  if (o.T_hist) CK(cudaMemcpyAsync(o.T_hist, a.T_hist, (k + 1) * 8, cudaMemcpyDefault, s), "copy T_hist");
  if (o.d_out && n > 0) CK(cudaMemcpyAsync(o.d_out, a.d, n * 8, cudaMemcpyDefault, s), "copy d");
  CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
  std::vector<double> th(k + 1, 0.0);
  CK(cudaMemcpyAsync(th.data(), a.T_hist, (k + 1) * 8, cudaMemcpyDeviceToHost, s), "read T");
  CK(cudaStreamSynchronize(s), "synchronize");
  ts.report();
  *k_done = hst.k_done;
  return finish_status(hst, o, k, th[hst.k_done]);
}

rplu_status rplu_cauchy_cur(const void* x, const void* y, int64_t n, int64_t m, int64_t k, uint64_t seed,
                            const rplu_opts* opts, int64_t* I, int64_t* J, void* core, int64_t* k_done) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  int64_t dummy_ij = 0;
  rplu_status st0 = check_common(o, n, m, k, I, J, k > 0 ? core : (void*)&dummy_ij, k > 0 ? core : (void*)&dummy_ij,
                                 k_done);
  if (st0 != RPLU_OK) return st0;
  if (o.pivot == RPLU_PIVOT_COMPLETE) return fail(RPLU_ERR_INVALID, "RPLU_PIVOT_COMPLETE needs the dense form");
  if ((n > 0 && !x) || (m > 0 && !y)) return fail(RPLU_ERR_INVALID, "x or y is NULL");
  *k_done = 0;
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  const int64_t w = dtype_bytes(o.dtype);
  CauchyLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.m = m; a.k = k;
  a.seed = seed; a.mode = o.pivot; a.tol = o.rel_tol; a.num_sms = di.num_sms;
  a.nchunk = cauchy_chunks(n, m, o.dtype, di.num_sms);
  Buf bx, by;
  CK(bind(ws, bx, x, n * w, true), "bind x");
  CK(bind(ws, by, y, m * w, true), "bind y");
  a.x = bx.dev; a.y = by.dev;
  JobState* dst = nullptr;
  CK(ws.alloc(&a.d, std::max<int64_t>(n, 1) * 8), "workspace d");
  CK(ws.alloc(&a.row_used, std::max<int64_t>(n, 1)), "workspace");
  CK(ws.alloc(&a.col_used, std::max<int64_t>(m, 1)), "workspace");
  CK(ws.alloc(&a.rhat, std::max<int64_t>(m, 1) * w), "workspace");
  CK(ws.alloc(&a.urow, std::max<int64_t>(m, 1) * w), "workspace");
  CK(ws.alloc(&a.lcol, std::max<int64_t>(n, 1) * w), "workspace");
  CK(ws.alloc(&a.T_hist, (k + 1) * 8), "workspace");
  CK(ws.alloc(&a.part, std::max<int64_t>((int64_t)a.nchunk * n, 1) * 16), "workspace");
  const int64_t kk = std::max<int64_t>(k, 1);
  CK(ws.alloc(&a.core, kk * kk * 16), "workspace core");
  CK(ws.alloc(&a.vb, kk * 16), "workspace");
  CK(ws.alloc(&a.ve, kk * 16), "workspace");
  CK(ws.alloc(&a.vg, kk * 16), "workspace");
  CK(ws.alloc(&a.vh, kk * 16), "workspace");
  CK(ws.alloc(&dst, (int64_t)sizeof(JobState)), "workspace");
  a.st = dst;
  if (n > 0) CK(cudaMemsetAsync(a.row_used, 0, n, s), "memset");
  if (m > 0) CK(cudaMemsetAsync(a.col_used, 0, m, s), "memset");
  CK(cudaMemsetAsync(dst, 0, sizeof(JobState), s), "memset");
  Buf bI, bJ, bC, bgI, bgJ;
  CK(bind(ws, bI, I, k * 8, false), "bind I");
  CK(bind(ws, bJ, J, k * 8, false), "bind J");
  const int64_t wc = (o.dtype == RPLU_C64 || o.dtype == RPLU_C128) ? 16 : 8;  // the core is FP64
  CK(bind(ws, bC, core, k * k * wc, false), "bind core");
  if (o.pivot == RPLU_PIVOT_GIVEN) {
    CK(bind(ws, bgI, o.given_I, k * 8, true), "bind given_I");
    CK(bind(ws, bgJ, o.given_J, k * 8, true), "bind given_J");
  }
  if (k > 0) {
    CK(cudaMemsetAsync(bI.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bJ.dev, 0xff, k * 8, s), "memset");
  }
  a.I = (int64_t*)bI.dev; a.J = (int64_t*)bJ.dev;
  a.gI = (const int64_t*)bgI.dev; a.gJ = (const int64_t*)bgJ.dev;

  TimerScope ts(o.prof, s);
  CK(cauchy_init(o.dtype, a, s, &ts.tm), "cauchy init");
  JobState hst;
  std::memset(&hst, 0, sizeof(hst));
  int64_t launched = 0;
  const int64_t max_seq = (int64_t)kMaxAttempts * (k + 1);
  while (k > 0 && n > 0 && m > 0) {
    const int64_t steps = k - hst.t;
    CK(cauchy_cur_run(o.dtype, a, s, steps, &ts.tm), "cauchy CUR kernels");
    launched += steps;
    CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (hst.done || hst.t >= k || launched >= max_seq) break;
  }
  if (n > 0 && m > 0) CK(cauchy_finish(a, s, &ts.tm), "cauchy finish");
  CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
  CK(cudaStreamSynchronize(s), "synchronize");
  if (k > 0) CK(cauchy_core_out(o.dtype, a.core, k, hst.k_done, bC.dev, di.num_sms, s), "core out");
  CK(copy_out(bI, s), "copy I");
  CK(copy_out(bJ, s), "copy J");
  CK(copy_out(bC, s), "copy core");
  if (o.T_hist) CK(cudaMemcpyAsync(o.T_hist, a.T_hist, (k + 1) * 8, cudaMemcpyDefault, s), "copy T_hist");
  if (o.d_out && n > 0) CK(cudaMemcpyAsync(o.d_out, a.d, n * 8, cudaMemcpyDefault, s), "copy d");
  std::vector<double> th(k + 1, 0.0);
  CK(cudaMemcpyAsync(th.data(), a.T_hist, (k + 1) * 8, cudaMemcpyDeviceToHost, s), "read T");
  CK(cudaStreamSynchronize(s), "synchronize");
  ts.report();
  *k_done = hst.k_done;
  return finish_status(hst, o, k, th[hst.k_done]);
}

rplu_status rplu_cauchy_like(const void* x, const void* y, const void* G, const void* B, int64_t n, int64_t m,
                             int64_t p, int64_t k, uint64_t seed, const rplu_opts* opts, int64_t* I, int64_t* J,
                             void* L, void* U, int64_t* k_done) {
  return rplu::cauchy_like_call(x, y, G, B, n, m, p, k, seed, opts, I, J, L, U, k_done, true);
}

}  // extern "C"

namespace rplu {
namespace {
// rplu_cauchy_like; exact_ends = false (bound-based draw with the max rule only)
// skips the exact row-norm passes before and after the loop.
rplu_status cauchy_like_call(const void* x, const void* y, const void* G, const void* B, int64_t n, int64_t m,
                             int64_t p, int64_t k, uint64_t seed, const rplu_opts* opts, int64_t* I, int64_t* J,
                             void* L, void* U, int64_t* k_done, bool exact_ends) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  rplu_status st0 = check_common(o, n, m, k, I, J, L, U, k_done);
  if (st0 != RPLU_OK) return st0;
  if (o.pivot == RPLU_PIVOT_COMPLETE) return fail(RPLU_ERR_INVALID, "RPLU_PIVOT_COMPLETE needs the dense form");
  if (p < 1 || p > 4) return fail(RPLU_ERR_INVALID, "displacement rank p must be 1..4");
  if ((n > 0 && (!x || !G)) || (m > 0 && (!y || !B))) return fail(RPLU_ERR_INVALID, "x, y, G or B is NULL");
  const bool bounded = o.bound_nu != 0.0;
  const int64_t leaf = o.bound_leaf > 0 ? o.bound_leaf : 32;
  if (bounded) {
    if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2)
      return fail(RPLU_ERR_INVALID, "bound_nu needs RPLU_PIVOT_RANDOM or RPLU_PIVOT_C2");
    if (o.bound_stop != 0 && o.bound_stop != 1) return fail(RPLU_ERR_INVALID, "bound_stop must be 0 or 1");
    if (o.bound_leaf < 0) return fail(RPLU_ERR_INVALID, "bound_leaf must be >= 0");
    st0 = check_bound_args(o.bound_nu, leaf, n, m);
    if (st0 != RPLU_OK) return st0;
  }
  *k_done = 0;
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  const int64_t w = dtype_bytes(o.dtype);

  CauchyLikeLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.m = m; a.p = p; a.k = k;
  a.seed = seed; a.mode = o.pivot; a.tol = o.rel_tol; a.num_sms = di.num_sms;
  a.nchunk = cauchy_like_chunks(n, m, o.dtype, p, di.num_sms);
  Buf bx, by;
  CK(bind(ws, bx, x, n * w, true), "bind x");
  CK(bind(ws, by, y, m * w, true), "bind y");
  a.x = bx.dev; a.y = by.dev;
  // private copies of the generators: they are updated in place
  CK(ws.alloc(&a.G, std::max<int64_t>(n * p * w, 16)), "workspace G");
  CK(ws.alloc(&a.B, std::max<int64_t>(p * m * w, 16)), "workspace B");
  if (n > 0) CK(cudaMemcpyAsync(a.G, G, n * p * w, cudaMemcpyDefault, s), "copy G");
  if (m > 0) CK(cudaMemcpyAsync(a.B, B, p * m * w, cudaMemcpyDefault, s), "copy B");
  JobState* dst = nullptr;
  CK(ws.alloc(&a.d, std::max<int64_t>(n, 1) * 8), "workspace d");
  CK(ws.alloc(&a.row_used, std::max<int64_t>(n, 1)), "workspace");
  CK(ws.alloc(&a.col_used, std::max<int64_t>(m, 1)), "workspace");
  CK(ws.alloc(&a.r, std::max<int64_t>(m, 1) * w), "workspace");
  CK(ws.alloc(&a.gi, 4 * w), "workspace");
  CK(ws.alloc(&a.bj, 4 * w), "workspace");
  CK(ws.alloc(&a.T_hist, (k + 1) * 8), "workspace");
  CK(cudaMemsetAsync(a.T_hist, 0, (k + 1) * 8, s), "memset");  // entries a run does not reach read as 0
  CK(ws.alloc(&a.part, std::max<int64_t>((int64_t)a.nchunk * n, 1) * 8), "workspace");
  CK(ws.alloc(&dst, (int64_t)sizeof(JobState)), "workspace");
  a.st = dst;
  if (n > 0) CK(cudaMemsetAsync(a.row_used, 0, n, s), "memset");
  if (m > 0) CK(cudaMemsetAsync(a.col_used, 0, m, s), "memset");
  CK(cudaMemsetAsync(dst, 0, sizeof(JobState), s), "memset");
  Buf bI, bJ, bL, bU, bgI, bgJ;
  CK(bind(ws, bI, I, k * 8, false), "bind I");
  CK(bind(ws, bJ, J, k * 8, false), "bind J");
  CK(bind(ws, bL, L, n * k * w, false), "bind L");
  CK(bind(ws, bU, U, k * m * w, false), "bind U");
  if (o.pivot == RPLU_PIVOT_GIVEN) {
    CK(bind(ws, bgI, o.given_I, k * 8, true), "bind given_I");
    CK(bind(ws, bgJ, o.given_J, k * 8, true), "bind given_J");
  }
  if (k > 0) {
    CK(cudaMemsetAsync(bI.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bJ.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bL.dev, 0, n * k * w, s), "memset");
    CK(cudaMemsetAsync(bU.dev, 0, k * m * w, s), "memset");
  }
  a.I = (int64_t*)bI.dev; a.J = (int64_t*)bJ.dev; a.L = bL.dev; a.U = bU.dev;
  a.gI = (const int64_t*)bgI.dev; a.gJ = (const int64_t*)bgJ.dev;

  TimerScope ts(o.prof, s);
  BhHost bh_host;
  BhLaunch bh;
  std::memset(&bh, 0, sizeof(bh));
  if (n > 0 && m > 0) {
    if (bounded) {
      st0 = make_bh(ws, o.dtype, a.x, a.y, n, m, p, o.bound_nu, leaf, k, bh_host, bh);
      if (st0 != RPLU_OK) return st0;
      bh.stop_max = o.bound_stop;
      bh.exact_ends = exact_ends || o.bound_stop == 0 ? 1 : 0;
      CK(cauchy_like_bh_run(o.dtype, a, bh, s, &ts.tm), "Cauchy-like bound kernels");
      if (o.attempts && k > 0) CK(cudaMemcpyAsync(o.attempts, bh.attempts, k * 4, cudaMemcpyDefault, s), "copy attempts");
    } else {
      CK(cauchy_like_run(o.dtype, a, s, &ts.tm), "Cauchy-like kernels");
    }
  }
  CK(copy_out(bI, s), "copy I");
  CK(copy_out(bJ, s), "copy J");
  CK(copy_out(bL, s), "copy L");
  CK(copy_out(bU, s), "copy U");
  JobState hst;
  std::memset(&hst, 0, sizeof(hst));
  std::vector<double> th(k + 1, 0.0);
  if (n > 0 && m > 0) {
    if (o.T_hist) CK(cudaMemcpyAsync(o.T_hist, a.T_hist, (k + 1) * 8, cudaMemcpyDefault, s), "copy T_hist");
    if (o.d_out) CK(cudaMemcpyAsync(o.d_out, a.d, n * 8, cudaMemcpyDefault, s), "copy d");
    CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
    CK(cudaMemcpyAsync(th.data(), a.T_hist, (k + 1) * 8, cudaMemcpyDeviceToHost, s), "read T");
  } else if (o.T_hist) {
    CK(cudaMemsetAsync(o.T_hist, 0, (k + 1) * 8, s), "zero T_hist");
  }
  CK(cudaStreamSynchronize(s), "synchronize");
  ts.report();
  *k_done = hst.k_done;
  return finish_status(hst, o, k, th[hst.k_done]);
}

}  // namespace
}  // namespace rplu

extern "C" {

rplu_status rplu_bh_bounds(const void* x, const void* y, const void* G, const void* B, int64_t n, int64_t m,
                           int64_t p, double nu, int64_t leaf, const rplu_opts* opts, double* u) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  if (dtype_bytes(o.dtype) < 0) return fail(RPLU_ERR_INVALID, "unknown dtype");
  if (n < 1 || m < 1) return fail(RPLU_ERR_INVALID, "n and m must be >= 1");
  if (p < 1 || p > 4) return fail(RPLU_ERR_INVALID, "displacement rank p must be 1..4");
  if (!x || !y || !G || !B || !u) return fail(RPLU_ERR_INVALID, "NULL pointer");
  rplu_status st0 = check_bound_args(nu, leaf, n, m);
  if (st0 != RPLU_OK) return st0;
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  const int64_t w = dtype_bytes(o.dtype);
  CauchyLikeLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.m = m; a.p = p; a.num_sms = di.num_sms;
  Buf bx, by, bG, bB, bu;
  CK(bind(ws, bx, x, n * w, true), "bind x");
  CK(bind(ws, by, y, m * w, true), "bind y");
  CK(bind(ws, bG, G, n * p * w, true), "bind G");
  CK(bind(ws, bB, B, p * m * w, true), "bind B");
  CK(bind(ws, bu, u, n * 8, false), "bind u");
  a.x = bx.dev; a.y = by.dev; a.G = bG.dev; a.B = bB.dev;
  JobState* dst = nullptr;
  CK(ws.alloc(&dst, (int64_t)sizeof(JobState)), "workspace");
  CK(cudaMemsetAsync(dst, 0, sizeof(JobState), s), "memset");
  a.st = dst;
  BhHost bh_host;
  BhLaunch bh;
  st0 = make_bh(ws, o.dtype, a.x, a.y, n, m, p, nu, leaf, 0, bh_host, bh);
  if (st0 != RPLU_OK) return st0;
  bh.u = (double*)bu.dev;
  bh.nslice = 1;
  CK(cauchy_like_bh_bounds(o.dtype, a, bh, s), "bound kernels");
  CK(copy_out(bu, s), "copy u");
  CK(cudaStreamSynchronize(s), "synchronize");
  return RPLU_OK;
}

rplu_status rplu_cur_aaa(const void* z, const void* f, int64_t m, double eps, int64_t k_max, uint64_t seed,
                         const rplu_opts* opts, int64_t* support, void* w, int64_t* k_out, int32_t* which,
                         double* err) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  if (o.dtype != RPLU_C128) return fail(RPLU_ERR_INVALID, "rplu_cur_aaa needs RPLU_C128 data");
  if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2)
    return fail(RPLU_ERR_INVALID, "rplu_cur_aaa needs RPLU_PIVOT_RANDOM or RPLU_PIVOT_C2");
  if (m < 2 || m >= INT32_MAX) return fail(RPLU_ERR_INVALID, "m must be in 2..2^31-1");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(RPLU_ERR_INVALID, "eps must be finite and > 0");
  if (k_max < 1) return fail(RPLU_ERR_INVALID, "k_max must be >= 1");
  if (!z || !f || !support || !w || !k_out || !which || !err) return fail(RPLU_ERR_INVALID, "NULL pointer");
  *k_out = 0;
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  const int64_t nx = (m + 1) / 2, ny = m / 2;
  AaaLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.m = m;
  a.seed = seed;
  a.num_sms = di.num_sms;
  Buf bz, bf;
  CK(bind(ws, bz, z, m * 16, true), "bind z");
  CK(bind(ws, bf, f, m * 16, true), "bind f");
  a.z = bz.dev;
  a.f = bf.dev;
  CK(ws.alloc(&a.flag, m), "workspace");
  CK(ws.alloc(&a.cnt, aaa_compact_blocks(m) * 4), "workspace");
  CK(ws.alloc(&a.total, 8), "workspace");
  CK(ws.alloc(&a.bad, 4), "workspace");
  CK(cudaMemsetAsync(a.bad, 0, 4, s), "memset");
  CK(ws.alloc(&a.xidx, nx * 8), "workspace");
  CK(ws.alloc(&a.yidx, ny * 8), "workspace");
  CK(ws.alloc(&a.x, nx * 16), "workspace");
  CK(ws.alloc(&a.fx, nx * 16), "workspace");
  CK(ws.alloc(&a.y, ny * 16), "workspace");
  CK(ws.alloc(&a.fy, ny * 16), "workspace");
  CK(ws.alloc(&a.G, nx * 32), "workspace");
  CK(ws.alloc(&a.B, ny * 32), "workspace");
  CK(ws.alloc(&a.fmax_bits, 8), "workspace");
  CK(aaa_split(a, s), "CUR-AAA split");
  int32_t bad = 0;
  CK(cudaMemcpyAsync(&bad, a.bad, 4, cudaMemcpyDeviceToHost, s), "read");
  CK(cudaStreamSynchronize(s), "synchronize");
  if (bad) return fail(RPLU_ERR_CUDA, "internal error: split permutation");
  // Algorithm 3 on the Loewner matrix of the split, the CUR-AAA stopping rule
  const int64_t k = std::min(k_max, std::min(nx, ny));
  int64_t *I = nullptr, *J = nullptr;
  void *L = nullptr, *U = nullptr;
  CK(ws.alloc(&I, k * 8), "workspace");
  CK(ws.alloc(&J, k * 8), "workspace");
  CK(ws.alloc(&L, k * nx * 16), "workspace");
  CK(ws.alloc(&U, k * ny * 16), "workspace");
  rplu_opts co = default_opts();
  co.dtype = RPLU_C128;
  co.pivot = o.pivot;
  co.rel_tol = eps;
  co.stream = o.stream;
  co.bound_nu = o.bound_nu != 0.0 ? o.bound_nu : 5.0;
  co.bound_leaf = o.bound_leaf;
  co.bound_stop = 1;
  int64_t kd = 0;
  const rplu_status fst = cauchy_like_call(a.x, a.y, a.G, a.B, nx, ny, 2, k, seed, &co, I, J, L, U, &kd, false);
  if (fst != RPLU_OK && fst != RPLU_NOT_CONVERGED) return fst;  // message set by the call
  if (kd == 0) return fail(RPLU_ERR_INVALID, "the Loewner matrix of the samples is zero (constant f)");
  // the two candidates: rows (X[I]) and columns (Y[J])
  const int64_t M = m - kd;
  const int64_t nrc = std::max<int64_t>(1, (M + kAaaRowChunk - 1) / kAaaRowChunk);
  AaaFit fit;
  std::memset(&fit, 0, sizeof(fit));
  CK(ws.alloc(&fit.rows, M * 8), "workspace");
  CK(ws.alloc(&fit.A, M * kd * 16), "workspace (Loewner matrix)");
  CK(ws.alloc(&fit.part, (int64_t)di.num_sms * 4 * 8), "workspace");
  CK(ws.alloc(&fit.s, kd * 8), "workspace");
  CK(ws.alloc(&fit.rdiag, kd * 16), "workspace");
  CK(ws.alloc(&fit.part2, kd * nrc * 16), "workspace");
  CK(ws.alloc(&fit.sw, kd * 16), "workspace");
  CK(ws.alloc(&fit.y, kd * 16), "workspace");
  CK(ws.alloc(&fit.iters, 4), "workspace");
  int64_t* sup2[2] = {nullptr, nullptr};
  void* w2[2] = {nullptr, nullptr};
  unsigned long long* eb2[2] = {nullptr, nullptr};
  for (int c = 0; c < 2; ++c) {
    CK(ws.alloc(&sup2[c], kd * 8), "workspace");
    CK(ws.alloc(&w2[c], kd * 16), "workspace");
    CK(ws.alloc(&eb2[c], 8), "workspace");
    fit.sup = sup2[c];
    fit.w = w2[c];
    fit.err_bits = eb2[c];
    CK(aaa_fit(a, c == 0 ? I : J, c == 0 ? a.xidx : a.yidx, kd, fit, s), "CUR-AAA fit");
  }
  unsigned long long ebits[2];
  CK(cudaMemcpyAsync(&ebits[0], eb2[0], 8, cudaMemcpyDeviceToHost, s), "read");
  CK(cudaMemcpyAsync(&ebits[1], eb2[1], 8, cudaMemcpyDeviceToHost, s), "read");
  CK(cudaStreamSynchronize(s), "synchronize");
  double e2[2];
  std::memcpy(&e2[0], &ebits[0], 8);
  std::memcpy(&e2[1], &ebits[1], 8);
  const int win = e2[0] < e2[1] ? 0 : 1;
  CK(cudaMemcpyAsync(support, sup2[win], kd * 8, cudaMemcpyDefault, s), "copy support");
  CK(cudaMemcpyAsync(w, w2[win], kd * 16, cudaMemcpyDefault, s), "copy weights");
  CK(cudaStreamSynchronize(s), "synchronize");
  *k_out = kd;
  *which = win;
  err[0] = e2[0];
  err[1] = e2[1];
  return kd == k && k < std::min(nx, ny) ? fail(RPLU_NOT_CONVERGED, "eps not reached within k_max steps") : RPLU_OK;
}

}  // extern "C"

namespace rplu {
namespace {
// Workspace of a grid-wide draw over n weights (zeroed maximum, chunk totals).
cudaError_t alloc_grid_draw(Workspace& ws, int64_t n, int num_sms, GridDraw* g) {
  grid_draw_shape(n, num_sms, &g->chunks, &g->len);
  cudaError_t e = ws.alloc(&g->maxb, 8);
  if (e == cudaSuccess) e = ws.alloc(&g->part, g->chunks * 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->maxb, 0, 8, ws.s);
  return e;
}
}  // namespace
}  // namespace rplu

extern "C" {

rplu_status rplu_toeplitz3_cur(int64_t N, double length, double delta, double sigma, int64_t k, uint64_t seed,
                               const rplu_opts* opts, int64_t* I, int64_t* J, double* core, int64_t* k_done) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2 && o.pivot != RPLU_PIVOT_GIVEN)
    return fail(RPLU_ERR_INVALID, "rplu_toeplitz3_cur takes RPLU_PIVOT_RANDOM, C2 or GIVEN");
  if (N < 1 || N > kToeplitzMaxN) return fail(RPLU_ERR_INVALID, "N must be in 1..640");
  if (!(length > 0.0) || !std::isfinite(length) || !(sigma > 0.0) || !std::isfinite(sigma) || !std::isfinite(delta))
    return fail(RPLU_ERR_INVALID, "length and sigma must be finite and > 0, delta finite");
  const int64_t n = N * N * N;
  if (k < 0 || k > n) return fail(RPLU_ERR_INVALID, "k must be in 0..N^3");
  if (!k_done) return fail(RPLU_ERR_INVALID, "k_done is NULL");
  if (k > 0 && (!I || !J || !core)) return fail(RPLU_ERR_INVALID, "NULL output with k > 0");
  if (!(o.rel_tol >= 0.0) || !std::isfinite(o.rel_tol)) return fail(RPLU_ERR_INVALID, "rel_tol must be finite and >= 0");
  if (o.pivot == RPLU_PIVOT_GIVEN && k > 0 && (!o.given_I || !o.given_J))
    return fail(RPLU_ERR_INVALID, "RPLU_PIVOT_GIVEN needs given_I and given_J");
  *k_done = 0;
  // the 2N - 1 taps of each factor: T1[a, a'] = K1((a - a') h), K1(s) = exp(-(s - delta)^2 / (2 sigma^2)),
  // and T0 likewise without the shift (Eq. kernel is the product of the three)
  const double h = length / (double)N;
  std::vector<double> taps(2 * (2 * N - 1));
  for (int64_t e = 0; e < 2 * N - 1; ++e) {
    const double s_ = (double)(e - (N - 1)) * h;
    taps[e] = std::exp(-((s_ - delta) * (s_ - delta)) / (2.0 * sigma * sigma));
    taps[2 * N - 1 + e] = std::exp(-(s_ * s_) / (2.0 * sigma * sigma));
  }
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  Toeplitz3Launch a;
  std::memset(&a, 0, sizeof(a));
  a.N = (int32_t)N; a.n = n; a.k = k;
  a.seed = seed; a.mode = o.pivot; a.tol = o.rel_tol; a.num_sms = di.num_sms;
  double* dtaps = nullptr;
  CK(ws.alloc(&dtaps, (int64_t)taps.size() * 8), "workspace taps");
  CK(cudaMemcpyAsync(dtaps, taps.data(), taps.size() * 8, cudaMemcpyHostToDevice, s), "copy taps");
  a.t1 = dtaps; a.t0 = dtaps + (2 * N - 1);
  JobState* dst = nullptr;
  CK(ws.alloc(&a.r1d, 2 * N * 8), "workspace");
  CK(ws.alloc(&a.d, n * 8), "workspace d");
  CK(ws.alloc(&a.row_used, n), "workspace");
  CK(ws.alloc(&a.col_used, n), "workspace");
  CK(ws.alloc(&a.rhat, n * 8), "workspace");
  CK(ws.alloc(&a.urow, n * 8), "workspace");
  CK(ws.alloc(&a.lcol, n * 8), "workspace");
  CK(ws.alloc(&a.g, n * 8), "workspace");
  CK(ws.alloc(&a.tmp, n * 8), "workspace");
  CK(alloc_grid_draw(ws, n, di.num_sms, &a.rdraw), "workspace draw");
  CK(alloc_grid_draw(ws, n, di.num_sms, &a.cdraw), "workspace draw");
  CK(ws.alloc(&a.T_hist, (k + 1) * 8), "workspace");
  CK(cudaMemsetAsync(a.T_hist, 0, (k + 1) * 8, s), "memset");
  const int64_t kk = std::max<int64_t>(k, 1);
  CK(ws.alloc(&a.core, kk * kk * 8), "workspace core");
  CK(ws.alloc(&a.core_lo, kk * kk * 8), "workspace core");
  CK(ws.alloc(&a.vb, kk * 8), "workspace");
  CK(ws.alloc(&a.vb_lo, kk * 8), "workspace");
  CK(ws.alloc(&a.ve, kk * 8), "workspace");
  CK(ws.alloc(&a.ve_lo, kk * 8), "workspace");
  CK(ws.alloc(&a.vg, kk * 8), "workspace");
  CK(ws.alloc(&a.vh, kk * 8), "workspace");
  CK(ws.alloc(&dst, (int64_t)sizeof(JobState)), "workspace");
  a.st = dst;
  CK(cudaMemsetAsync(a.row_used, 0, n, s), "memset");
  CK(cudaMemsetAsync(a.col_used, 0, n, s), "memset");
  CK(cudaMemsetAsync(dst, 0, sizeof(JobState), s), "memset");
  Buf bI, bJ, bC, bgI, bgJ;
  CK(bind(ws, bI, I, k * 8, false), "bind I");
  CK(bind(ws, bJ, J, k * 8, false), "bind J");
  CK(bind(ws, bC, core, k * k * 8, false), "bind core");
  if (o.pivot == RPLU_PIVOT_GIVEN) {
    CK(bind(ws, bgI, o.given_I, k * 8, true), "bind given_I");
    CK(bind(ws, bgJ, o.given_J, k * 8, true), "bind given_J");
  }
  if (k > 0) {
    CK(cudaMemsetAsync(bI.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bJ.dev, 0xff, k * 8, s), "memset");
  }
  a.I = (int64_t*)bI.dev; a.J = (int64_t*)bJ.dev;
  a.gI = (const int64_t*)bgI.dev; a.gJ = (const int64_t*)bgJ.dev;

  TimerScope ts(o.prof, s);
  CK(toeplitz3_init(a, s, &ts.tm), "toeplitz init");
  JobState hst;
  std::memset(&hst, 0, sizeof(hst));
  int64_t launched = 0;
  const int64_t max_seq = (int64_t)kMaxAttempts * (k + 1);
  while (k > 0) {
    const int64_t steps = k - hst.t;
    CK(toeplitz3_cur_run(a, s, steps, &ts.tm), "toeplitz CUR kernels");
    launched += steps;
    CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (hst.done || hst.t >= k || launched >= max_seq) break;
  }
  CK(toeplitz3_finish(a, s, &ts.tm), "toeplitz finish");
  CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
  CK(cudaStreamSynchronize(s), "synchronize");
  if (k > 0) CK(toeplitz3_core_out(a.core, k, hst.k_done, (double*)bC.dev, di.num_sms, s), "core out");
  CK(copy_out(bI, s), "copy I");
  CK(copy_out(bJ, s), "copy J");
  CK(copy_out(bC, s), "copy core");
  if (o.T_hist) CK(cudaMemcpyAsync(o.T_hist, a.T_hist, (k + 1) * 8, cudaMemcpyDefault, s), "copy T_hist");
  if (o.d_out) CK(cudaMemcpyAsync(o.d_out, a.d, n * 8, cudaMemcpyDefault, s), "copy d");
  std::vector<double> th(k + 1, 0.0);
  CK(cudaMemcpyAsync(th.data(), a.T_hist, (k + 1) * 8, cudaMemcpyDeviceToHost, s), "read T");
  CK(cudaStreamSynchronize(s), "synchronize");
  ts.report();
  *k_done = hst.k_done;
  return finish_status(hst, o, k, th[hst.k_done]);
}

rplu_status rplu_sparse_cur(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                            int64_t k, uint64_t seed, const rplu_opts* opts, int64_t* I, int64_t* J, double* core,
                            int64_t* k_done) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2 && o.pivot != RPLU_PIVOT_GIVEN)
    return fail(RPLU_ERR_INVALID, "rplu_sparse_cur takes RPLU_PIVOT_RANDOM, C2 or GIVEN");
  if (n < 1 || m < 1 || n >= INT32_MAX || m >= INT32_MAX) return fail(RPLU_ERR_INVALID, "n and m must be in 1..2^31-2");
  if (k < 0 || k > std::min(n, m)) return fail(RPLU_ERR_INVALID, "k must be in 0..min(n, m)");
  if (!row_ptr || !k_done) return fail(RPLU_ERR_INVALID, "NULL pointer");
  if (k > 0 && (!I || !J || !core)) return fail(RPLU_ERR_INVALID, "NULL output with k > 0");
  if (!(o.rel_tol >= 0.0) || !std::isfinite(o.rel_tol)) return fail(RPLU_ERR_INVALID, "rel_tol must be finite and >= 0");
  if (o.pivot == RPLU_PIVOT_GIVEN && k > 0 && (!o.given_I || !o.given_J))
    return fail(RPLU_ERR_INVALID, "RPLU_PIVOT_GIVEN needs given_I and given_J");
  *k_done = 0;
  cudaStream_t s = (cudaStream_t)o.stream;
  // host copies of the CSR arrays (checked, and transposed into CSC here)
  std::vector<int64_t> rp((size_t)n + 1);
  if (on_device(row_ptr)) {
    CK(cudaMemcpyAsync(rp.data(), row_ptr, (n + 1) * 8, cudaMemcpyDeviceToHost, s), "read row_ptr");
    CK(cudaStreamSynchronize(s), "synchronize");
  } else {
    std::memcpy(rp.data(), row_ptr, (size_t)(n + 1) * 8);
  }
  if (rp[0] != 0) return fail(RPLU_ERR_INVALID, "row_ptr[0] must be 0");
  for (int64_t p = 0; p < n; ++p)
    if (rp[(size_t)p + 1] < rp[(size_t)p]) return fail(RPLU_ERR_INVALID, "row_ptr must be nondecreasing");
  const int64_t nnz = rp[(size_t)n];  // the arrays below are read only once row_ptr is known to be sane
  if (nnz > 0 && (!col_idx || !val)) return fail(RPLU_ERR_INVALID, "col_idx or val is NULL");
  std::vector<int32_t> ci((size_t)std::max<int64_t>(nnz, 1));
  std::vector<double> rv((size_t)std::max<int64_t>(nnz, 1));
  if (nnz > 0) {
    bool read_dev = false;
    if (on_device(col_idx)) {
      CK(cudaMemcpyAsync(ci.data(), col_idx, nnz * 4, cudaMemcpyDeviceToHost, s), "read col_idx");
      read_dev = true;
    } else {
      std::memcpy(ci.data(), col_idx, (size_t)nnz * 4);
    }
    if (on_device(val)) {
      CK(cudaMemcpyAsync(rv.data(), val, nnz * 8, cudaMemcpyDeviceToHost, s), "read val");
      read_dev = true;
    } else {
      std::memcpy(rv.data(), val, (size_t)nnz * 8);
    }
    if (read_dev) CK(cudaStreamSynchronize(s), "synchronize");
  }
  const char* bad = csr_check(n, m, rp.data(), ci.data(), rv.data());
  if (bad[0]) return fail(RPLU_ERR_INVALID, bad);
  // CSC by a stable counting sort: rows ascend within each column
  std::vector<int64_t> cp;
  std::vector<int32_t> ri;
  std::vector<double> cv;
  csr_to_csc(n, m, rp.data(), ci.data(), rv.data(), cp, ri, cv);
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  Workspace ws(s);
  SparseCurLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.m = m; a.k = k;
  a.seed = seed; a.mode = o.pivot; a.tol = o.rel_tol; a.num_sms = di.num_sms;
  const int64_t nz1 = std::max<int64_t>(nnz, 1);
  int64_t *drp = nullptr, *dcp = nullptr;
  int32_t *dci = nullptr, *dri = nullptr;
  double *drv = nullptr, *dcv = nullptr;
  CK(ws.alloc(&drp, (n + 1) * 8), "workspace CSR");
  CK(ws.alloc(&dci, nz1 * 4), "workspace CSR");
  CK(ws.alloc(&drv, nz1 * 8), "workspace CSR");
  CK(ws.alloc(&dcp, (m + 1) * 8), "workspace CSC");
  CK(ws.alloc(&dri, nz1 * 4), "workspace CSC");
  CK(ws.alloc(&dcv, nz1 * 8), "workspace CSC");
  CK(cudaMemcpyAsync(drp, rp.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s), "copy CSR");
  CK(cudaMemcpyAsync(dci, ci.data(), nz1 * 4, cudaMemcpyHostToDevice, s), "copy CSR");
  CK(cudaMemcpyAsync(drv, rv.data(), nz1 * 8, cudaMemcpyHostToDevice, s), "copy CSR");
  CK(cudaMemcpyAsync(dcp, cp.data(), (m + 1) * 8, cudaMemcpyHostToDevice, s), "copy CSC");
  CK(cudaMemcpyAsync(dri, ri.data(), nz1 * 4, cudaMemcpyHostToDevice, s), "copy CSC");
  CK(cudaMemcpyAsync(dcv, cv.data(), nz1 * 8, cudaMemcpyHostToDevice, s), "copy CSC");
  a.rp = drp; a.ci = dci; a.rv = drv; a.cp = dcp; a.ri = dri; a.cv = dcv;
  // how the kernels walk the rows and the columns: G lanes per short one, a CTA per long one
  std::vector<int32_t> lrows, lcols;
  a.row_lanes = segment_lanes(n, rp.data(), kSpLongDeg, lrows);
  a.col_lanes = segment_lanes(m, cp.data(), kSpLongDeg, lcols);
  int32_t *dlr = nullptr, *dlc = nullptr;
  CK(ws.alloc(&dlr, std::max<int64_t>((int64_t)lrows.size(), 1) * 4), "workspace long rows");
  CK(ws.alloc(&dlc, std::max<int64_t>((int64_t)lcols.size(), 1) * 4), "workspace long columns");
  if (!lrows.empty())
    CK(cudaMemcpyAsync(dlr, lrows.data(), lrows.size() * 4, cudaMemcpyHostToDevice, s), "copy long rows");
  if (!lcols.empty())
    CK(cudaMemcpyAsync(dlc, lcols.data(), lcols.size() * 4, cudaMemcpyHostToDevice, s), "copy long columns");
  a.long_rows = dlr; a.n_long_rows = (int64_t)lrows.size();
  a.long_cols = dlc; a.n_long_cols = (int64_t)lcols.size();
  JobState* dst = nullptr;
  CK(ws.alloc(&a.d, n * 8), "workspace d");
  CK(ws.alloc(&a.row_used, n), "workspace");
  CK(ws.alloc(&a.col_used, m), "workspace");
  CK(ws.alloc(&a.rhat, m * 8), "workspace");
  CK(ws.alloc(&a.urow, m * 8), "workspace");
  CK(ws.alloc(&a.ccol, n * 8), "workspace");
  CK(ws.alloc(&a.row_piv, n * 4), "workspace");
  CK(ws.alloc(&a.col_piv, m * 4), "workspace");
  CK(cudaMemsetAsync(a.row_piv, 0xff, n * 4, s), "memset");  // -1: not a pivot
  CK(cudaMemsetAsync(a.col_piv, 0xff, m * 4, s), "memset");
  CK(alloc_grid_draw(ws, n, di.num_sms, &a.rdraw), "workspace draw");
  CK(alloc_grid_draw(ws, m, di.num_sms, &a.cdraw), "workspace draw");
  CK(ws.alloc(&a.lcol, n * 8), "workspace");
  CK(ws.alloc(&a.g, n * 8), "workspace");
  CK(ws.alloc(&a.T_hist, (k + 1) * 8), "workspace");
  CK(cudaMemsetAsync(a.T_hist, 0, (k + 1) * 8, s), "memset");
  const int64_t kk = std::max<int64_t>(k, 1);
  CK(ws.alloc(&a.core, kk * kk * 8), "workspace core");
  CK(ws.alloc(&a.core_lo, kk * kk * 8), "workspace core");
  CK(ws.alloc(&a.vb, kk * 8), "workspace");
  CK(ws.alloc(&a.vb_lo, kk * 8), "workspace");
  CK(ws.alloc(&a.ve, kk * 8), "workspace");
  CK(ws.alloc(&a.ve_lo, kk * 8), "workspace");
  CK(ws.alloc(&a.vg, kk * 8), "workspace");
  CK(ws.alloc(&a.vh, kk * 8), "workspace");
  CK(ws.alloc(&dst, (int64_t)sizeof(JobState)), "workspace");
  a.st = dst;
  CK(cudaMemsetAsync(a.row_used, 0, n, s), "memset");
  CK(cudaMemsetAsync(a.col_used, 0, m, s), "memset");
  CK(cudaMemsetAsync(dst, 0, sizeof(JobState), s), "memset");
  Buf bI, bJ, bC, bgI, bgJ;
  CK(bind(ws, bI, I, k * 8, false), "bind I");
  CK(bind(ws, bJ, J, k * 8, false), "bind J");
  CK(bind(ws, bC, core, k * k * 8, false), "bind core");
  if (o.pivot == RPLU_PIVOT_GIVEN) {
    CK(bind(ws, bgI, o.given_I, k * 8, true), "bind given_I");
    CK(bind(ws, bgJ, o.given_J, k * 8, true), "bind given_J");
  }
  if (k > 0) {
    CK(cudaMemsetAsync(bI.dev, 0xff, k * 8, s), "memset");
    CK(cudaMemsetAsync(bJ.dev, 0xff, k * 8, s), "memset");
  }
  a.I = (int64_t*)bI.dev; a.J = (int64_t*)bJ.dev;
  a.gI = (const int64_t*)bgI.dev; a.gJ = (const int64_t*)bgJ.dev;

  TimerScope ts(o.prof, s);
  CK(sparse_cur_init(a, s, &ts.tm), "sparse init");
  JobState hst;
  std::memset(&hst, 0, sizeof(hst));
  int64_t launched = 0;
  const int64_t max_seq = (int64_t)kMaxAttempts * (k + 1);
  while (k > 0) {
    const int64_t steps = k - hst.t;
    CK(sparse_cur_run(a, s, steps, &ts.tm), "sparse CUR kernels");
    launched += steps;
    CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (hst.done || hst.t >= k || launched >= max_seq) break;
  }
  CK(sparse_cur_finish(a, s, &ts.tm), "sparse finish");
  CK(cudaMemcpyAsync(&hst, dst, sizeof(JobState), cudaMemcpyDeviceToHost, s), "read state");
  CK(cudaStreamSynchronize(s), "synchronize");
  if (k > 0) CK(toeplitz3_core_out(a.core, k, hst.k_done, (double*)bC.dev, di.num_sms, s), "core out");
  CK(copy_out(bI, s), "copy I");
  CK(copy_out(bJ, s), "copy J");
  CK(copy_out(bC, s), "copy core");
  if (o.T_hist) CK(cudaMemcpyAsync(o.T_hist, a.T_hist, (k + 1) * 8, cudaMemcpyDefault, s), "copy T_hist");
  if (o.d_out) CK(cudaMemcpyAsync(o.d_out, a.d, n * 8, cudaMemcpyDefault, s), "copy d");
  std::vector<double> th(k + 1, 0.0);
  CK(cudaMemcpyAsync(th.data(), a.T_hist, (k + 1) * 8, cudaMemcpyDeviceToHost, s), "read T");
  CK(cudaStreamSynchronize(s), "synchronize");
  ts.report();
  *k_done = hst.k_done;
  return finish_status(hst, o, k, th[hst.k_done]);
}

rplu_status rplu_barycentric(const void* t, const void* ft, const void* w, int64_t k, const void* zq, int64_t nq,
                             const rplu_opts* opts, void* rq) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  if (k < 1 || nq < 0) return fail(RPLU_ERR_INVALID, "k must be >= 1 and nq >= 0");
  if (!t || !ft || !w || (nq > 0 && (!zq || !rq))) return fail(RPLU_ERR_INVALID, "NULL pointer");
  DeviceInfo di;
  CK(device_info(&di), "device set-up");
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  Buf bt, bf, bw, bz, br;
  CK(bind(ws, bt, t, k * 16, true), "bind t");
  CK(bind(ws, bf, ft, k * 16, true), "bind ft");
  CK(bind(ws, bw, w, k * 16, true), "bind w");
  CK(bind(ws, bz, zq, nq * 16, true), "bind zq");
  CK(bind(ws, br, rq, nq * 16, false), "bind rq");
  CK(aaa_query(bt.dev, bf.dev, bw.dev, k, bz.dev, nq, br.dev, di.num_sms, s), "barycentric kernel");
  CK(copy_out(br, s), "copy rq");
  CK(cudaStreamSynchronize(s), "synchronize");
  return RPLU_OK;
}

rplu_status rplu_bh_plan_stats(const void* x, const void* y, int64_t n, int64_t m, double nu, int64_t leaf,
                               const rplu_opts* opts, int64_t* stats) {
  g_last_error.clear();
  const rplu_opts o = opts ? *opts : default_opts();
  if (dtype_bytes(o.dtype) < 0) return fail(RPLU_ERR_INVALID, "unknown dtype");
  if (n < 1 || m < 1) return fail(RPLU_ERR_INVALID, "n and m must be >= 1");
  if (!x || !y || !stats) return fail(RPLU_ERR_INVALID, "NULL pointer");
  rplu_status st0 = check_bound_args(nu, leaf, n, m);
  if (st0 != RPLU_OK) return st0;
  cudaStream_t s = (cudaStream_t)o.stream;
  Workspace ws(s);
  const int64_t w = dtype_bytes(o.dtype);
  Buf bx, by;
  CK(bind(ws, bx, x, n * w, true), "bind x");
  CK(bind(ws, by, y, m * w, true), "bind y");
  std::vector<double> xr, xi, yr, yi;
  CK(points_host(bx.dev, n, o.dtype, s, xr, xi), "read points");
  CK(points_host(by.dev, m, o.dtype, s, yr, yi), "read points");
  BhPlan plan;
  bh_make_plan(plan, xr.data(), xi.data(), n, yr.data(), yi.data(), m, nu, leaf);
  int64_t leaves = 0, exact = 0, tmax = 0;
  for (const BhNode& nd : plan.src.nodes) leaves += nd.leaf ? 1 : 0;
  for (size_t l = 0; l < plan.tleaf.size(); ++l) {
    const BhNode& tl = plan.tgt.nodes[(size_t)plan.tleaf[l]];
    int64_t src = 0;
    for (int64_t e = plan.e_off[l]; e < plan.e_off[l + 1]; ++e) {
      const BhNode& sn = plan.src.nodes[(size_t)plan.e_node[(size_t)e]];
      src += sn.hi - sn.lo;
    }
    exact += (tl.hi - tl.lo) * src;
    tmax = std::max<int64_t>(tmax, tl.hi - tl.lo);
  }
  stats[0] = (int64_t)plan.tleaf.size();
  stats[1] = (int64_t)plan.src.nodes.size();
  stats[2] = leaves;
  stats[3] = (int64_t)plan.a_node.size();
  stats[4] = exact;
  stats[5] = tmax;
  CK(cudaStreamSynchronize(s), "synchronize");
  return RPLU_OK;
}

}  // extern "C"
