// rplu_dense_noalloc: the dense-form factorization without any memory
// allocation by the library.
//
// Some callers cannot let a library allocate device memory: code that runs
// while a framework owns the whole device through its own pooled allocator
// (a raw cudaMalloc there fails or fragments the pool), real-time or embedded
// services that reserve every byte at start-up and forbid allocation
// afterwards, and hosts that must not trigger the device-wide
// synchronisation that cudaMalloc/cudaFree can imply.  For them this entry
// point takes its working memory from one fixed array compiled into the
// library.
//
// The array holds kNoAllocBytes bytes on every GPU that loads the library, for
// the life of the process.  All calls share it, so calls whose GPU work
// overlaps (for example on two streams at once) corrupt each other: issue them
// on one stream or synchronise between them.  Each call clears the parts that
// must start at zero.  The first call on a device looks up the array's device
// address with cudaGetSymbolAddress (a host-side symbol is not a device
// address); make that first call before any stream capture begins.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "rplu.h"

namespace rplu {
namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;  // 32 MiB per GPU

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_na_mu;
std::vector<void*> g_na_base;  // per device: device address of g_noalloc_scratch
std::vector<int> g_na_sms;

// Failures are reported by status code only (the reason is in the comment at
// each call site).
rplu_status na_fail(rplu_status s, const char*) { return s; }

// One-time per-device set-up, with that device current.
cudaError_t na_setup(void** base, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if ((int)g_na_base.size() <= dev) {
    g_na_base.resize(dev + 1, nullptr);
    g_na_sms.resize(dev + 1, 0);
  }
  if (!g_na_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n_sms = 0;
    e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_na_base[dev] = p;
    g_na_sms[dev] = n_sms;
  }
  *base = g_na_base[dev];
  *sms = g_na_sms[dev];
  return cudaSuccess;
}

bool na_on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Bump carving of the fixed array, 256-byte aligned pieces.
struct Carve {
  unsigned char* base;
  size_t off = 0;
  bool ok = true;
  template <typename P>
  P* take(size_t bytes) {
    const size_t a = (off + 255) & ~(size_t)255;
    if (a + bytes > kNoAllocBytes) {
      ok = false;
      return nullptr;
    }
    off = a + bytes;
    return (P*)(base + a);
  }
};

}  // namespace
}  // namespace rplu

using namespace rplu;

extern "C" rplu_status rplu_dense_noalloc(const void* A, int64_t n, int64_t m, int64_t k, uint64_t seed,
                                          const rplu_opts* opts, int64_t* I, int64_t* J, void* L, void* U,
                                          int64_t* k_done) {
  rplu_opts o;
  if (opts) o = *opts;
  else rplu_opts_init(&o);
  const int64_t w = o.dtype == RPLU_F32 ? 4 : o.dtype == RPLU_F64 ? 8 : o.dtype == RPLU_C64 ? 8 :
                    o.dtype == RPLU_C128 ? 16 : -1;
  if (w < 0) return na_fail(RPLU_ERR_INVALID, "unknown dtype");
  if (o.pivot < RPLU_PIVOT_RANDOM || o.pivot > RPLU_PIVOT_GIVEN) return na_fail(RPLU_ERR_INVALID, "unknown pivot");
  if (!k_done) return na_fail(RPLU_ERR_INVALID, "k_done is NULL");
  if (n < 0 || m < 0 || k < 0 || k > (n < m ? n : m)) return na_fail(RPLU_ERR_INVALID, "bad sizes");
  if (n > ((int64_t)1 << 31) || m > ((int64_t)1 << 31)) return na_fail(RPLU_ERR_NOMEM, "far beyond the fixed array");
  if (!(o.rel_tol >= 0.0)) return na_fail(RPLU_ERR_INVALID, "rel_tol must be >= 0");
  if (o.pivot == RPLU_PIVOT_COMPLETE && o.rel_tol > 0.0) return na_fail(RPLU_ERR_INVALID, "COMPLETE takes no rel_tol");
  const int64_t lda = o.lda ? o.lda : m;
  if (lda < m) return na_fail(RPLU_ERR_INVALID, "lda < m");
  *k_done = 0;
  if (n * m > 0 && !na_on_device(A)) return na_fail(RPLU_ERR_INVALID, "A must be device memory");
  if (k > 0 && (!na_on_device(I) || !na_on_device(J) || !na_on_device(L) || !na_on_device(U)))
    return na_fail(RPLU_ERR_INVALID, "I, J, L and U must be device memory");
  if (o.pivot == RPLU_PIVOT_GIVEN && k > 0 && (!na_on_device(o.given_I) || !na_on_device(o.given_J)))
    return na_fail(RPLU_ERR_INVALID, "given pivots must be device memory");

  void* base = nullptr;
  int sms = 0;
  cudaError_t e = na_setup(&base, &sms);
  if (e != cudaSuccess) return na_fail(RPLU_ERR_CUDA, "scratch set-up");
  cudaStream_t s = (cudaStream_t)o.stream;

  const int64_t V = 16 / w;
  int32_t blk = o.pass_block;
  if (blk <= 0) blk = default_pass_block(o.dtype);
  if (blk > 8) return na_fail(RPLU_ERR_INVALID, "pass_block must be at most 8");
  if (o.pivot == RPLU_PIVOT_COMPLETE) blk = 1;

  DenseLaunch a;
  std::memset(&a, 0, sizeof(a));
  a.n = n; a.m = m; a.k = k; a.seed = seed; a.mode = o.pivot; a.tol = o.rel_tol; a.num_sms = sms;
  a.blk = blk;
  a.lds = (m + V - 1) / V * V;
  if (a.lds == 0) a.lds = V;
  Carve c{(unsigned char*)base};
  a.S = c.take<unsigned char>((size_t)(n * a.lds * w));
  a.d = c.take<double>((size_t)(n > 0 ? n : 1) * 8);
  a.row_used = c.take<uint8_t>((size_t)(n > 0 ? n : 1));
  a.col_used = c.take<uint8_t>((size_t)(m > 0 ? m : 1));
  a.ublk = c.take<unsigned char>((size_t)(blk * a.lds * w));
  a.T_hist = c.take<double>((size_t)(k + 1) * 8);
  a.st = c.take<JobState>(sizeof(JobState));
  if (o.pivot == RPLU_PIVOT_COMPLETE) {
    a.rowmax = c.take<double>((size_t)(n > 0 ? n : 1) * 8);
    a.rowarg = c.take<int64_t>((size_t)(n > 0 ? n : 1) * 8);
  }
  if (!c.ok) return na_fail(RPLU_ERR_NOMEM, "workspace exceeds the fixed array");
  a.A = A;
  a.lda = lda;
  a.L = L; a.U = U; a.I = I; a.J = J;
  a.gI = o.given_I; a.gJ = o.given_J;

#define NA_CK(expr)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return na_fail(RPLU_ERR_CUDA, #expr);                             \
  } while (0)
  if (n > 0) NA_CK(cudaMemsetAsync(a.row_used, 0, (size_t)n, s));
  if (m > 0) NA_CK(cudaMemsetAsync(a.col_used, 0, (size_t)m, s));
  NA_CK(cudaMemsetAsync(a.st, 0, sizeof(JobState), s));
  if (k > 0) {
    NA_CK(cudaMemsetAsync(I, 0xff, (size_t)k * 8, s));
    NA_CK(cudaMemsetAsync(J, 0xff, (size_t)k * 8, s));
    NA_CK(cudaMemsetAsync(L, 0, (size_t)(n * k * w), s));
    NA_CK(cudaMemsetAsync(U, 0, (size_t)(k * m * w), s));
  }
  HotTimer tm;  // off: no events
  NA_CK(dense_run(o.dtype, a, s, &tm));
  if (o.T_hist) NA_CK(cudaMemcpyAsync(o.T_hist, a.T_hist, (size_t)(k + 1) * 8, cudaMemcpyDefault, s));
  if (o.d_out && n > 0) NA_CK(cudaMemcpyAsync(o.d_out, a.d, (size_t)n * 8, cudaMemcpyDefault, s));
  JobState hst;
  double Tfin = 0.0;
  NA_CK(cudaMemcpyAsync(&hst, a.st, sizeof(JobState), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (hst.k_done >= 0 && hst.k_done <= k)
    NA_CK(cudaMemcpy(&Tfin, a.T_hist + hst.k_done, 8, cudaMemcpyDeviceToHost));
#undef NA_CK
  *k_done = hst.k_done;
  const char* why = "";
  return job_status(hst, o.rel_tol, k, Tfin, &why);
}

