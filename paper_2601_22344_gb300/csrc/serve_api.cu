// Serving session (include/rplu.h): continuous batching of RPLU requests.
//
// Requests are queued by rplu_session_submit.  A worker thread admits them in
// arrival order as device memory (a session arena with a first-fit allocator,
// arena.h) and ring slots allow: it copies the inputs into the arena, writes
// the job descriptor into a ring in host-mapped memory and publishes it.  One
// persistent serving kernel (k_serve, batch.cu) serves every request type --
// FP32 and complex64, dense and Cauchy -- and claims published jobs in
// arrival order while it runs, so requests that arrive while others are on
// the GPU start as soon as a CTA frees up; CTAs that stay idle exit, and the
// worker launches CTAs in their place when published work waits.
// Completions are seen through per-slot sequence numbers in mapped memory;
// the factors stay in the arena until the caller fetches or releases them.
// Cauchy requests run in the generator form, whose shared memory grows only
// with n + m, so the kernel takes them up to cauchy_max_dim (4096); dense
// requests up to max_dim.  Larger requests run one at a time per
// large-request stream, concurrently with the kernel, with their memory taken
// from the same arena: dense ones through rplu_dense, Cauchy ones through
// rplu_cauchy_like with unit generators (exact row norms each step, the
// residual never stored).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "batch.h"
#include "common.cuh"
#include "rplu.h"

namespace rplu {
namespace {

constexpr int kServeMaxBlk = 6;
constexpr int32_t kServeMaxDim = 4096;
constexpr int kLaunches = 32;  // launches of the serving kernel that may be live at once (a stream each)
int64_t elem_w(int32_t dtype) { return dtype == RPLU_C64 ? 8 : 4; }
// rows padded to the kernels' 16-byte vectors
int64_t pad_row(int64_t m, int64_t w) { return std::max<int64_t>((m + 16 / w - 1) / (16 / w) * (16 / w), 16 / w); }

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Block {
  int64_t off = -1, bytes = 0;
};

struct Ticket {
  int64_t id = 0;
  rplu_request req{};
  int32_t state = RPLU_TICKET_QUEUED;
  bool big = false;
  int64_t w = 4;  // element bytes: 4 FP32, 8 complex64
  long long h = -1;  // ring ticket
  int64_t slot = -1;
  Block in, out, ws;
  char* in_p = nullptr;
  char* out_p = nullptr;
  char* ws_p = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int32_t status = RPLU_OK;
  int64_t k_done = 0;
  double rel_res = NAN;
  bool cancel_req = false;
};

// Unit generators (G = B = 1, p = 1) for a plain Cauchy request run through
// the generator form: n + m ones of the request's type.
__global__ void k_fill_ones(float* v, int64_t count, int complex_) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    if (complex_) {
      v[2 * e] = 1.f;
      v[2 * e + 1] = 0.f;
    } else {
      v[e] = 1.f;
    }
  }
}

// One launch of the persistent kernel (several may run at once on the ring).
struct Launch {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  bool live = false;
  int grid = 0;
};

// The persistent kernel's ring of job descriptors.
struct Ring {
  BatchDesc* ring_h = nullptr;
  BatchDesc* ring_d = nullptr;
  long long* tail_h = nullptr;
  long long* tail_d = nullptr;
  int64_t* done_h = nullptr;
  int64_t* done_d = nullptr;
  int32_t* cancel_h = nullptr;
  int32_t* cancel_d = nullptr;
  long long* head_d = nullptr;
  std::vector<int64_t> slot_owner;
  long long published = 0;
  int64_t* claimed_h = nullptr;  // per slot: ticket + 1 once claimed by a CTA
  int64_t* claimed_d = nullptr;
  int32_t* exited_h = nullptr;   // kLaunches x grid: per CTA of each launch, 1 once exited
  int32_t* exited_d = nullptr;
  Launch run[kLaunches];
  bool admitted = false;  // published since the last tail store
  BatchArgs args{};
  int grid = 0;
};

}  // namespace
}  // namespace rplu

using namespace rplu;

struct rplu_session {
  rplu_session_opts o{};
  int dev = 0, sms = 0;
  char* base = nullptr;
  Arena arena;
  int64_t cap = 0;
  Ring ring;
  int32_t* stop_h = nullptr;
  int32_t* stop_d = nullptr;
  cudaStream_t s_copy = nullptr;
  std::vector<cudaStream_t> s_big;
  long long idle_cycles = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::unordered_map<int64_t, Ticket> tk;
  std::deque<int64_t> queue, big_queue;
  std::deque<int64_t> completions;  // finished tickets not yet reported by rplu_session_completed
  std::vector<int64_t> on_gpu;
  std::thread worker;
  std::vector<std::thread> big_workers;
  std::atomic<bool> quit{false};
  int64_t next_id = 1;
  int64_t launches = 0, completed = 0, big_completed = 0, cancelled = 0;
  int64_t big_running = 0;

  ~rplu_session();
  bool fits_kernel(const rplu_request& r) const {
    if (r.kind == 1) return r.n <= o.cauchy_max_dim && r.m <= o.cauchy_max_dim;
    return r.n <= o.max_dim && r.m <= o.max_dim && r.n * r.m <= o.dense_kernel_cells;
  }
  bool try_admit(Ticket& t);
  void harvest();
  void maybe_launch();
  void work();
  void big_work(cudaStream_t sb);
  void free_blocks(Ticket& t);
};

namespace {

bool alloc_block(Arena& a, Block& b, int64_t bytes) {
  b.bytes = bytes;
  b.off = bytes > 0 ? a.alloc(bytes) : -1;
  return bytes <= 0 || b.off >= 0;
}

const char* request_invalid(const rplu_request& r) {
  if (r.kind != 0 && r.kind != 1) return "request kind must be 0 (dense) or 1 (Cauchy)";
  if (r.dtype != RPLU_F32 && r.dtype != RPLU_C64) return "served requests are RPLU_F32 or RPLU_C64";
  if (r.n <= 0 || r.m <= 0 || r.k_max < 0 || r.k_max > std::min(r.n, r.m)) return "bad sizes";
  if (!(r.rel_tol >= 0.0) || !std::isfinite(r.rel_tol)) return "rel_tol must be finite and >= 0";
  if (r.kind == 0 && (!r.A || (r.lda != 0 && r.lda < r.m))) return "dense request needs A (lda >= m)";
  if (r.kind == 1 && (!r.x || !r.y)) return "Cauchy request needs x and y";
  return nullptr;
}

}  // namespace

void rplu_session::free_blocks(Ticket& t) {
  if (t.in.off >= 0) arena.release(t.in.off, t.in.bytes);
  if (t.out.off >= 0) arena.release(t.out.off, t.out.bytes);
  if (t.ws.off >= 0) arena.release(t.ws.off, t.ws.bytes);
  t.in = t.out = t.ws = Block{};
}

// Small path: inputs, outputs and (if the job may outlive one write-back
// block) the residual workspace in the arena, then a slot of the ring.
bool rplu_session::try_admit(Ticket& t) {
  const rplu_request& r = t.req;
  Ring& L = ring;
  const int64_t w = t.w;
  const int64_t n = r.n, m = r.m, k = r.k_max, ldp = pad_row(m, w);
  if (L.slot_owner[L.published % cap] >= 0) return false;  // ring slot still busy
  const int64_t in_bytes = r.kind == 0 ? n * ldp * w : Arena::round_up(n * w) + m * w;
  const int64_t kk = std::max<int64_t>(k, 1);
  const int64_t out_bytes = 2 * Arena::round_up(kk * 8) + Arena::round_up(n * kk * w) + kk * m * w;
  const int64_t ws_bytes = r.kind == 0 && k > L.args.blk ? n * ldp * w : 0;  // Cauchy: generator form
  if (!alloc_block(arena, t.in, in_bytes) || !alloc_block(arena, t.out, out_bytes) ||
      !alloc_block(arena, t.ws, ws_bytes)) {
    free_blocks(t);
    return false;
  }
  t.in_p = base + t.in.off;
  t.out_p = base + t.out.off;
  t.ws_p = t.ws.off >= 0 ? base + t.ws.off : nullptr;
  BatchDesc d;
  std::memset(&d, 0, sizeof(d));
  d.n = n; d.m = m; d.k_max = k; d.tol = r.rel_tol; d.seed = r.seed; d.kind = r.kind; d.dtype = r.dtype;
  if (r.kind == 0) {
    const int64_t lda = r.lda ? r.lda : m;
    cudaMemcpy2DAsync(t.in_p, ldp * w, r.A, lda * w, m * w, n, cudaMemcpyDefault, s_copy);
    d.A = t.in_p;
    d.lda = ldp;
  } else {
    cudaMemcpyAsync(t.in_p, r.x, n * w, cudaMemcpyDefault, s_copy);
    cudaMemcpyAsync(t.in_p + Arena::round_up(n * w), r.y, m * w, cudaMemcpyDefault, s_copy);
    d.x = t.in_p;
    d.y = t.in_p + Arena::round_up(n * w);
    d.lda = m;
  }
  char* p = t.out_p;
  d.I = (int64_t*)p;
  p += Arena::round_up(kk * 8);
  d.J = (int64_t*)p;
  p += Arena::round_up(kk * 8);
  d.L = p;
  p += Arena::round_up(n * kk * w);
  d.U = p;
  d.S = t.ws_p;
  d.lds = ldp;
  const int64_t slot = L.published % cap;
  t.h = L.published;
  t.slot = slot;
  L.slot_owner[slot] = t.id;
  L.ring_h[slot] = d;
  __atomic_store_n(&L.cancel_h[slot], 0, __ATOMIC_RELAXED);
  __atomic_store_n(&L.done_h[slot], (int64_t)0, __ATOMIC_RELAXED);
  ++L.published;
  L.admitted = true;
  t.state = RPLU_TICKET_RUNNING;
  t.t_admit = now_s();
  on_gpu.push_back(t.id);
  return true;
}

void rplu_session::harvest() {
  for (size_t q = 0; q < on_gpu.size();) {
    Ticket& t = tk[on_gpu[q]];
    Ring& L = ring;
    const int64_t v = __atomic_load_n(&L.done_h[t.slot], __ATOMIC_ACQUIRE);
    if (v != (int64_t)(t.h + 1)) {
      ++q;
      continue;
    }
    const BatchDesc& d = L.ring_h[t.slot];
    t.k_done = d.k_done;
    t.rel_res = d.T0 > 0.0 ? std::sqrt(std::max(d.T_final, 0.0) / d.T0) : 0.0;
    if (d.err & kErrCancelled) {
      t.status = RPLU_CANCELLED;
      t.state = RPLU_TICKET_CANCELLED;
      ++cancelled;
    } else {
      if (d.err) t.status = RPLU_ERR_INVALID, t.rel_res = NAN;
      else if (t.req.rel_tol > 0.0 && d.k_done == t.req.k_max && t.req.k_max > 0 &&
               d.T_final > t.req.rel_tol * t.req.rel_tol * d.T0)
        t.status = RPLU_NOT_CONVERGED;
      else t.status = RPLU_OK;
      t.state = RPLU_TICKET_DONE;
    }
    t.t_done = now_s();
    L.slot_owner[t.slot] = -1;
    // inputs and workspace are free again; the factors stay until fetched
    if (t.in.off >= 0) arena.release(t.in.off, t.in.bytes);
    if (t.ws.off >= 0) arena.release(t.ws.off, t.ws.bytes);
    t.in = t.ws = Block{};
    ++completed;
    completions.push_back(t.id);
    on_gpu[q] = on_gpu.back();
    on_gpu.pop_back();
  }
}

// CTAs leave the kernel when they find no ticket for idle_us, so the CTAs of
// a launch may thin out while it still runs.  Published tickets that no CTA
// has claimed while fewer CTAs than the full grid remain get a new launch (on
// another stream, so that it runs beside the old ones) of as many CTAs as have
// exited; with no launch live, a full grid.
void rplu_session::maybe_launch() {
  Ring& L = ring;
  int remaining = 0, free_launch = -1;
  for (int li = 0; li < kLaunches; ++li) {
    Launch& r = L.run[li];
    if (r.live && cudaEventQuery(r.ev) == cudaSuccess) r.live = false;
    if (!r.live) {
      if (free_launch < 0) free_launch = li;
      continue;
    }
    const int32_t* ex = L.exited_h + (int64_t)li * L.grid;
    int gone = 0;
    for (int b = 0; b < r.grid; ++b) gone += __atomic_load_n(ex + b, __ATOMIC_ACQUIRE);
    remaining += r.grid - gone;
  }
  if (on_gpu.empty() || remaining >= L.grid || free_launch < 0) return;
  bool unclaimed = false;
  for (int64_t id : on_gpu) {
    const Ticket& t = tk[id];
    if (__atomic_load_n(&L.claimed_h[t.slot], __ATOMIC_ACQUIRE) != (int64_t)(t.h + 1)) {
      unclaimed = true;
      break;
    }
  }
  if (!unclaimed) return;
  Launch& r = L.run[free_launch];
  r.grid = L.grid - remaining;
  int32_t* ex = L.exited_h + (int64_t)free_launch * L.grid;
  for (int b = 0; b < r.grid; ++b) __atomic_store_n(ex + b, 0, __ATOMIC_RELAXED);
  std::atomic_thread_fence(std::memory_order_seq_cst);
  ServeRing q;
  q.desc = L.ring_d;
  q.tail = L.tail_d;
  q.head = L.head_d;
  q.done = L.done_d;
  q.cancel = L.cancel_d;
  q.stop = stop_d;
  q.claimed = L.claimed_d;
  q.exited = L.exited_d + (int64_t)free_launch * L.grid;
  q.cap = cap;
  q.idle_cycles = idle_cycles;
  if (serve_launch(L.args, q, r.grid, r.s) == cudaSuccess) {
    cudaEventRecord(r.ev, r.s);
    r.live = true;
    ++launches;
  }
}

void rplu_session::work() {
  cudaSetDevice(dev);
  std::unique_lock<std::mutex> lk(mu);
  while (!quit.load()) {
    harvest();
    // admit in arrival order while memory and ring slots allow
    bool admitted = false;
    while (!queue.empty()) {
      Ticket& t = tk[queue.front()];
      if (!try_admit(t)) break;
      queue.pop_front();
      admitted = true;
    }
    if (admitted) {
      // inputs complete before the jobs become visible to the kernels
      cudaStreamSynchronize(s_copy);
      if (ring.admitted) {
        __atomic_store_n(ring.tail_h, ring.published, __ATOMIC_RELEASE);
        ring.admitted = false;
      }
    }
    maybe_launch();
    cv.notify_all();
    cv.wait_for(lk, std::chrono::microseconds(40));
  }
}

// Requests above the kernels' size limit, one at a time per stream: dense ones
// through rplu_dense (the arena copy of A serving as the residual,
// overwrite_input), Cauchy ones through rplu_cauchy_like with unit generators
// (G = B = 1): the residual is never stored; the row norms are exact, or with
// bound_nu the rows are drawn by Algorithm 3 against Barnes-Hut bounds, and
// ||A||_F^2 for the request's rel_res comes from a zero-step exact-norm call.
void rplu_session::big_work(cudaStream_t s_big) {
  cudaSetDevice(dev);
  std::unique_lock<std::mutex> lk(mu);
  while (!quit.load()) {
    if (big_queue.empty()) {
      cv.wait_for(lk, std::chrono::microseconds(200));
      continue;
    }
    Ticket& t = tk[big_queue.front()];
    const rplu_request r = t.req;
    const int64_t w = t.w;
    const int64_t n = r.n, m = r.m, k = r.k_max, ldp = pad_row(m, w), kk = std::max<int64_t>(k, 1);
    const int64_t in_bytes = r.kind == 0 ? n * ldp * w
                                         : 2 * (Arena::round_up(n * w) + Arena::round_up(m * w));
    const int64_t out_bytes = 2 * Arena::round_up(kk * 8) + Arena::round_up(n * kk * w) + kk * m * w;
    if (Arena::round_up(in_bytes) + Arena::round_up(out_bytes) > arena.size()) {
      t.status = RPLU_ERR_NOMEM;
      t.state = RPLU_TICKET_DONE;
      t.t_done = now_s();
      completions.push_back(t.id);
      big_queue.pop_front();
      ++completed;
      cv.notify_all();
      continue;
    }
    if (!alloc_block(arena, t.in, in_bytes) || !alloc_block(arena, t.out, out_bytes)) {
      free_blocks(t);
      cv.wait_for(lk, std::chrono::microseconds(200));  // wait for memory
      continue;
    }
    big_queue.pop_front();
    t.state = RPLU_TICKET_RUNNING;
    t.t_admit = now_s();
    ++big_running;
    char* in = base + t.in.off;
    char* ob = base + t.out.off;
    lk.unlock();
    rplu_opts jo;
    rplu_opts_init(&jo);
    jo.dtype = r.dtype;
    jo.pivot = o.pivot;
    jo.rel_tol = r.rel_tol;
    jo.stream = s_big;
    std::vector<double> T(k + 1, 0.0);
    jo.T_hist = T.data();
    int64_t kd = 0;
    char* p = ob;
    int64_t* I = (int64_t*)p;
    p += Arena::round_up(kk * 8);
    int64_t* J = (int64_t*)p;
    p += Arena::round_up(kk * 8);
    void* L = p;
    p += Arena::round_up(n * kk * w);
    void* U = p;
    rplu_status st;
    if (r.kind == 0) {
      cudaMemcpy2DAsync(in, ldp * w, r.A, (r.lda ? r.lda : m) * w, m * w, n, cudaMemcpyDefault, s_big);
      jo.lda = ldp;
      jo.overwrite_input = 1;
      st = rplu_dense(in, n, m, k, r.seed, &jo, I, J, L, U, &kd);
    } else {
      char* xs = in;
      char* ys = xs + Arena::round_up(n * w);
      char* gs = ys + Arena::round_up(m * w);
      char* bs = gs + Arena::round_up(n * w);
      cudaMemcpyAsync(xs, r.x, n * w, cudaMemcpyDefault, s_big);
      cudaMemcpyAsync(ys, r.y, m * w, cudaMemcpyDefault, s_big);
      k_fill_ones<<<sms * 2, 256, 0, s_big>>>((float*)gs, n, w == 8);
      k_fill_ones<<<sms * 2, 256, 0, s_big>>>((float*)bs, m, w == 8);
      jo.bound_nu = o.bound_nu;
      st = rplu_cauchy_like(xs, ys, gs, bs, n, m, 1, k, r.seed, &jo, I, J, L, U, &kd);
      if (o.bound_nu >= 1.0 && (st == RPLU_OK || st == RPLU_NOT_CONVERGED)) {
        // T[0] holds the bounds' sum there: ||A||_F^2 from the exact norms of a zero-step call
        rplu_opts eo = jo;
        eo.bound_nu = 0.0;
        eo.rel_tol = 0.0;
        double T0 = 0.0;
        eo.T_hist = &T0;
        int64_t k0 = 0;
        const rplu_status e0 = rplu_cauchy_like(xs, ys, gs, bs, n, m, 1, 0, r.seed, &eo, I, J, L, U, &k0);
        T[0] = e0 == RPLU_OK ? T0 : NAN;
      }
    }
    lk.lock();
    --big_running;
    t.k_done = kd;
    t.status = st;
    t.rel_res = (st == RPLU_OK || st == RPLU_NOT_CONVERGED) && T[0] > 0 ? std::sqrt(T[kd] / T[0]) : NAN;
    t.state = t.cancel_req ? RPLU_TICKET_CANCELLED : RPLU_TICKET_DONE;
    if (t.cancel_req) t.status = RPLU_CANCELLED, ++cancelled;
    t.t_done = now_s();
    // the input copy is no longer needed
    arena.release(t.in.off, t.in.bytes);
    t.in = Block{};
    ++completed;
    ++big_completed;
    completions.push_back(t.id);
    cv.notify_all();
  }
}

rplu_session::~rplu_session() {
  quit.store(true);
  if (stop_h) __atomic_store_n(stop_h, 1, __ATOMIC_RELEASE);
  cv.notify_all();
  if (worker.joinable()) worker.join();
  for (auto& w : big_workers)
    if (w.joinable()) w.join();
  for (Launch& r : ring.run)
    if (r.s) cudaStreamSynchronize(r.s);
  for (cudaStream_t s : s_big) cudaStreamSynchronize(s);
  if (s_copy) cudaStreamSynchronize(s_copy);
  for (cudaStream_t s : s_big) cudaStreamDestroy(s);
  if (s_copy) cudaStreamDestroy(s_copy);
  {
    Ring& L = ring;
    for (Launch& r : L.run) {
      if (r.ev) cudaEventDestroy(r.ev);
      if (r.s) cudaStreamDestroy(r.s);
    }
    if (L.head_d) cudaFree(L.head_d);
    for (void* h : {(void*)L.ring_h, (void*)L.tail_h, (void*)L.done_h, (void*)L.cancel_h, (void*)L.claimed_h,
                    (void*)L.exited_h})
      if (h) cudaFreeHost(h);
  }
  if (base) cudaFree(base);
  if (stop_h) cudaFreeHost(stop_h);
}

extern "C" {

void rplu_session_opts_init(rplu_session_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_jobs = 4096;
  o->max_dim = 2048;
  o->idle_us = 1000.0;
  o->pivot = RPLU_PIVOT_RANDOM;
  o->large_streams = 8;
  o->dense_kernel_cells = 0;  // 0: every dense request within max_dim runs in the persistent kernel
  o->cauchy_max_dim = 0;      // 0: 4096
}

rplu_status rplu_session_create(const rplu_session_opts* opts, rplu_session** out) {
  if (!out) return host_fail(RPLU_ERR_INVALID, "session is NULL");
  *out = nullptr;
  rplu_session_opts o;
  if (opts) o = *opts;
  else rplu_session_opts_init(&o);
  if (o.max_jobs <= 0) o.max_jobs = 4096;
  if (o.max_dim <= 0) o.max_dim = 2048;
  if (o.large_streams <= 0) o.large_streams = 8;
  if (o.dense_kernel_cells <= 0) o.dense_kernel_cells = (int64_t)o.max_dim * o.max_dim;
  if (o.large_streams > 64) return host_fail(RPLU_ERR_INVALID, "large_streams must be at most 64");
  if (o.cauchy_max_dim <= 0) o.cauchy_max_dim = kServeMaxDim;
  if (o.max_dim > kServeMaxDim) return host_fail(RPLU_ERR_INVALID, "max_dim must be at most 4096");
  if (o.cauchy_max_dim > kServeMaxDim) return host_fail(RPLU_ERR_INVALID, "cauchy_max_dim must be at most 4096");
  if (!(o.idle_us > 0.0)) o.idle_us = 1000.0;
  if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2)
    return host_fail(RPLU_ERR_INVALID, "sessions support RPLU_PIVOT_RANDOM and RPLU_PIVOT_C2");
  if (!(o.bound_nu == 0.0 || (std::isfinite(o.bound_nu) && o.bound_nu >= 1.0)))
    return host_fail(RPLU_ERR_INVALID, "bound_nu must be 0 or a finite number >= 1");
  rplu_session* s = new rplu_session;
  s->o = o;
  auto bail = [s](rplu_status st, const char* msg) {
    delete s;
    return host_fail(st, msg);
  };
  if (cudaGetDevice(&s->dev) != cudaSuccess || host_num_sms(&s->sms) != cudaSuccess)
    return bail(RPLU_ERR_CUDA, "device query");
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  int64_t budget = o.hbm_budget > 0 ? o.hbm_budget : (int64_t)(0.8 * (double)fr);
  budget = std::min<int64_t>(budget, (int64_t)fr - ((int64_t)1 << 30));
  if (budget < ((int64_t)1 << 20)) return bail(RPLU_ERR_NOMEM, "no device memory for the session");
  if (cudaMalloc(&s->base, (size_t)budget) != cudaSuccess) return bail(RPLU_ERR_NOMEM, "session arena");
  s->arena.reset(budget);
  s->cap = o.max_jobs;
  const unsigned fl = cudaHostAllocMapped;
  if (cudaHostAlloc((void**)&s->stop_h, 64, fl) != cudaSuccess) return bail(RPLU_ERR_NOMEM, "pinned ring");
  *s->stop_h = 0;
  cudaHostGetDevicePointer((void**)&s->stop_d, s->stop_h, 0);
  if (cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) != cudaSuccess)
    return bail(RPLU_ERR_CUDA, "streams");
  {
    Ring& L = s->ring;
    L.slot_owner.assign((size_t)s->cap, -1);
    if (cudaHostAlloc((void**)&L.ring_h, sizeof(BatchDesc) * s->cap, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&L.tail_h, 64, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&L.done_h, sizeof(int64_t) * s->cap, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&L.cancel_h, sizeof(int32_t) * s->cap, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&L.claimed_h, sizeof(int64_t) * s->cap, fl) != cudaSuccess)
      return bail(RPLU_ERR_NOMEM, "pinned ring");
    std::memset(L.ring_h, 0, sizeof(BatchDesc) * s->cap);
    std::memset(L.done_h, 0, sizeof(int64_t) * s->cap);
    std::memset(L.cancel_h, 0, sizeof(int32_t) * s->cap);
    std::memset(L.claimed_h, 0, sizeof(int64_t) * s->cap);
    *L.tail_h = 0;
    cudaHostGetDevicePointer((void**)&L.ring_d, L.ring_h, 0);
    cudaHostGetDevicePointer((void**)&L.tail_d, L.tail_h, 0);
    cudaHostGetDevicePointer((void**)&L.done_d, L.done_h, 0);
    cudaHostGetDevicePointer((void**)&L.cancel_d, L.cancel_h, 0);
    cudaHostGetDevicePointer((void**)&L.claimed_d, L.claimed_h, 0);
    if (cudaMalloc(&L.head_d, 64) != cudaSuccess) return bail(RPLU_ERR_NOMEM, "ring head");
    cudaMemset(L.head_d, 0, 64);
    for (Launch& r : L.run)
      if (cudaStreamCreateWithFlags(&r.s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(RPLU_ERR_CUDA, "streams");
    // kernel shape: shared memory for the largest served job of either type (dense up to
    // max_dim, Cauchy up to cauchy_max_dim; rows padded to 16 bytes for both types), as many
    // CTAs per SM as fit; write-back interval: the largest (<= 6) that keeps two CTAs per SM,
    // else the largest that fits
    L.args.n_max = o.max_dim;
    L.args.lds_max = pad_row(o.max_dim, 4);
    L.args.gn_max = o.cauchy_max_dim;
    L.args.gm_max = pad_row(o.cauchy_max_dim, 4);
    L.args.mode = o.pivot;
    L.args.kinds = kKindDense | kKindCauchy;
    int best_blk = 0, best_occ = 0;
    for (int b = kServeMaxBlk; b >= 1; --b) {
      int occ = 0;
      L.args.blk = b;
      if (serve_occupancy(serve_smem_bytes(L.args), &occ) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      if (occ > best_occ && (best_occ < 2 || b == kServeMaxBlk)) {
        best_occ = occ;
        best_blk = b;
      }
      if (occ >= 2) break;
    }
    if (best_occ < 1) return bail(RPLU_ERR_CUDA, "serving kernel does not fit on an SM");
    L.args.blk = best_blk;
    L.grid = s->sms * best_occ;
    if (cudaHostAlloc((void**)&L.exited_h, sizeof(int32_t) * kLaunches * L.grid, fl) != cudaSuccess)
      return bail(RPLU_ERR_NOMEM, "pinned ring");
    std::memset(L.exited_h, 0, sizeof(int32_t) * kLaunches * L.grid);
    cudaHostGetDevicePointer((void**)&L.exited_d, L.exited_h, 0);
  }
  for (int q = 0; q < o.large_streams; ++q) {
    cudaStream_t sb;
    if (cudaStreamCreateWithFlags(&sb, cudaStreamNonBlocking) != cudaSuccess) return bail(RPLU_ERR_CUDA, "streams");
    s->s_big.push_back(sb);
  }
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, s->dev);
  s->idle_cycles = (long long)(o.idle_us * (double)(clk_khz > 0 ? clk_khz : 2000000) / 1000.0);
  cudaDeviceSynchronize();
  s->worker = std::thread([s] { s->work(); });
  for (cudaStream_t sb : s->s_big) s->big_workers.push_back(std::thread([s, sb] { s->big_work(sb); }));
  *out = s;
  return RPLU_OK;
}

rplu_status rplu_session_submit(rplu_session* s, const rplu_request* r, int64_t* ticket) {
  if (!s || !r || !ticket) return host_fail(RPLU_ERR_INVALID, "NULL argument");
  if (const char* why = request_invalid(*r)) return host_fail(RPLU_ERR_INVALID, why);
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t id = s->next_id++;
  Ticket& t = s->tk[id];
  t.id = id;
  t.req = *r;
  t.t_submit = now_s();
  t.big = !s->fits_kernel(*r);
  t.w = elem_w(r->dtype);
  if (t.big) s->big_queue.push_back(id);
  else s->queue.push_back(id);
  *ticket = id;
  s->cv.notify_all();
  return RPLU_OK;
}

rplu_status rplu_session_poll(rplu_session* s, int64_t ticket, rplu_ticket_info* info) {
  if (!s || !info) return host_fail(RPLU_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tk.find(ticket);
  if (it == s->tk.end()) return host_fail(RPLU_ERR_INVALID, "unknown ticket");
  const Ticket& t = it->second;
  info->state = t.state;
  info->status = t.status;
  info->k_done = t.k_done;
  info->rel_res = t.rel_res;
  info->latency_ms = t.state >= RPLU_TICKET_DONE ? (t.t_done - t.t_submit) * 1e3 : NAN;
  info->queue_ms = t.t_admit > 0 ? (t.t_admit - t.t_submit) * 1e3 : NAN;
  return RPLU_OK;
}

rplu_status rplu_session_wait(rplu_session* s, int64_t ticket, double timeout_s, rplu_ticket_info* info) {
  if (!s || !info) return host_fail(RPLU_ERR_INVALID, "NULL argument");
  const double t_end = now_s() + (timeout_s > 0 ? timeout_s : 1e30);
  {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
      auto it = s->tk.find(ticket);
      if (it == s->tk.end()) return host_fail(RPLU_ERR_INVALID, "unknown ticket");
      if (it->second.state >= RPLU_TICKET_DONE) break;
      if (now_s() > t_end) break;
      s->cv.wait_for(lk, std::chrono::microseconds(100));
    }
  }
  rplu_status st = rplu_session_poll(s, ticket, info);
  if (st != RPLU_OK) return st;
  return info->state >= RPLU_TICKET_DONE ? RPLU_OK : host_fail(RPLU_ERR_TIMEOUT, "ticket not finished in time");
}

rplu_status rplu_session_fetch(rplu_session* s, int64_t ticket, int64_t* I, int64_t* J, void* L, void* U) {
  if (!s) return host_fail(RPLU_ERR_INVALID, "NULL session");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tk.find(ticket);
  if (it == s->tk.end()) return host_fail(RPLU_ERR_INVALID, "unknown ticket");
  Ticket& t = it->second;
  if (t.state < RPLU_TICKET_DONE) return host_fail(RPLU_ERR_INVALID, "ticket not finished");
  const int64_t n = t.req.n, m = t.req.m, kk = std::max<int64_t>(t.req.k_max, 1), kd = t.k_done;
  const int64_t w = t.w;
  cudaError_t e = cudaSuccess;
  if (t.out.off >= 0 && kd > 0) {
    char* p = s->base + t.out.off;
    if (I) e = cudaMemcpy(I, p, kd * 8, cudaMemcpyDefault);
    p += Arena::round_up(kk * 8);
    if (J && e == cudaSuccess) e = cudaMemcpy(J, p, kd * 8, cudaMemcpyDefault);
    p += Arena::round_up(kk * 8);
    if (L && e == cudaSuccess) e = cudaMemcpy(L, p, n * kd * w, cudaMemcpyDefault);
    p += Arena::round_up(n * kk * w);
    if (U && e == cudaSuccess) e = cudaMemcpy(U, p, kd * m * w, cudaMemcpyDefault);
  }
  s->free_blocks(t);
  s->tk.erase(it);
  if (e != cudaSuccess) return host_fail(RPLU_ERR_CUDA, cudaGetErrorString(e));
  return RPLU_OK;
}

rplu_status rplu_session_cancel(rplu_session* s, int64_t ticket) {
  if (!s) return host_fail(RPLU_ERR_INVALID, "NULL session");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tk.find(ticket);
  if (it == s->tk.end()) return host_fail(RPLU_ERR_INVALID, "unknown ticket");
  Ticket& t = it->second;
  if (t.state == RPLU_TICKET_QUEUED) {
    auto& q = t.big ? s->big_queue : s->queue;
    q.erase(std::remove(q.begin(), q.end(), ticket), q.end());
    t.state = RPLU_TICKET_CANCELLED;
    t.status = RPLU_CANCELLED;
    t.t_done = now_s();
    s->completions.push_back(ticket);
    ++s->cancelled;
  } else if (t.state == RPLU_TICKET_RUNNING) {
    if (t.big) t.cancel_req = true;
    else __atomic_store_n(&s->ring.cancel_h[t.slot], 1, __ATOMIC_RELEASE);
  }
  s->cv.notify_all();
  return RPLU_OK;
}

rplu_status rplu_session_completed(rplu_session* s, int64_t* tickets, rplu_ticket_info* infos, int32_t max_n,
                                   int32_t* count) {
  if (!s || !count || max_n < 0 || (max_n > 0 && (!tickets || !infos))) return host_fail(RPLU_ERR_INVALID, "bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int32_t c = 0;
  while (c < max_n && !s->completions.empty()) {
    const int64_t id = s->completions.front();
    s->completions.pop_front();
    auto it = s->tk.find(id);
    if (it == s->tk.end()) continue;  // fetched meanwhile
    const Ticket& t = it->second;
    tickets[c] = id;
    infos[c].state = t.state;
    infos[c].status = t.status;
    infos[c].k_done = t.k_done;
    infos[c].rel_res = t.rel_res;
    infos[c].latency_ms = (t.t_done - t.t_submit) * 1e3;
    infos[c].queue_ms = t.t_admit > 0 ? (t.t_admit - t.t_submit) * 1e3 : NAN;
    ++c;
  }
  *count = c;
  return RPLU_OK;
}

rplu_status rplu_session_stats(rplu_session* s, double out[8]) {
  if (!s || !out) return host_fail(RPLU_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = (double)s->completed;
  out[1] = (double)(s->queue.size() + s->big_queue.size());
  out[2] = (double)(s->on_gpu.size() + s->big_running);
  out[3] = (double)s->arena.used();
  out[4] = (double)s->arena.size();
  out[5] = (double)s->launches;
  out[6] = (double)s->big_completed;
  out[7] = (double)s->cancelled;
  return RPLU_OK;
}

void rplu_session_destroy(rplu_session* s) { delete s; }

}  // extern "C"
