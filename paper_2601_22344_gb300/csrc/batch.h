// Launch descriptors of the persistent batch kernel (batch.cu) and the host
// helpers the batch entry points share with the single-job ones (abi.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rplu.h"

namespace rplu {

// One job as the kernel sees it.  All pointers are device memory.
struct BatchDesc {
  const void* A;   // kind 0: n x m row-major, row stride lda
  const void* x;   // kind 1: n points
  const void* y;   // kind 1: m points
  void* S;         // workspace n x lds (16-byte aligned rows); null when k_max <= blk
  int64_t* I;      // k_max
  int64_t* J;      // k_max
  void* L;         // n x k_max column-major
  void* U;         // k_max x m row-major
  int64_t n, m, k_max, lda, lds;
  double tol;
  uint64_t seed;
  int32_t kind;    // 0 dense (A's rows 16-byte aligned: base and lda * elem_size), 1 Cauchy
  int32_t dtype;   // serving: RPLU_F32 or RPLU_C64 (one kernel serves both); batch launches: unused
  // written by the kernel
  int64_t k_done;
  double T0;       // ||A||_F^2
  double T_final;  // ||S||_F^2 after the last step (at the stop test when stopped early)
  int32_t err;     // kErr* bits
  int32_t pad;
};

struct BatchArgs {
  BatchDesc* jobs;
  const int32_t* order;  // visiting order (largest first)
  int32_t njobs;
  int32_t blk;           // steps between write-backs, 1..8
  int32_t* counter;      // next job; zero before the launch
  int32_t mode;          // RPLU_PIVOT_RANDOM or RPLU_PIVOT_C2
  int64_t n_max;         // largest n of the dense jobs
  int64_t lds_max;       // largest padded row length of the dense jobs (m rounded up to the 16-byte vector)
  int32_t kinds;         // bit 0: dense jobs in the launch, bit 1: Cauchy jobs (shared-memory sizing)
  int64_t gn_max;        // largest n of the Cauchy jobs (generator form)
  int64_t gm_max;        // largest padded m of the Cauchy jobs
};

constexpr int32_t kKindDense = 1, kKindCauchy = 2;

// Launch shape: threads per CTA (256 or 512), rows per warp tile (2 or 4), CTAs.
struct BatchShape {
  int threads;
  int rows;
  int grid;
};

// Serving ring (host-mapped pinned memory unless noted); ticket h uses slot h % cap.
struct ServeRing {
  BatchDesc* desc;               // cap descriptors; results written back by the kernel
  const volatile long long* tail;  // tickets published by the host
  long long* head;               // device memory: next ticket to claim
  volatile int64_t* done;        // per slot: ticket + 1 once its results are written
  const volatile int32_t* cancel;  // per slot: nonzero asks the job to stop between steps
  const volatile int32_t* stop;  // nonzero: CTAs exit at their next claim
  volatile int64_t* claimed;     // per slot: ticket + 1 once a CTA has claimed it
  volatile int32_t* exited;      // per CTA of this launch: 1 once the CTA has exited
  int64_t cap;
  long long idle_cycles;         // a CTA exits after this many SM clocks without a ticket
};

// Dynamic shared memory of a launch of element type dtype: the residual layout
// for its dense jobs (n_max, lds_max, blk), the generator layout for its Cauchy
// jobs (gn_max, gm_max), the larger (a.kinds says which are present).
int64_t batch_smem_bytes(int32_t dtype, const BatchArgs& a);
// The serving kernel (256 threads) serves FP32 and complex64 jobs of both
// kinds: its shared memory is the largest of the four layouts.
int64_t serve_smem_bytes(const BatchArgs& a);
cudaError_t serve_occupancy(int64_t smem, int* blocks);
cudaError_t serve_launch(const BatchArgs& a, const ServeRing& q, int grid, cudaStream_t s);
// Sets the kernel's dynamic shared-memory limit and returns its CTAs per SM.
cudaError_t batch_occupancy(int32_t dtype, int threads, int rows, int64_t smem, int* blocks);
// batch_occupancy must have been called for the same kernel and smem first.
cudaError_t batch_launch(int32_t dtype, const BatchArgs& a, const BatchShape& sh, cudaStream_t s);

// abi.cu
rplu_status host_fail(rplu_status s, const char* msg);
bool host_on_device(const void* p);
cudaError_t host_num_sms(int* sms);
// Whether the current device accesses pageable host memory in place
// (cudaDevAttrPageableMemoryAccess: a coherent host link with address translation).
cudaError_t host_pageable_access(bool* yes);

}  // namespace rplu
