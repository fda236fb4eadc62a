// CUR-AAA (Sec. 5.3, Algorithm "CUR-AAA using RPLU") around Algorithm 3:
// the random split of the samples, the Loewner generators, and the fit and
// evaluation of the barycentric rational functions (Eq. aaa-barycentric) on
// the two pivot sets.  The factorization itself is rplu_cauchy_like with the
// bounds (cauchy_bh.cu).  All data complex128.
//
//   k_aaa_split / compaction     X = {i : pi(i) < ceil(m/2)}, Y = the rest, in
//                                index order; pi a keyed Feistel permutation of
//                                [0, m) (4 rounds on 2h-bit words, SplitMix64
//                                output function as the round function, cycle
//                                walking: Black & Rogaway 2002)
//   k_aaa_absmax, k_aaa_gen      alpha = sqrt(max |f|), G = [f^x/alpha, alpha],
//                                B = [alpha; -f^y/alpha] (Eq. loewner-generators)
//   k_aaa_loewner                the Loewner matrix (f_i - f_tj)/(z_i - t_j)
//                                over the non-support samples (Eq. Laaa),
//                                column-major
//   k_hh_*                       Householder QR of that tall matrix, one
//                                column at a time (norm, reflector, dot
//                                products with the trailing columns, update)
//   k_aaa_invit                  the right singular vector of the smallest
//                                singular value of R by inverse iteration
//                                (two triangular solves per iteration)
//   k_aaa_eval                   r(z_i) on all samples and max |f_i - r(z_i)|
#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace rplu {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPartKey = 0x632BE59BD9B4E019ull;
constexpr int kT = 256;
constexpr int kScanBlock = 1024;  // elements per compaction block (4 per thread)

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t feistel(int64_t i, int64_t m, uint64_t key, int h) {
  const uint64_t mask = (1ull << h) - 1;
  uint64_t x = (uint64_t)i;
  for (int walk = 0; walk < 4096; ++walk) {  // expected < 4 walks (2^(2h) < 4m)
    uint64_t left = x >> h, right = x & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint64_t f = mix64(key ^ (kGamma * (uint64_t)(r + 1)) ^ right) & mask;
      const uint64_t nl = right;
      right = left ^ f;
      left = nl;
    }
    x = (left << h) | right;
    if (x < (uint64_t)m) return (int64_t)x;
  }
  return -1;  // not reached for m >= 1 (a cycle of the permutation returns to [0, m))
}

__global__ void k_aaa_split(int64_t m, uint64_t key, int h, uint8_t* flag, int32_t* bad) {
  const int64_t half = (m + 1) / 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = feistel(i, m, key, h);
    if (p < 0) atomicOr(bad, 1);
    flag[i] = p >= 0 && p < half ? 1 : 0;
  }
}

// Stable compaction by a 0/1 flag: block counts, their exclusive scan (one
// CTA), then each block places its elements (flag 1 into `one`, flag 0 into
// `zero`) in index order.
__global__ void __launch_bounds__(kT) k_flag_count(const uint8_t* flag, int64_t m, int32_t* cnt) {
  __shared__ int red[kT / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int c = 0;
  for (int e = threadIdx.x; e < kScanBlock; e += kT) {
    const int64_t i = base + e;
    c += (i < m && flag[i]) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kT / 32; ++w) s += red[w];
    cnt[blockIdx.x] = s;
  }
}

__global__ void k_flag_scan(int32_t* cnt, int nb, int64_t* total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t run = 0;
  for (int b = 0; b < nb; ++b) {
    const int32_t c = cnt[b];
    cnt[b] = (int32_t)run;
    run += c;
  }
  *total = run;
}

__global__ void __launch_bounds__(kT) k_flag_place(const uint8_t* flag, int64_t m, const int32_t* off,
                                                   int64_t* one, int64_t* zero) {
  __shared__ int wsum[kT / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // each thread owns 4 consecutive elements
  const int64_t i0 = base + 4 * threadIdx.x;
  int f[4], c = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    f[e] = (i0 + e < m && flag[i0 + e]) ? 1 : 0;
    c += f[e];
  }
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += wsum[w];
  int pos1 = off[blockIdx.x] + wbase + incl - c;  // ones before this thread's first element
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t i = i0 + e;
    if (i >= m) break;
    if (f[e]) {
      one[pos1++] = i;
    } else if (zero) {
      zero[i - pos1] = i;  // zeros before i = i - (ones before i)
    }
  }
}

__global__ void k_gather(const cf64* z, const cf64* f, const int64_t* idx, int64_t n, cf64* zo, cf64* fo) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx[q];
    zo[q] = z[i];
    if (fo) fo[q] = f[i];
  }
}

// max |f_i| as the bit pattern of a non-negative double (atomicMax orders it)
__global__ void k_aaa_absmax(const cf64* f, int64_t m, unsigned long long* out) {
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, hypot(f[i].re, f[i].im));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

__global__ void k_aaa_gen(const cf64* fx, int64_t nx, const cf64* fy, int64_t ny, const unsigned long long* fmax_bits,
                          cf64* G, cf64* B) {
  const double alpha = sqrt(__longlong_as_double((long long)*fmax_bits));
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nx + ny;
       q += (int64_t)gridDim.x * blockDim.x) {
    if (q < nx) {
      G[2 * q] = cf64{fx[q].re / alpha, fx[q].im / alpha};
      G[2 * q + 1] = cf64{alpha, 0.0};
    } else {
      const int64_t j = q - nx;
      B[j] = cf64{alpha, 0.0};
      B[ny + j] = cf64{-fy[j].re / alpha, -fy[j].im / alpha};
    }
  }
}

__device__ __forceinline__ cf64 cdiv(cf64 a, cf64 b) {
  double qr, qi;
  cdiv_d(a.re, a.im, b.re, b.im, qr, qi);
  return cf64{qr, qi};
}

// A (M x k, column-major, leading dimension M): (f_r - f_t) / (z_r - t) for the
// non-support samples r (rows) and the support points t (columns)
__global__ void k_aaa_loewner(const cf64* z, const cf64* f, const int64_t* rows, int64_t M, const int64_t* sup,
                              int64_t k, cf64* A) {
  const int64_t total = M * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / M, r = e - c * M;
    const int64_t i = rows[r], t = sup[c];
    const cf64 num{f[i].re - f[t].re, f[i].im - f[t].im};
    const cf64 den{z[i].re - z[t].re, z[i].im - z[t].im};
    A[e] = cdiv(num, den);
  }
}

// ------------------------------------------------------- Householder QR
// Column j: x = A(j:M, j).  v = x with v_0 = x_0 + e^{i arg x_0} ||x||, H = I - s v v^*
// with s = 2 / (v^* v) = 1 / (||x|| (||x|| + |x_0|)); H x = -e^{i arg x_0} ||x|| e_1.
__global__ void __launch_bounds__(kT) k_hh_norm(const cf64* A, int64_t M, int64_t j, double* part) {
  const cf64* col = A + j * M;
  double s = 0.0;
  for (int64_t r = j + (int64_t)blockIdx.x * kT + threadIdx.x; r < M; r += (int64_t)gridDim.x * kT)
    s = fma(col[r].re, col[r].re, fma(col[r].im, col[r].im, s));
  __shared__ double red[kT / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// one thread: the reflector of column j from the partial sums
__global__ void k_hh_reflect(cf64* A, int64_t M, int64_t j, const double* part, int nb, double* s_out, cf64* rdiag) {
  if (threadIdx.x != 0) return;
  double n2 = 0.0;
  for (int b = 0; b < nb; ++b) n2 += part[b];
  const double nrm = sqrt(n2);
  cf64 x0 = A[j * M + j];
  const double a0 = hypot(x0.re, x0.im);
  if (nrm == 0.0) {
    s_out[j] = 0.0;
    rdiag[j] = cf64{0.0, 0.0};
    return;
  }
  const double pr = a0 > 0.0 ? x0.re / a0 : 1.0, pi = a0 > 0.0 ? x0.im / a0 : 0.0;
  A[j * M + j] = cf64{x0.re + pr * nrm, x0.im + pi * nrm};
  s_out[j] = 1.0 / (nrm * (nrm + a0));
  rdiag[j] = cf64{-pr * nrm, -pi * nrm};
}

// Partial products w_c = v^* A(j:M, c) for the trailing columns: block
// (rchunk, cgroup) covers rows [j + rchunk*RC, ...) and 16 columns; lanes run
// down the rows, each warp a share of the chunk, then fixed-order reductions.
constexpr int kRC = 2048;  // rows per chunk
constexpr int kCG = 16;    // trailing columns per block
__global__ void __launch_bounds__(kT) k_hh_dots(const cf64* A, int64_t M, int64_t k, int64_t j, double* part2,
                                                int nrc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = j + 1 + (int64_t)blockIdx.y * kCG;
  const int nc = (int)min((int64_t)kCG, k - c0);
  const int64_t r0 = j + (int64_t)blockIdx.x * kRC;
  const int64_t r1 = min(M, r0 + kRC);
  const cf64* v = A + j * M;
  double ar[kCG], ai[kCG];
#pragma unroll
  for (int c = 0; c < kCG; ++c) ar[c] = ai[c] = 0.0;
  for (int64_t r = r0 + warp * 32 + lane; r < r1; r += kT) {
    const cf64 vr = v[r];
#pragma unroll
    for (int c = 0; c < kCG; ++c) {
      if (c < nc) {
        const cf64 a = A[(c0 + c) * M + r];
        // conj(v) * a
        ar[c] = fma(vr.re, a.re, fma(vr.im, a.im, ar[c]));
        ai[c] = fma(vr.re, a.im, fma(-vr.im, a.re, ai[c]));
      }
    }
  }
  __shared__ double sr[kT / 32][kCG], si[kT / 32][kCG];
#pragma unroll
  for (int c = 0; c < kCG; ++c) {
    double x = ar[c], y = ai[c];
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == c) {
      sr[warp][c] = x;
      si[warp][c] = y;
    }
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < kT / 32; ++w) {
      x += sr[w][threadIdx.x];
      y += si[w][threadIdx.x];
    }
    const int64_t c = c0 + threadIdx.x;
    part2[(c * (int64_t)nrc + blockIdx.x) * 2] = x;
    part2[(c * (int64_t)nrc + blockIdx.x) * 2 + 1] = y;
  }
}

// w_c (scaled by s) from the chunk partials, in chunk order
__global__ void k_hh_wfin(const double* part2, int nrc, int64_t k, int64_t j, const double* s, cf64* sw) {
  for (int64_t c = j + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < k; c += (int64_t)gridDim.x * blockDim.x) {
    double x = 0.0, y = 0.0;
    for (int b = 0; b < nrc; ++b) {
      x += part2[(c * (int64_t)nrc + b) * 2];
      y += part2[(c * (int64_t)nrc + b) * 2 + 1];
    }
    sw[c] = cf64{s[j] * x, s[j] * y};
  }
}

// A(j:M, c) -= v * (s w_c) for the trailing columns
__global__ void k_hh_update(cf64* A, int64_t M, int64_t k, int64_t j, const cf64* sw) {
  const int64_t rows = M - j, cols = k - j - 1;
  const int64_t total = rows * cols;
  const cf64* v = A + j * M;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cc = e / rows, rr = e - cc * rows;
    const int64_t c = j + 1 + cc, r = j + rr;
    const cf64 vr = v[r], w = sw[c];
    cf64& a = A[c * M + r];
    a.re -= vr.re * w.re - vr.im * w.im;
    a.im -= vr.re * w.im + vr.im * w.re;
  }
}

// ------------------------------------------------------ inverse iteration
// R (k x k upper triangular): R(i, c) = A[c * M + i] for i < c, R(i, i) =
// rdiag[i].  x <- (R^* R)^{-1} x / norm, from x = (1, ..., 1)/sqrt(k), until
// the change (up to a unit factor) is below 1e-14 or 60 iterations.  Diagonal
// entries below 1e-15 of the largest are raised to that size so that the
// solves stay finite when R is singular to working precision.
__global__ void __launch_bounds__(1024) k_aaa_invit(const cf64* A, int64_t M, int64_t k, const cf64* rdiag, cf64* x,
                                                    cf64* y, int32_t* iters) {
  __shared__ double red[32];
  __shared__ double dmax_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto block_sum = [&](double v) -> double {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (tid == 0) {
      for (int w = 0; w < nt / 32; ++w) t += red[w];
      red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
  };
  double dm = 0.0;
  for (int64_t i = tid; i < k; i += nt) dm = fmax(dm, hypot(rdiag[i].re, rdiag[i].im));
  for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((tid & 31) == 0) red[tid >> 5] = dm;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nt / 32; ++w) t = fmax(t, red[w]);
    dmax_s = t > 0.0 ? t : 1.0;
  }
  __syncthreads();
  const double floor_d = 1e-15 * dmax_s;
  auto diag = [&](int64_t i) -> cf64 {
    const cf64 d = rdiag[i];
    const double a = hypot(d.re, d.im);
    if (a >= floor_d) return d;
    return a > 0.0 ? cf64{d.re / a * floor_d, d.im / a * floor_d} : cf64{floor_d, 0.0};
  };
  const double inv = 1.0 / sqrt((double)k);
  for (int64_t i = tid; i < k; i += nt) x[i] = cf64{inv, 0.0};
  __syncthreads();
  int it = 0;
  for (; it < 60; ++it) {
    // R^* y = x (forward): y_i = (x_i - sum_{l<i} conj(R(l,i)) y_l) / conj(R(i,i)), column by column
    for (int64_t i = tid; i < k; i += nt) y[i] = x[i];
    __syncthreads();
    for (int64_t i = 0; i < k; ++i) {
      const cf64 d = diag(i);
      const cf64 yi = cdiv(y[i], cf64{d.re, -d.im});
      __syncthreads();
      if (tid == 0) y[i] = yi;
      for (int64_t l = i + 1 + tid; l < k; l += nt) {
        const cf64 r = A[l * M + i];  // R(i, l)
        // y_l -= conj(r) * yi
        y[l].re -= r.re * yi.re + r.im * yi.im;
        y[l].im -= r.re * yi.im - r.im * yi.re;
      }
      __syncthreads();
    }
    // R z = y (backward), z into y in place: z_i = (y_i - sum_{c>i} R(i,c) z_c) / R(i,i)
    for (int64_t i = k - 1; i >= 0; --i) {
      const cf64 zi = cdiv(y[i], diag(i));
      __syncthreads();
      if (tid == 0) y[i] = zi;
      for (int64_t l = tid; l < i; l += nt) {
        const cf64 r = A[i * M + l];  // R(l, i)
        y[l].re -= r.re * zi.re - r.im * zi.im;
        y[l].im -= r.re * zi.im + r.im * zi.re;
      }
      __syncthreads();
    }
    double n2 = 0.0;
    for (int64_t i = tid; i < k; i += nt) n2 += y[i].re * y[i].re + y[i].im * y[i].im;
    const double nrm = sqrt(block_sum(n2));
    // change up to a unit factor: 1 - |<x, y/|y|>|
    double pr = 0.0, pi = 0.0;
    for (int64_t i = tid; i < k; i += nt) {
      pr += x[i].re * y[i].re + x[i].im * y[i].im;
      pi += x[i].re * y[i].im - x[i].im * y[i].re;
    }
    pr = block_sum(pr);
    pi = block_sum(pi);
    const double ov = hypot(pr, pi) / nrm;
    for (int64_t i = tid; i < k; i += nt) x[i] = cf64{y[i].re / nrm, y[i].im / nrm};
    __syncthreads();
    if (1.0 - ov < 1e-14) {
      ++it;
      break;
    }
  }
  if (tid == 0) *iters = it;
}

// r(z_i) of Eq. aaa-barycentric on every sample and the largest |f_i - r(z_i)|
// (support samples interpolate exactly: error 0)
__global__ void __launch_bounds__(kT) k_aaa_eval(const cf64* z, const cf64* f, int64_t m, const int64_t* sup, int64_t k,
                                                 const cf64* w, const uint8_t* is_sup, unsigned long long* err_bits) {
  double mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < m; i += (int64_t)gridDim.x * kT) {
    if (is_sup[i]) continue;
    const cf64 zi = z[i];
    double nr = 0.0, ni = 0.0, dr = 0.0, di = 0.0;
    for (int64_t c = 0; c < k; ++c) {
      const int64_t t = sup[c];
      const cf64 q = cdiv(w[c], cf64{zi.re - z[t].re, zi.im - z[t].im});
      dr += q.re;
      di += q.im;
      nr += q.re * f[t].re - q.im * f[t].im;
      ni += q.re * f[t].im + q.im * f[t].re;
    }
    const cf64 r = cdiv(cf64{nr, ni}, cf64{dr, di});
    mx = fmax(mx, hypot(f[i].re - r.re, f[i].im - r.im));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(err_bits, (unsigned long long)__double_as_longlong(mx));
}

// r at query points (a query on a support point takes its value)
__global__ void __launch_bounds__(kT) k_aaa_query(const cf64* t, const cf64* ft, const cf64* w, int64_t k,
                                                  const cf64* zq, int64_t nq, cf64* rq) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < nq; i += (int64_t)gridDim.x * kT) {
    const cf64 zi = zq[i];
    double nr = 0.0, ni = 0.0, dr = 0.0, di = 0.0;
    int64_t hit = -1;
    for (int64_t c = 0; c < k; ++c) {
      const cf64 d{zi.re - t[c].re, zi.im - t[c].im};
      if (d.re == 0.0 && d.im == 0.0) {
        if (hit < 0) hit = c;
        continue;
      }
      const cf64 q = cdiv(w[c], d);
      dr += q.re;
      di += q.im;
      nr += q.re * ft[c].re - q.im * ft[c].im;
      ni += q.re * ft[c].im + q.im * ft[c].re;
    }
    rq[i] = hit >= 0 ? ft[hit] : cdiv(cf64{nr, ni}, cf64{dr, di});
  }
}

__global__ void k_mark(const int64_t* idx, int64_t n, uint8_t* flag, uint8_t v) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    flag[idx[q]] = v;
}

__global__ void k_map(const int64_t* piv, const int64_t* set, int64_t k, int64_t* out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < k; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = set[piv[q]];
}

unsigned grid_for(int64_t n, int sms) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kT - 1) / kT, (int64_t)sms * 8));
}

cudaError_t compact(const uint8_t* flag, int64_t m, int64_t* one, int64_t* zero, int32_t* cnt, int64_t* total,
                    cudaStream_t s) {
  const int nb = (int)((m + kScanBlock - 1) / kScanBlock);
  k_flag_count<<<nb, kT, 0, s>>>(flag, m, cnt);
  k_flag_scan<<<1, 32, 0, s>>>(cnt, nb, total);
  k_flag_place<<<nb, kT, 0, s>>>(flag, m, cnt, one, zero);
  return cudaGetLastError();
}

}  // namespace

int64_t aaa_compact_blocks(int64_t m) { return (m + kScanBlock - 1) / kScanBlock; }

cudaError_t aaa_split(const AaaLaunch& a, cudaStream_t s) {
  int h = 1;
  while ((1ll << (2 * h)) < a.m) ++h;
  const cf64* z = (const cf64*)a.z;
  const cf64* f = (const cf64*)a.f;
  k_aaa_split<<<grid_for(a.m, a.num_sms), kT, 0, s>>>(a.m, a.seed ^ kPartKey, h, a.flag, a.bad);
  cudaError_t e = compact(a.flag, a.m, a.xidx, a.yidx, a.cnt, a.total, s);
  if (e != cudaSuccess) return e;
  const int64_t nx = (a.m + 1) / 2, ny = a.m / 2;
  k_gather<<<grid_for(nx, a.num_sms), kT, 0, s>>>(z, f, a.xidx, nx, (cf64*)a.x, (cf64*)a.fx);
  k_gather<<<grid_for(ny, a.num_sms), kT, 0, s>>>(z, f, a.yidx, ny, (cf64*)a.y, (cf64*)a.fy);
  e = cudaMemsetAsync(a.fmax_bits, 0, 8, s);
  if (e != cudaSuccess) return e;
  k_aaa_absmax<<<grid_for(a.m, a.num_sms), kT, 0, s>>>(f, a.m, a.fmax_bits);
  k_aaa_gen<<<grid_for(nx + ny, a.num_sms), kT, 0, s>>>((const cf64*)a.fx, nx, (const cf64*)a.fy, ny, a.fmax_bits,
                                                        (cf64*)a.G, (cf64*)a.B);
  return cudaGetLastError();
}

cudaError_t aaa_fit(const AaaLaunch& a, const int64_t* piv, const int64_t* set, int64_t k, AaaFit& o,
                    cudaStream_t s) {
  const int sms = a.num_sms;
  const cf64* z = (const cf64*)a.z;
  const cf64* f = (const cf64*)a.f;
  cf64* A = (cf64*)o.A;
  // support points (indices into z) and the rows of the Loewner matrix
  k_map<<<grid_for(k, sms), kT, 0, s>>>(piv, set, k, o.sup);
  cudaError_t e = cudaMemsetAsync(a.flag, 1, (size_t)a.m, s);
  if (e != cudaSuccess) return e;
  k_mark<<<grid_for(k, sms), kT, 0, s>>>(o.sup, k, a.flag, 0);
  e = compact(a.flag, a.m, o.rows, nullptr, a.cnt, a.total, s);
  if (e != cudaSuccess) return e;
  const int64_t M = a.m - k;
  k_aaa_loewner<<<grid_for(M * k, sms), kT, 0, s>>>(z, f, o.rows, M, o.sup, k, A);
  const int nrc = (int)std::max<int64_t>(1, (M + kRC - 1) / kRC);
  for (int64_t j = 0; j < k; ++j) {
    const int nb = (int)std::min<int64_t>(std::max<int64_t>(1, (M - j + kT - 1) / kT), (int64_t)sms * 4);
    k_hh_norm<<<nb, kT, 0, s>>>(A, M, j, o.part);
    k_hh_reflect<<<1, 32, 0, s>>>(A, M, j, o.part, nb, o.s, (cf64*)o.rdiag);
    if (j + 1 < k) {
      const int nrcj = (int)std::max<int64_t>(1, (M - j + kRC - 1) / kRC);
      const dim3 gd((unsigned)nrcj, (unsigned)((k - j - 1 + kCG - 1) / kCG));
      k_hh_dots<<<gd, kT, 0, s>>>(A, M, k, j, o.part2, nrc);
      k_hh_wfin<<<grid_for(k - j - 1, sms), kT, 0, s>>>(o.part2, nrcj, k, j, o.s, (cf64*)o.sw);
      k_hh_update<<<grid_for((M - j) * (k - j - 1), sms), kT, 0, s>>>(A, M, k, j, (const cf64*)o.sw);
    }
  }
  k_aaa_invit<<<1, 1024, 0, s>>>(A, M, k, (const cf64*)o.rdiag, (cf64*)o.w, (cf64*)o.y, o.iters);
  // evaluation: flag = 1 on the support
  e = cudaMemsetAsync(a.flag, 0, (size_t)a.m, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(o.err_bits, 0, 8, s);
  if (e != cudaSuccess) return e;
  k_mark<<<grid_for(k, sms), kT, 0, s>>>(o.sup, k, a.flag, 1);
  k_aaa_eval<<<grid_for(a.m, sms), kT, 0, s>>>(z, f, a.m, o.sup, k, (const cf64*)o.w, a.flag, o.err_bits);
  return cudaGetLastError();
}

cudaError_t aaa_query(const void* t, const void* ft, const void* w, int64_t k, const void* zq, int64_t nq, void* rq,
                      int num_sms, cudaStream_t s) {
  if (nq > 0)
    k_aaa_query<<<grid_for(nq, num_sms), kT, 0, s>>>((const cf64*)t, (const cf64*)ft, (const cf64*)w, k,
                                                      (const cf64*)zq, nq, (cf64*)rq);
  return cudaGetLastError();
}

}  // namespace rplu
