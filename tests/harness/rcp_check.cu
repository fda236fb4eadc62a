// Exhaustive check of rplu::rcp_nr against the correctly rounded reciprocal
// __frcp_rn: every significand of [1, 2), both signs, exponents -124..123.
// Prints the number of mismatches and the first few operands.
#include <cstdio>
#include <cstdint>
#include <cstring>

#include "rcp.cuh"

__global__ void k_check(int exp_lo, int exp_hi, unsigned long long* bad, uint32_t* first) {
  const uint32_t nsig = 1u << 23;
  const int nexp = exp_hi - exp_lo + 1;
  const uint64_t total = (uint64_t)nsig * nexp * 2;
  for (uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
       id += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t sig = (uint32_t)(id % nsig);
    const uint64_t rest = id / nsig;
    const int e = exp_lo + (int)(rest % nexp);
    const uint32_t sign = (uint32_t)(rest / nexp);
    const uint32_t bits = (sign << 31) | ((uint32_t)(e + 127) << 23) | sig;
    float b;
    memcpy(&b, &bits, 4);
    const float r1 = rplu::rcp_nr(b), r2 = __frcp_rn(b);
    uint32_t u1, u2;
    memcpy(&u1, &r1, 4);
    memcpy(&u2, &r2, 4);
    if (u1 != u2) {
      const unsigned long long k = atomicAdd(bad, 1ull);
      if (k < 8) first[k] = bits;
    }
  }
}

// rcp_nr64 against 1.0/b on operands spread over the exponent range
// [-1000, 1000] (both signs, pseudo-random significands): the largest
// difference in ulps of 1.0/b.
__global__ void k_check64(unsigned long long* maxulp) {
  const uint64_t total = 1ull << 26;
  unsigned long long worst = 0;
  for (uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
       id += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t h = id * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    const uint64_t sig = h & ((1ull << 52) - 1);
    const int e = -1000 + (int)(id % 2001);
    const uint64_t sign = (id >> 20) & 1;
    const uint64_t bits = (sign << 63) | ((uint64_t)(e + 1023) << 52) | sig;
    double b;
    memcpy(&b, &bits, 8);
    const double r1 = rplu::rcp_nr64(b), r2 = 1.0 / b;
    int64_t u1, u2;
    memcpy(&u1, &r1, 8);
    memcpy(&u2, &r2, 8);
    const unsigned long long d = (unsigned long long)(u1 > u2 ? u1 - u2 : u2 - u1);
    worst = d > worst ? d : worst;
  }
  atomicMax(maxulp, worst);
}

int main() {
  unsigned long long* bad;
  uint32_t* first;
  cudaMalloc(&bad, 8);
  cudaMalloc(&first, 32);
  cudaMemset(bad, 0, 8);
  cudaMemset(first, 0, 32);
  k_check<<<152 * 8, 256>>>(-124, 123, bad, first);
  cudaError_t err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    printf("error %s\n", cudaGetErrorString(err));
    return 2;
  }
  unsigned long long h = 0;
  uint32_t f[8];
  cudaMemcpy(&h, bad, 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(f, first, 32, cudaMemcpyDeviceToHost);
  printf("mismatches %llu\n", h);
  for (unsigned long long k = 0; k < h && k < 8; ++k) printf("operand 0x%08x\n", f[k]);
  cudaMemset(bad, 0, 8);
  k_check64<<<152 * 8, 256>>>(bad);
  err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    printf("error %s\n", cudaGetErrorString(err));
    return 2;
  }
  cudaMemcpy(&h, bad, 8, cudaMemcpyDeviceToHost);
  printf("f64 max ulp %llu\n", h);
  return 0;
}
