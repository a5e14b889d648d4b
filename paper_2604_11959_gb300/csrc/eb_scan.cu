// eb_scan.cu -- exclusive prefix sum over 64-bit counts (set-up only).
// Three passes: per-block sums, a single-block scan of the block sums, and a
// per-block scan that adds the block's offset.
#include "eb_kernels.cuh"

namespace {
constexpr int SCAN_T = 512;

__device__ long long block_exclusive(long long v, long long *sh, long long *total) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < SCAN_T; o <<= 1) {
    long long add = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  const long long incl = sh[t];
  if (total) *total = sh[SCAN_T - 1];
  __syncthreads();
  return incl - v;
}

__global__ void k_block_sums(const long long *d, long long n, long long *sums) {
  __shared__ long long sh[SCAN_T];
  const long long c = blockIdx.x * (long long)SCAN_T + threadIdx.x;
  long long tot;
  block_exclusive(c < n ? d[c] : 0, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long *sums, long long nb, long long *total) {
  __shared__ long long sh[SCAN_T];
  long long carry = 0;
  for (long long base = 0; base < nb; base += SCAN_T) {
    const long long c = base + threadIdx.x;
    long long tot;
    const long long ex = block_exclusive(c < nb ? sums[c] : 0, sh, &tot);
    if (c < nb) sums[c] = ex + carry;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(long long *d, long long n, const long long *sums) {
  __shared__ long long sh[SCAN_T];
  const long long c = blockIdx.x * (long long)SCAN_T + threadIdx.x;
  const long long ex = block_exclusive(c < n ? d[c] : 0, sh, nullptr);
  if (c < n) d[c] = ex + sums[blockIdx.x];
}
}  // namespace

void scan_exclusive(long long *data, long long n, long long *total, cudaStream_t s) {
  const long long nb = (n + SCAN_T - 1) / SCAN_T;
  long long *sums = total + 1;   // caller provides room for 1 + nb values after `total`
  if (n == 0) {
    cudaMemsetAsync(total, 0, sizeof(long long), s);
    return;
  }
  k_block_sums<<<(unsigned)nb, SCAN_T, 0, s>>>(data, n, sums);
  k_scan_sums<<<1, SCAN_T, 0, s>>>(sums, nb, total);
  k_scan_apply<<<(unsigned)nb, SCAN_T, 0, s>>>(data, n, sums);
}
