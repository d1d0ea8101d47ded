// Block-wide int64 inclusive scan (1024 threads), shared by the single-image and
// the batched post-processing kernels (Sec. 3 "Post-Processing": the curve is
// the running sum of the VCEC).
#pragma once

#include <cstdint>

namespace ecc {

constexpr int kScanThreads = 1024;

__device__ inline long long block_inclusive_scan_i64(long long v, long long* total) {
  __shared__ long long warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    long long w = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long n = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += n;
    }
    warp_tot[lane] = w;
  }
  __syncthreads();
  const long long prefix = warp > 0 ? warp_tot[warp - 1] : 0;
  *total = warp_tot[kScanThreads / 32 - 1];
  __syncthreads();
  return v + prefix;
}

// curve[t] = vcec[0] + ... + vcec[t], walking the bins in coalesced rounds.
__device__ inline void block_scan_curve(const long long* vcec, long long* curve, int64_t bins) {
  long long carry = 0;
  for (int64_t base = 0; base < bins; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const long long v = i < bins ? vcec[i] : 0;
    long long total;
    const long long inc = block_inclusive_scan_i64(v, &total);
    if (i < bins) curve[i] = carry + inc;
    carry += total;
  }
}

}  // namespace ecc
