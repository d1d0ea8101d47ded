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

// Rounds of kScanThreads bins in one pass of block_scan_curve.
constexpr int kScanRun = 16;

// curve[t] = vcec[0] + ... + vcec[t] (blockDim.x == kScanThreads), in passes
// of kScanRun rounds of kScanThreads consecutive bins: all the pass's loads
// are issued first (coalesced, one per round and thread), every round is
// scanned within its warps by shuffles, warp r then scans round r's warp
// totals, and each thread adds its offsets: three barriers per pass instead
// of three per round.
__device__ inline void block_scan_curve(const long long* vcec, long long* curve, int64_t bins) {
  constexpr int kWarps = kScanThreads / 32;
  static_assert(kWarps == 32 && kScanRun <= kWarps, "one warp total per lane, one warp per round");
  __shared__ long long wpre[kScanRun][kWarps];  // exclusive prefix of each warp in its round
  __shared__ long long rtot[kScanRun];          // round totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned FULL = 0xFFFFFFFFu;
  long long carry = 0;
  const int64_t pass = (int64_t)kScanThreads * kScanRun;
  for (int64_t base = 0; base < bins; base += pass) {
    long long v[kScanRun];
#pragma unroll
    for (int r = 0; r < kScanRun; ++r) {
      const int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
      v[r] = i < bins ? vcec[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < kScanRun; ++r) {
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long n = __shfl_up_sync(FULL, v[r], o);
        if (lane >= o) v[r] += n;
      }
      if (lane == 31) wpre[r][warp] = v[r];
    }
    __syncthreads();
    if (warp < kScanRun) {
      const long long t = wpre[warp][lane];
      long long inc = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long n = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += n;
      }
      wpre[warp][lane] = inc - t;
      if (lane == 31) rtot[warp] = inc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScanRun; ++r) {
      const int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
      if (i < bins) curve[i] = carry + wpre[r][warp] + v[r];
      carry += rtot[r];
    }
    __syncthreads();  // wpre and rtot are rewritten by the next pass
  }
}

}  // namespace ecc
