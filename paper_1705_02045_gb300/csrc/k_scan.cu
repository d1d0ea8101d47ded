// Post-processing of Sec. 3: the curve is the running sum of the VCEC,
// curve[t] = a_0 + ... + a_t (int64 counters, Sec. 3 "Analysis").
#include "ecc_internal.h"

namespace ecc {

namespace {

constexpr int kScanThreads = 1024;

// Inclusive scan of one value per thread across the block; returns the
// block total through *total.
__device__ long long block_inclusive_scan(long long v, long long* total) {
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

// One block walks the bins in rounds of 1024 consecutive entries (coalesced),
// carrying the running total between rounds.
__global__ void __launch_bounds__(kScanThreads)
k_scan(const long long* __restrict__ vcec, long long* __restrict__ curve, int64_t bins) {
  long long carry = 0;
  for (int64_t base = 0; base < bins; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const long long v = i < bins ? vcec[i] : 0;
    long long total;
    const long long inc = block_inclusive_scan(v, &total);
    if (i < bins) curve[i] = carry + inc;
    carry += total;
  }
}

}  // namespace

cudaError_t launch_scan(const long long* vcec, long long* curve, int64_t bins,
                        cudaStream_t stream, int64_t* launches) {
  if (bins <= 0) return cudaSuccess;
  k_scan<<<1, kScanThreads, 0, stream>>>(vcec, curve, bins);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace ecc
