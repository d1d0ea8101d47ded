// Post-processing of Sec. 3: the curve is the running sum of the VCEC,
// curve[t] = a_0 + ... + a_t (int64 counters, Sec. 3 "Analysis").
#include "ecc_internal.h"
#include "ecc_scan.cuh"

namespace ecc {

namespace {

__global__ void __launch_bounds__(kScanThreads)
k_scan(const long long* __restrict__ vcec, long long* __restrict__ curve, int64_t bins) {
  block_scan_curve(vcec, curve, bins);
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
