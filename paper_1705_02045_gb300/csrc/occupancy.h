// Cached occupancy queries for the contribution kernels (host code).
#pragma once

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include <cuda_runtime.h>

namespace ecc {

// Resident blocks per SM of a kernel for (device, block size, shared memory),
// with the kernel's dynamic shared-memory limit raised as needed: the CUDA
// queries run once per combination, not on every launch (small images are
// bound by the host-side cost of a call).
template <typename Kern>
inline cudaError_t blocks_per_sm(Kern kern, int threads, size_t smem, int* per_sm) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> occ;
  static std::map<std::pair<int, const void*>, size_t> attr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  const void* fn = reinterpret_cast<const void*>(kern);
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple(dev, fn, threads, smem);
  auto it = occ.find(key);
  if (it != occ.end()) {
    *per_sm = it->second;
    return cudaSuccess;
  }
  size_t& limit = attr[std::make_pair(dev, fn)];
  if (limit < smem) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    limit = smem;
  }
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, threads, smem))) return e;
  occ[key] = *per_sm;
  return cudaSuccess;
}

}  // namespace ecc
