// Float images (Sec. 3, "Other Ranges of Gray Values"): the paper keys the
// VCEC by the value in a hash map. Here the contribution kernel emits one
// (key, change) pair per voxel with a non-zero change; this file sorts the
// pairs by key (LSD radix sort, 4 passes of 8 bits over the order-preserving
// 32-bit key), sums the changes of equal keys (the VCEC entry a_t), drops the
// values with a_t = 0, and prefix-sums (Sec. 3 "Post-Processing") so that each
// remaining threshold t carries chi(K_t).
//
// Pair layout: (uint64) key << 32 | (uint32)(int32)change.
//
// chi(K_t) at the last pair of key t is the inclusive prefix sum P of the
// changes over the sorted pairs; a_t = P(end of t) - P(end of the previous
// key). So: (1) compact the segment ends with their P, (2) keep the ends whose
// P differs from the previous end's.
#include "ecc_internal.h"

#include <algorithm>

namespace ecc {

namespace {

using u64 = unsigned long long;

constexpr int kRThreads = 256, kRItems = 4, kRTile = kRThreads * kRItems;
constexpr int kSThreads = 256, kSItems = 8, kSTile = kSThreads * kSItems;
constexpr int kWarps = kRThreads / 32;

__device__ __forceinline__ uint32_t key_of(u64 p) { return (uint32_t)(p >> 32); }
__device__ __forceinline__ int change_of(u64 p) { return (int)(uint32_t)p; }

// ---- radix sort -----------------------------------------------------------

__global__ void __launch_bounds__(kRThreads)
k_radix_hist(const u64* __restrict__ in, int64_t n, int shift, unsigned* __restrict__ counts,
             int64_t nblocks, unsigned* __restrict__ digit_tot) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRTile;
  for (int i = threadIdx.x; i < kRTile; i += kRThreads) {
    const int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(in[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  const unsigned c = h[threadIdx.x];
  counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = c;
  if (c) atomicAdd(&digit_tot[threadIdx.x], c);
}

// Block d turns row d of `counts` into global output offsets: the number of
// items with a smaller digit, plus those with digit d in earlier tiles.
__global__ void __launch_bounds__(1024)
k_radix_offsets(unsigned* __restrict__ counts, int64_t nblocks,
                const unsigned* __restrict__ digit_tot) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned s_base;
  const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    unsigned b = 0;
    for (int e = 0; e < d; ++e) b += digit_tot[e];
    s_base = b;
  }
  __syncthreads();
  unsigned carry = s_base;
  unsigned* row = counts + (int64_t)d * nblocks;
  for (int64_t b0 = 0; b0 < nblocks; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    const unsigned v = i < nblocks ? row[i] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned w = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += y;
      }
      warp_tot[lane] = w;
    }
    __syncthreads();
    const unsigned excl = carry + (warp ? warp_tot[warp - 1] : 0u) + x - v;
    if (i < nblocks) row[i] = excl;
    carry += warp_tot[31];
    __syncthreads();
  }
}

// Stable scatter: items are taken in rounds of 256 (round-major, then thread
// order, which is the input order), ranked among equal digits by warp match
// and a per-round prefix over warps.
__global__ void __launch_bounds__(kRThreads)
k_radix_scatter(const u64* __restrict__ in, u64* __restrict__ out, int64_t n, int shift,
                const unsigned* __restrict__ offsets, int64_t nblocks) {
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[kWarps][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offsets[(int64_t)tid * nblocks + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kRItems; ++r) {
    const int64_t idx = base + (int64_t)r * kRThreads + tid;
    const bool ok = idx < n;
    const u64 item = ok ? in[idx] : 0ull;
    const unsigned d = ok ? (unsigned)((item >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    const unsigned rank = __popc(peers & lt);
    if (ok && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    unsigned acc = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const unsigned c = wcnt[w][tid];
      wcnt[w][tid] = acc;
      acc += c;
    }
    __syncthreads();
    if (ok) out[run[d] + wcnt[warp][d] + rank] = item;
    __syncthreads();
    run[tid] += acc;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
  }
}

// ---- block scan helpers (blocked arrangement, kSThreads threads) ------------

template <typename V>
__device__ V block_excl_scan(V v, V* total) {
  __shared__ V warp_tot[kSThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    V w = lane < kSThreads / 32 ? warp_tot[lane] : V(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const V y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kSThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  const V excl = (warp ? warp_tot[warp - 1] : V(0)) + x - v;
  *total = warp_tot[kSThreads / 32 - 1];
  __syncthreads();
  return excl;
}

__device__ __forceinline__ bool is_end(const u64* s, int64_t i, int64_t n) {
  return i == n - 1 || key_of(s[i + 1]) != key_of(s[i]);
}

// Per tile: sum of changes and number of segment ends.
__global__ void __launch_bounds__(kSThreads)
k_seg_totals(const u64* __restrict__ s, int64_t n, long long* __restrict__ tile_sum,
             unsigned* __restrict__ tile_ends) {
  const int64_t base = (int64_t)blockIdx.x * kSTile + (int64_t)threadIdx.x * kSItems;
  long long sum = 0;
  unsigned ends = 0;
  for (int j = 0; j < kSItems; ++j) {
    const int64_t i = base + j;
    if (i < n) {
      sum += change_of(s[i]);
      ends += is_end(s, i, n) ? 1u : 0u;
    }
  }
  long long ts;
  unsigned te;
  block_excl_scan<long long>(sum, &ts);
  block_excl_scan<unsigned>(ends, &te);
  if (threadIdx.x == 0) {
    tile_sum[blockIdx.x] = ts;
    tile_ends[blockIdx.x] = te;
  }
}

// Exclusive scans of per-tile totals (one block); writes the grand totals.
template <typename V>
__global__ void __launch_bounds__(kSThreads)
k_scan_tiles(V* __restrict__ t, int64_t ntiles, V* __restrict__ grand) {
  V carry = 0;
  for (int64_t b0 = 0; b0 < ntiles; b0 += kSThreads) {
    const int64_t i = b0 + threadIdx.x;
    const V v = i < ntiles ? t[i] : V(0);
    V tot;
    const V ex = block_excl_scan<V>(v, &tot);
    if (i < ntiles) t[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *grand = carry;
}

// Writes every segment end's key and inclusive prefix sum P.
__global__ void __launch_bounds__(kSThreads)
k_seg_emit(const u64* __restrict__ s, int64_t n, const long long* __restrict__ tile_sum,
           const unsigned* __restrict__ tile_ends, uint32_t* __restrict__ e_key,
           long long* __restrict__ e_p) {
  const int64_t base = (int64_t)blockIdx.x * kSTile + (int64_t)threadIdx.x * kSItems;
  long long sum = 0;
  unsigned ends = 0;
  for (int j = 0; j < kSItems; ++j) {
    const int64_t i = base + j;
    if (i < n) {
      sum += change_of(s[i]);
      ends += is_end(s, i, n) ? 1u : 0u;
    }
  }
  long long ts;
  unsigned te;
  long long p = tile_sum[blockIdx.x] + block_excl_scan<long long>(sum, &ts);
  unsigned pos = tile_ends[blockIdx.x] + block_excl_scan<unsigned>(ends, &te);
  for (int j = 0; j < kSItems; ++j) {
    const int64_t i = base + j;
    if (i < n) {
      p += change_of(s[i]);
      if (is_end(s, i, n)) {
        e_key[pos] = key_of(s[i]);
        e_p[pos] = p;
        ++pos;
      }
    }
  }
}

__device__ __forceinline__ bool nz_at(const long long* e_p, int64_t k) {
  return e_p[k] != (k ? e_p[k - 1] : 0ll);
}

__global__ void __launch_bounds__(kSThreads)
k_nz_totals(const long long* __restrict__ e_p, const unsigned* __restrict__ m_ptr,
            unsigned* __restrict__ tile_nz) {
  const int64_t m = *m_ptr;
  const int64_t base = (int64_t)blockIdx.x * kSTile + (int64_t)threadIdx.x * kSItems;
  unsigned cnt = 0;
  for (int j = 0; j < kSItems; ++j) {
    const int64_t k = base + j;
    if (k < m && nz_at(e_p, k)) ++cnt;
  }
  unsigned tot;
  block_excl_scan<unsigned>(cnt, &tot);
  if (threadIdx.x == 0) tile_nz[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kSThreads)
k_nz_emit(const uint32_t* __restrict__ e_key, const long long* __restrict__ e_p,
          const unsigned* __restrict__ m_ptr, const unsigned* __restrict__ tile_nz,
          uint32_t* __restrict__ out_val, long long* __restrict__ out_chi) {
  const int64_t m = *m_ptr;
  const int64_t base = (int64_t)blockIdx.x * kSTile + (int64_t)threadIdx.x * kSItems;
  unsigned cnt = 0;
  for (int j = 0; j < kSItems; ++j) {
    const int64_t k = base + j;
    if (k < m && nz_at(e_p, k)) ++cnt;
  }
  unsigned tot;
  unsigned pos = tile_nz[blockIdx.x] + block_excl_scan<unsigned>(cnt, &tot);
  for (int j = 0; j < kSItems; ++j) {
    const int64_t k = base + j;
    if (k < m && nz_at(e_p, k)) {
      // the threshold itself: the order-preserving key mapped back to the
      // float's bits (negative values were stored complemented)
      const uint32_t key = e_key[k];
      out_val[pos] = (key & 0x80000000u) ? (key & 0x7FFFFFFFu) : ~key;
      out_chi[pos] = e_p[k];
      ++pos;
    }
  }
}

__global__ void k_count_to_u64(const unsigned* src, unsigned long long* dst) { *dst = *src; }

struct TmpLayout {
  size_t alt, counts, digit_tot, tile_sum, tile_ends, tile_nz, e_key, e_p, m, nz, grand, total;
};

TmpLayout layout(int64_t n) {
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const int64_t rb = (n + kRTile - 1) / kRTile, sb = (n + kSTile - 1) / kSTile;
  TmpLayout L{};
  size_t o = 0;
  L.alt = o; o += up(sizeof(u64) * std::max<int64_t>(n, 1));
  L.counts = o; o += up(sizeof(unsigned) * 256 * std::max<int64_t>(rb, 1));
  L.digit_tot = o; o += up(sizeof(unsigned) * 256);
  L.tile_sum = o; o += up(sizeof(long long) * std::max<int64_t>(sb, 1));
  L.tile_ends = o; o += up(sizeof(unsigned) * std::max<int64_t>(sb, 1));
  L.tile_nz = o; o += up(sizeof(unsigned) * std::max<int64_t>(sb, 1));
  L.e_key = o; o += up(sizeof(uint32_t) * std::max<int64_t>(n, 1));
  L.e_p = o; o += up(sizeof(long long) * std::max<int64_t>(n, 1));
  L.m = o; o += up(sizeof(unsigned));
  L.nz = o; o += up(sizeof(unsigned));
  L.grand = o; o += up(sizeof(long long));
  L.total = o;
  return L;
}

}  // namespace

size_t float_tail_tmp_bytes(int64_t n) { return layout(n).total; }

cudaError_t launch_float_tail(unsigned long long* pairs, int64_t n, void* tmp, size_t tmp_bytes,
                              uint32_t* out_vals, long long* out_chi,
                              unsigned long long* out_count, cudaStream_t stream,
                              int64_t* launches) {
  const TmpLayout L = layout(n);
  if (tmp_bytes < L.total) return cudaErrorInvalidValue;
  char* t = static_cast<char*>(tmp);
  if (n <= 0) return cudaMemsetAsync(out_count, 0, sizeof(unsigned long long), stream);
  u64* a = pairs;
  u64* b = reinterpret_cast<u64*>(t + L.alt);
  unsigned* counts = reinterpret_cast<unsigned*>(t + L.counts);
  unsigned* digit_tot = reinterpret_cast<unsigned*>(t + L.digit_tot);
  const int64_t rb = (n + kRTile - 1) / kRTile;
  cudaError_t e;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 32 + 8 * pass;
    if ((e = cudaMemsetAsync(digit_tot, 0, 256 * sizeof(unsigned), stream)) != cudaSuccess)
      return e;
    k_radix_hist<<<(unsigned)rb, kRThreads, 0, stream>>>(a, n, shift, counts, rb, digit_tot);
    k_radix_offsets<<<256, 1024, 0, stream>>>(counts, rb, digit_tot);
    k_radix_scatter<<<(unsigned)rb, kRThreads, 0, stream>>>(a, b, n, shift, counts, rb);
    *launches += 3;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(a, b);
  }
  // after 4 passes the sorted pairs are back in `pairs` (a == pairs)
  const int64_t sb = (n + kSTile - 1) / kSTile;
  long long* tile_sum = reinterpret_cast<long long*>(t + L.tile_sum);
  unsigned* tile_ends = reinterpret_cast<unsigned*>(t + L.tile_ends);
  unsigned* tile_nz = reinterpret_cast<unsigned*>(t + L.tile_nz);
  uint32_t* e_key = reinterpret_cast<uint32_t*>(t + L.e_key);
  long long* e_p = reinterpret_cast<long long*>(t + L.e_p);
  unsigned* m = reinterpret_cast<unsigned*>(t + L.m);
  unsigned* nz = reinterpret_cast<unsigned*>(t + L.nz);
  long long* grand_sum = reinterpret_cast<long long*>(t + L.grand);  // unused grand total
  k_seg_totals<<<(unsigned)sb, kSThreads, 0, stream>>>(a, n, tile_sum, tile_ends);
  k_scan_tiles<long long><<<1, kSThreads, 0, stream>>>(tile_sum, sb, grand_sum);
  k_scan_tiles<unsigned><<<1, kSThreads, 0, stream>>>(tile_ends, sb, m);
  k_seg_emit<<<(unsigned)sb, kSThreads, 0, stream>>>(a, n, tile_sum, tile_ends, e_key, e_p);
  k_nz_totals<<<(unsigned)sb, kSThreads, 0, stream>>>(e_p, m, tile_nz);
  k_scan_tiles<unsigned><<<1, kSThreads, 0, stream>>>(tile_nz, sb, nz);
  k_nz_emit<<<(unsigned)sb, kSThreads, 0, stream>>>(e_key, e_p, m, tile_nz, out_vals, out_chi);
  k_count_to_u64<<<1, 1, 0, stream>>>(nz, out_count);
  *launches += 8;
  return cudaGetLastError();
}

}  // namespace ecc
