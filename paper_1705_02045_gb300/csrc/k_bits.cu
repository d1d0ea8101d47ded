// Single-image launch of the bit-sliced contribution kernel (ecc_bits.cuh):
// a persistent grid walks the tiles of one image, each block keeping a
// private histogram that it adds to the int64 VCEC at the end.
#include "ecc_bits.cuh"
#include "ecc_bitsw.cuh"
#include "occupancy.h"

#include <algorithm>
#include <cstdlib>

namespace ecc {

namespace {

// Warps per block: at most 16 (the launch bound); the default gives 16 rows per
// block (two blocks of 8 warps per SM for rows of <= 512 voxels overlap each
// other's barrier waits: measured faster than one block of 16 warps).
constexpr int kBitsWarps = 16;

// Persistent blocks over the tiles of one image, each with a private
// histogram added to the VCEC at the end.
// Post-processing fused into the contribution launch (Sec. 3 "Post-Processing":
// the curve is the running sum of the VCEC): the block that finishes last
// scans the VCEC into the curve and leaves VCEC and counter at zero for the
// next launch. Any block size that is a multiple of 32.
__device__ void scan_and_clear(long long* vcec, long long* curve, int64_t bins) {
  __shared__ long long wt[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long carry = 0;
  for (int64_t base = 0; base < bins; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    long long v = i < bins ? __ldcg(vcec + i) : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long n = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += n;
    }
    if (lane == 31) wt[warp] = v;
    __syncthreads();
    if (warp == 0) {
      long long w = lane < nw ? wt[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long n = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += n;
      }
      wt[lane] = w;
    }
    __syncthreads();
    if (i < bins) {
      curve[i] = carry + v + (warp > 0 ? wt[warp - 1] : 0);
      vcec[i] = 0;
    }
    carry += wt[nw - 1];
    __syncthreads();
  }
}

template <int HM>
__device__ __forceinline__ void finish_block(const BitsImg& im, int* hist);

template <int NB, int CONV, int HM>
__device__ __forceinline__ void bits_blocks(const BitsImg& im, const BitsGeo& geo, int pl_rec) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int recs = geo.RB * geo.L;  // = blockDim.x
  uint32_t* pl = sm;
  uint32_t* g0 = pl + recs * pl_rec;
  uint32_t* g1 = g0 + recs * kBitsG0Rec;
  int* hist = reinterpret_cast<int*>(g1 + 2 * recs * kBitsG1Rec);
  if (HM == kBitsSmem)
    for (int64_t b = threadIdx.x; b < im.bins; b += blockDim.x) hist[b] = 0;
  if (geo.zc > 0) {
    for (int64_t t = blockIdx.x; t < geo.n_tiles; t += gridDim.x)
      bits_tile<NB, CONV, HM>(im, geo, t, pl, g0, g1, pl_rec, hist);
  } else {
    // balanced: the row columns laid end to end along z, split into equal
    // plane counts per block (a span may cross into the next column)
    const int64_t wn = im.w_hi - im.w_lo, cols = geo.tiles_x * geo.tiles_y;
    const int64_t total = cols * wn;
    int64_t lo = total * blockIdx.x / gridDim.x;
    const int64_t hi = total * (blockIdx.x + 1) / gridDim.x;
    while (lo < hi) {
      const int64_t col = lo / wn, z0 = lo - col * wn;
      const int64_t z1 = min(wn, z0 + (hi - lo));
      const int64_t ty = col / geo.tiles_x, tx = col - ty * geo.tiles_x;
      bits_span<NB, CONV, HM>(im, geo, tx, ty, im.w_lo + z0, im.w_lo + z1, pl, g0, g1, pl_rec,
                              hist);
      lo += z1 - z0;
    }
  }
  finish_block<HM>(im, hist);
}

// End of a block: its shared histogram added to the VCEC, and, with a fused
// scan, the block that finishes last writes the curve.
template <int HM>
__device__ __forceinline__ void finish_block(const BitsImg& im, int* hist) {
  if (HM == kBitsSmem) {
    __syncthreads();
    for (int64_t b = threadIdx.x; b < im.bins; b += blockDim.x) {
      const int v = hist[b];
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(im.vcec) + b,
                       (unsigned long long)(long long)v);
    }
  }
  if (im.curve) {
    __shared__ int last;
    __threadfence();  // this thread's VCEC atomics before the block's ticket
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(im.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      scan_and_clear(im.vcec, im.curve, im.bins);
      if (threadIdx.x == 0) *im.done = 0u;
    }
  }
}

template <int NB, int CONV, int HM>
__global__ void __launch_bounds__(32 * kBitsWarps)
k_bits3(const BitsImg im, const BitsGeo geo, int pl_rec) {
  bits_blocks<NB, CONV, HM>(im, geo, pl_rec);
}

// Warp-column layout (ecc_bitsw.cuh): the planes are cut into K chunks of
// equal depth and the work units (chunk, column) taken in that order, warp
// gw of the grid taking units gw, gw + GW, ...: warps on neighbouring
// columns march through the same planes at the same time, so the rows and
// bytes they share (collar rows and words) are read from DRAM once. The
// block's warps share its histogram only.
constexpr int kBitswWarpsMax = 8;

template <int NB, int CONV, int HM>
__global__ void __launch_bounds__(32 * kBitswWarpsMax, 2)
k_bitsw3(const BitsImg im, const WcGeo geo, int64_t chunks) {
  extern __shared__ __align__(16) int whist[];
  if (HM == kBitsSmem) {
    for (int64_t b = threadIdx.x; b < im.bins; b += blockDim.x) whist[b] = 0;
    __syncthreads();
  }
  const int W = blockDim.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * W + (threadIdx.x >> 5);
  const int64_t GW = (int64_t)gridDim.x * W;
  const bool fast = ((reinterpret_cast<uintptr_t>(im.img) | (uintptr_t)im.row_pitch) & 15u) == 0;
  const int64_t wn = im.w_hi - im.w_lo, units = geo.cols * chunks;
  for (int64_t u = gw; u < units; u += GW) {
    const int64_t k = u / geo.cols, col = u - k * geo.cols;
    const int64_t z0 = wn * k / chunks, z1 = wn * (k + 1) / chunks;
    if (z0 >= z1) continue;
    const int64_t ty = col / geo.tiles_x, tx = col - ty * geo.tiles_x;
    bitsw_span<NB, CONV, HM>(im, tx, ty, im.w_lo + z0, im.w_lo + z1, fast, whist);
  }
  finish_block<HM>(im, whist);
}

// Chunks per column: the count that keeps the most warp slots busy over the
// rounds of units, discounted by the priming plane each chunk adds (about
// 0.6 of a plane's work), with chunks of at least 16 planes where the image
// has them.
inline int64_t bitsw_chunks(int64_t cols, int64_t wn, int64_t warp_slots) {
  int64_t best = 1;
  double best_eff = -1.0;
  const int64_t kmax = std::max<int64_t>(1, std::min<int64_t>(wn / 16, 4096));
  for (int64_t K = 1; K <= kmax; ++K) {
    const int64_t units = cols * K;
    const int64_t rounds = (units + warp_slots - 1) / warp_slots;
    const double depth = (double)wn / (double)K;
    const double eff = (double)units / (double)(rounds * warp_slots) * (1.0 - 0.6 / (depth + 0.6));
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = K;
    }
  }
  return best;
}

template <int NB, int CONV, int HM>
cudaError_t launch_w(const BitsImg& im, int W, int grid_req, int num_sms, cudaStream_t stream,
                     int64_t* launches) {
  const int threads = 32 * W;
  const size_t smem = HM == kBitsSmem ? sizeof(int) * (size_t)im.bins : 0;
  auto kern = k_bitsw3<NB, CONV, HM>;
  int per_sm = 0;
  cudaError_t e = blocks_per_sm(kern, threads, smem, &per_sm);
  if (e) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  const WcGeo g = wc_geo(im.n[2], im.n[1]);
  const int64_t wn = im.w_hi - im.w_lo;
  const int64_t slots = grid_req > 0 ? (int64_t)grid_req * W : (int64_t)per_sm * num_sms * W;
  const int64_t chunks = bitsw_chunks(g.cols, std::max<int64_t>(wn, 1), slots);
  const int64_t units = g.cols * chunks;
  const int64_t grid = grid_req > 0 ? grid_req : std::min<int64_t>((units + W - 1) / W, slots / W);
  kern<<<(unsigned)std::max<int64_t>(grid, 1), threads, smem, stream>>>(im, g, chunks);
  ++*launches;
  return cudaGetLastError();
}

template <int NB>
cudaError_t launch_wnb(const BitsImg& im, int conv, int hist, int W, int grid, int num_sms,
                       cudaStream_t st, int64_t* launches) {
  const bool smem_hist = im.bins <= kSmemBinsMax && hist != 2;
  if (conv == kConvT)
    return smem_hist ? launch_w<NB, kConvT, kBitsSmem>(im, W, grid, num_sms, st, launches)
                     : launch_w<NB, kConvT, kBitsGlobal>(im, W, grid, num_sms, st, launches);
  return smem_hist ? launch_w<NB, kConvV, kBitsSmem>(im, W, grid, num_sms, st, launches)
                   : launch_w<NB, kConvV, kBitsGlobal>(im, W, grid, num_sms, st, launches);
}

template <int NB, int CONV, int HM>
cudaError_t launch_t(const BitsImg& im, int W, int64_t zc, int grid_req, int num_sms,
                     cudaStream_t stream, int64_t* launches) {
  constexpr int pl_rec = (NB + 1) | 1;
  const int threads = 32 * W;
  const size_t words = (size_t)threads * (pl_rec + kBitsG0Rec + 2 * kBitsG1Rec);
  const size_t smem = words * 4 + (HM == kBitsSmem ? sizeof(int) * (size_t)im.bins : 0);
  auto kern = k_bits3<NB, CONV, HM>;
  int per_sm = 0;
  cudaError_t e = blocks_per_sm(kern, threads, smem, &per_sm);
  if (e) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  const int64_t grid_cap = (int64_t)per_sm * num_sms;
  const int64_t wn = im.w_hi - im.w_lo;
  BitsGeo g = bits_geo(im.n[2], im.n[1], wn, W, std::max<int64_t>(zc, 1));
  int64_t grid;
  if (zc <= 0) {
    // balanced spans: every resident block gets the same number of planes
    // (at least 8 where the image has enough, so the one priming plane per
    // span stays small; at least one block per row column for thin images)
    g.zc = 0;
    const int64_t cols = g.tiles_x * g.tiles_y, steps = cols * wn;
    grid = grid_req > 0 ? grid_req
                        : std::max<int64_t>(1, std::min(grid_cap, std::max(cols, steps / 8)));
  } else {
    grid = grid_req > 0 ? grid_req : std::min(g.n_tiles, grid_cap);
  }
  kern<<<(unsigned)grid, threads, smem, stream>>>(im, g, pl_rec);
  ++*launches;
  return cudaGetLastError();
}

template <int NB>
cudaError_t launch_nb(const BitsImg& im, int conv, int hist, int W, int64_t zc, int grid,
                      int num_sms, cudaStream_t st, int64_t* launches) {
  const bool smem_hist = im.bins <= kSmemBinsMax && hist != 2;
  if (conv == kConvT)
    return smem_hist ? launch_t<NB, kConvT, kBitsSmem>(im, W, zc, grid, num_sms, st, launches)
                     : launch_t<NB, kConvT, kBitsGlobal>(im, W, zc, grid, num_sms, st, launches);
  return smem_hist ? launch_t<NB, kConvV, kBitsSmem>(im, W, zc, grid, num_sms, st, launches)
                   : launch_t<NB, kConvV, kBitsGlobal>(im, W, zc, grid, num_sms, st, launches);
}

}  // namespace

int bits_nb(int dtype, int64_t bins) {
  if (dtype == kU8 && bins == 256) return 8;
  if (dtype == kU16 && bins == 16384) return 14;
  if (dtype == kU16 && bins == 65536) return 16;
  return 0;
}

// Returns cudaErrorNotSupported when the bit-sliced kernel does not apply
// (4D view, float values, bins not 256 / 16384 / 65536, a misaligned uint16
// pointer); the caller then uses the generic kernel. Rows may start at any
// byte (16-byte aligned rows take the 128-bit load path).
cudaError_t launch_local_bits(const LocalArgs& a, int num_sms, int64_t* launches) {
  if (a.view != 3 || a.pairs != nullptr) return cudaErrorNotSupported;
  const int nb = bits_nb(a.dtype, a.bins);
  if (!nb) return cudaErrorNotSupported;
  const int eb = a.dtype == kU8 ? 1 : 2;
  const int64_t nx = a.n[2];
  const int64_t pitch = a.row_pitch > 0 ? a.row_pitch : nx * eb;
  if (pitch < nx * eb || (reinterpret_cast<uintptr_t>(a.img) & (uintptr_t)(eb - 1)) != 0)
    return cudaErrorNotSupported;
  BitsImg im{};
  im.img = static_cast<const unsigned char*>(a.img);
  im.n[0] = a.n[0];
  im.n[1] = a.n[1];
  im.n[2] = a.n[2];
  im.row_pitch = pitch;
  im.w_lo = a.w_lo;
  im.w_hi = a.w_hi;
  im.w_mem_lo = a.w_mem_lo;
  im.w_mem_hi = a.w_mem_hi;
  im.bins = a.bins;
  im.vcec = a.vcec;
  im.err = a.err;
  im.curve = a.fused_curve;
  im.done = a.done;
  // layout: warp columns by default for 14- and 16-bit values (measured
  // 1.5x faster on the 14-bit two-phase volume), row groups for 8-bit values
  // (whose 512-voxel rows the 30-voxel column tiles overhang by 12 %)
  const int layout = a.layout != 0 ? a.layout : (nb >= 14 ? 2 : 1);
  if (layout == 2) {
    // warp columns: 8 warps per block by default; a.warps overrides
    const int W = a.warps > 0 ? std::min(a.warps, kBitswWarpsMax) : kBitswWarpsMax;
    switch (nb) {
      case 8: return launch_wnb<8>(im, a.conv, a.hist, W, a.grid, num_sms, a.stream, launches);
      case 14: return launch_wnb<14>(im, a.conv, a.hist, W, a.grid, num_sms, a.stream, launches);
      default: return launch_wnb<16>(im, a.conv, a.hist, W, a.grid, num_sms, a.stream, launches);
    }
  }
  // 16 rows per block by default (8 warps of two 16-lane row groups for rows
  // of <= 512 voxels, 16 warps for rows wider than 1024); a.warps overrides
  int L = 1;
  while (L < (nx + 31) / 32 && L < 32) L <<= 1;
  const int R = 32 / L;  // row groups per warp
  int W = std::max(1, std::min(kBitsWarps, 16 / R));
  if (a.warps > 0) W = std::min(a.warps, kBitsWarps);
  if (W * R < 3) W = (3 + R - 1) / R;  // at least one own row between the collars
  const int64_t zc = a.zc > 0 ? a.zc : 0;
  switch (nb) {
    case 8: return launch_nb<8>(im, a.conv, a.hist, W, zc, a.grid, num_sms, a.stream, launches);
    case 14: return launch_nb<14>(im, a.conv, a.hist, W, zc, a.grid, num_sms, a.stream, launches);
    default: return launch_nb<16>(im, a.conv, a.hist, W, zc, a.grid, num_sms, a.stream, launches);
  }
}

}  // namespace ecc
