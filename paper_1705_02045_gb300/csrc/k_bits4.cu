// Launch of the 4D bit-sliced contribution kernel (ecc_bits4.cuh): blocks
// take (chunk of w, column tile) units chunk-major, so blocks on neighbouring
// tiles march through the same volumes together and share their collar bytes
// in L2.
#include "ecc_bits4.cuh"
#include "occupancy.h"

#include <algorithm>

namespace ecc {

int bits_nb(int dtype, int64_t bins);  // k_bits.cu

namespace {

template <int NB, int CONV, int MODE>
__global__ void __launch_bounds__(32 * k4Warps, 1)
k_bits4(const Bits4Img im, const Bits4Geo geo, int64_t w_lo, int64_t w_hi, int64_t chunks) {
  extern __shared__ __align__(16) uint32_t sm4[];
  constexpr int EB = NB == 32 ? 4 : NB <= 8 ? 1 : 2;
  int* hist = reinterpret_cast<int*>(sm4 + bits4_smem_words<NB>());
  if (MODE == k4Smem)
    for (int64_t b = threadIdx.x; b < im.bins; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const bool fast = ((reinterpret_cast<uintptr_t>(im.img) | (uintptr_t)(im.n[3] * EB)) & 15u) == 0;
  const int64_t wn = w_hi - w_lo, units = geo.cols * chunks;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t k = u / geo.cols, col = u - k * geo.cols;
    const int64_t c0 = wn * k / chunks, c1 = wn * (k + 1) / chunks;
    if (c0 >= c1) continue;
    const int64_t tx = col % geo.tiles_x, r = col / geo.tiles_x;
    const int64_t ty = r % geo.tiles_y, tz = r / geo.tiles_y;
    bits4_span<NB, CONV, MODE>(im, tx, ty, tz, w_lo + c0, w_lo + c1, fast, sm4, hist);
  }
  if (MODE == k4Smem) {
    __syncthreads();
    for (int64_t b = threadIdx.x; b < im.bins; b += blockDim.x) {
      const int v = hist[b];
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(im.vcec) + b,
                       (unsigned long long)(long long)v);
    }
  }
}

// Chunks of w per column: the count that keeps the most block slots busy over
// the rounds of units, discounted by the priming volume each chunk adds.
int64_t bits4_chunks(int64_t cols, int64_t wn, int64_t slots) {
  int64_t best = 1;
  double best_eff = -1.0;
  const int64_t kmax = std::max<int64_t>(1, std::min<int64_t>(wn / 8, 4096));
  for (int64_t K = 1; K <= kmax; ++K) {
    const int64_t units = cols * K;
    const int64_t rounds = (units + slots - 1) / slots;
    const double depth = (double)wn / (double)K;
    const double eff = (double)units / (double)(rounds * slots) * (1.0 - 0.7 / (depth + 0.7));
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = K;
    }
  }
  return best;
}

template <int NB, int CONV, int MODE>
cudaError_t launch4(const LocalArgs& a, int num_sms, int64_t* launches) {
  Bits4Img im{};
  im.img = static_cast<const unsigned char*>(a.img);
  for (int i = 0; i < 4; ++i) im.n[i] = a.n[i];
  im.w_mem_lo = a.w_mem_lo;
  im.w_mem_hi = a.w_mem_hi;
  im.bins = a.bins;
  im.vcec = a.vcec;
  im.err = a.err;
  im.pairs = a.pairs;
  im.pair_count = a.pair_count;
  im.pair_cap = a.pair_cap;
  const size_t smem = bits4_smem_words<NB>() * 4 +
                      (MODE == k4Smem ? sizeof(int) * (size_t)a.bins
                       : MODE == k4Pairs ? sizeof(unsigned long long) * k4Warps * k4PairBuf : 0);
  auto kern = k_bits4<NB, CONV, MODE>;
  int per_sm = 0;
  cudaError_t e = blocks_per_sm(kern, 32 * k4Warps, smem, &per_sm);
  if (e) return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  const Bits4Geo g = bits4_geo(a.n[1], a.n[2], a.n[3]);
  const int64_t wn = a.w_hi - a.w_lo;
  const int64_t slots = a.grid > 0 ? a.grid : (int64_t)per_sm * num_sms;
  const int64_t chunks = bits4_chunks(g.cols, std::max<int64_t>(wn, 1), slots);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(g.cols * chunks, slots));
  kern<<<(unsigned)grid, 32 * k4Warps, smem, a.stream>>>(im, g, a.w_lo, a.w_hi, chunks);
  ++*launches;
  return cudaGetLastError();
}

template <int NB, int MODE>
cudaError_t launch4_conv(const LocalArgs& a, int num_sms, int64_t* launches) {
  return a.conv == kConvT ? launch4<NB, kConvT, MODE>(a, num_sms, launches)
                          : launch4<NB, kConvV, MODE>(a, num_sms, launches);
}

template <int NB>
cudaError_t launch4_hist(const LocalArgs& a, int num_sms, int64_t* launches) {
  return a.bins <= kSmemBinsMax ? launch4_conv<NB, k4Smem>(a, num_sms, launches)
                                : launch4_conv<NB, k4Global>(a, num_sms, launches);
}

}  // namespace

// The 4D bit-sliced kernel where it applies: float32 images emitting pairs,
// or integer images with 256, 16384 or 65536 bins; cudaErrorNotSupported
// otherwise (the caller then uses the generic kernel).
cudaError_t launch_local_bits4(const LocalArgs& a, int num_sms, int64_t* launches) {
  if (a.view != 4) return cudaErrorNotSupported;
  const int64_t eb = a.dtype == kU8 ? 1 : a.dtype == kU16 ? 2 : 4;
  if ((reinterpret_cast<uintptr_t>(a.img) & (uintptr_t)(eb - 1)) != 0) return cudaErrorNotSupported;
  if (a.w_hi <= a.w_lo) return cudaSuccess;
  if (a.pairs != nullptr) {
    if (a.dtype != kF32) return cudaErrorNotSupported;
    return launch4_conv<32, k4Pairs>(a, num_sms, launches);
  }
  switch (bits_nb(a.dtype, a.bins)) {
    case 8: return launch4_hist<8>(a, num_sms, launches);
    case 14: return launch4_hist<14>(a, num_sms, launches);
    case 16: return launch4_hist<16>(a, num_sms, launches);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace ecc
