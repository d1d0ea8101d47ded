// Generic per-voxel contribution kernels (any dtype, conventions V and T).
//
// Algorithm 1 of Sec. 3 ("Computing the VCEC") for every voxel: the signed
// count of the faces the voxel introduces, added at its gray value (integer
// images: block-private shared-memory histogram, then int64 global), or
// emitted as a (key, change) pair (float images, Sec. 3 "Other Ranges of Gray
// Values"). Each block owns a tile in the fast axes and marches along the
// slowest axis through a 4-slot ring of halo planes in shared memory, so every
// voxel is read from global memory once per tile plus the one-voxel collar of
// Sec. 3 ("Processing one Chunk"). Outside voxels are +inf (Sec. 4,
// limitations: the second collar of infinite voxels), here by a bounds test.
#include "ecc_tile.cuh"

#include <algorithm>

namespace ecc {

namespace {

constexpr int kThreads = kTileThreads;

template <int MODE>
__device__ void flush_hist(const Sink& s) {
  if (MODE == kSmemHist) flush_smem_hist(s);
}

// ---------------------------------------------------------------------------
// 3D view (z, y, x); tile 32 x 8 in (x, y), marching along z.
// ---------------------------------------------------------------------------
template <typename T, int CONV, int MODE>
__global__ void __launch_bounds__(kThreads)
k_local3(const LocalArgs a, int64_t zc, int64_t tiles_x, int64_t tiles_y, int64_t n_tiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem);
  int8_t* g2 = reinterpret_cast<int8_t*>(ring + 4 * kT3PL);
  Sink s;
  s.bins = a.bins;
  s.vcec = a.vcec;
  s.hist = reinterpret_cast<int*>(g2 + 256);
  s.err = a.err;
  s.pairs = a.pairs;
  s.pair_count = a.pair_count;
  s.pair_cap = a.pair_cap;
  g2[threadIdx.x] = (int8_t)g2_entry(threadIdx.x);
  if (MODE == kSmemHist) clear_smem_hist(s);
  __syncthreads();
  const T* img = static_cast<const T*>(a.img);
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t txy = tiles_x * tiles_y;
    const int64_t tz = t / txy, rem = t - tz * txy;
    const int64_t y0 = (rem / tiles_x) * kT3Y, x0 = (rem % tiles_x) * kT3X;
    const int64_t z0 = a.w_lo + tz * zc, z1 = min(z0 + zc, a.w_hi);
    run_tile3<T, CONV, MODE>(img, a.n[0], a.n[1], a.n[2], a.w_mem_lo, a.w_mem_hi, x0, y0, z0,
                             z1, ring, g2, s);
  }
  flush_hist<MODE>(s);
}

// ---------------------------------------------------------------------------
// 4D view (w, z, y, x); tile 32 x 4 x 2 in (x, y, z), marching along w.
// ---------------------------------------------------------------------------
template <typename T, int CONV, int MODE>
__global__ void __launch_bounds__(kThreads)
k_local4(const LocalArgs a, int64_t wc, int64_t tiles_x, int64_t tiles_y, int64_t tiles_z,
         int64_t n_tiles) {
  constexpr int TX = 32, TY = 4, TZ = 2, PW = TX + 2, PH = TY + 2, PD = TZ + 2;
  constexpr int PL = PW * PH * PD;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem);
  int8_t* g2 = reinterpret_cast<int8_t*>(ring + 4 * PL);
  Sink s;
  s.bins = a.bins;
  s.vcec = a.vcec;
  s.hist = reinterpret_cast<int*>(g2 + 256);
  s.err = a.err;
  s.pairs = a.pairs;
  s.pair_count = a.pair_count;
  s.pair_cap = a.pair_cap;

  const int tid = threadIdx.x, tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
  g2[tid] = (int8_t)g2_entry(tid);
  if (MODE == kSmemHist) clear_smem_hist(s);
  __syncthreads();

  const T* img = static_cast<const T*>(a.img);
  const int64_t nw = a.n[0], nz = a.n[1], ny = a.n[2], nx = a.n[3];
  const int64_t vol = nz * ny * nx;

  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    int64_t r = t;
    const int64_t ix = r % tiles_x; r /= tiles_x;
    const int64_t iy = r % tiles_y; r /= tiles_y;
    const int64_t iz = r % tiles_z; r /= tiles_z;
    const int64_t x0 = ix * TX, y0 = iy * TY, z0 = iz * TZ;
    const int64_t w0 = a.w_lo + r * wc, w1 = min(w0 + wc, a.w_hi);

    auto load_vol = [&](int64_t wp) {
      uint32_t* dst = ring + (int)(wp & 3) * PL;
      for (int i = tid; i < PL; i += kThreads) {
        const int lz = i / (PW * PH), rr = i - lz * PW * PH, ly = rr / PW, lx = rr - ly * PW;
        const int64_t gz = z0 + lz - 1, gy = y0 + ly - 1, gx = x0 + lx - 1;
        uint32_t key = kOutside;
        if (wp >= 0 && wp < nw && gz >= 0 && gz < nz && gy >= 0 && gy < ny && gx >= 0 &&
            gx < nx) {
          if (wp >= a.w_mem_lo && wp < a.w_mem_hi)
            key = load_key(img, (wp - a.w_mem_lo) * vol + (gz * ny + gy) * nx + gx, a.err);
          else
            atomicOr(a.err, kErrOverflow);
        }
        dst[i] = key;
      }
    };

    load_vol(w0 - 1);
    load_vol(w0);
    load_vol(w0 + 1);
    __syncthreads();

    const int64_t gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    const bool valid = gx < nx && gy < ny && gz < nz;
    const int c0 = ((tz + 1) * PH + ty + 1) * PW + tx + 1;
    for (int64_t w = w0; w < w1; ++w) {
      if (w + 2 <= w1) load_vol(w + 2);
      const uint32_t* vm = ring + (int)((w - 1) & 3) * PL;
      const uint32_t* v0 = ring + (int)(w & 3) * PL;
      const uint32_t* vp = ring + (int)((w + 1) & 3) * PL;
      const uint32_t kv = v0[c0];
      // 26-bit masks of the volumes w-1, w, w+1 (layout of g3_of_mask) and the
      // straight neighbours along w.
      uint32_t M0 = 0, Mp = 0, Mm = 0;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            if (dz == 0 && dy == 0 && dx == 0) continue;
            const int o = c0 + (dz * PH + dy) * PW + dx;
            const int bit = dz == 0 ? ring_pos(dy, dx)
                            : (dy == 0 && dx == 0) ? (dz > 0 ? 24 : 25)
                            : (dz > 0 ? 8 : 16) + ring_pos(dy, dx);
            const bool fwd = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
            M0 |= (fwd ? after<true>(v0[o], kv) : after<false>(v0[o], kv)) << bit;
            Mp |= after<true>(vp[o], kv) << bit;
            Mm |= after<false>(vm[o], kv) << bit;
          }
      uint32_t bp = after<true>(vp[c0], kv), bm = after<false>(vm[c0], kv);
      if (CONV == kConvT) {
        M0 = ~M0 & 0x3FFFFFFu; Mp = ~Mp & 0x3FFFFFFu; Mm = ~Mm & 0x3FFFFFFu;
        bp ^= 1u; bm ^= 1u;
      }
      int g = g3_of_mask(M0, g2);
      if (bp) g -= g3_of_mask(M0 & Mp, g2);
      if (bm) g -= g3_of_mask(M0 & Mm, g2);
      const int c = g;  // (-1)^4 G_4 for V; G_4 of the complement for T
      deposit<MODE>(valid, kv, c, s);
      __syncthreads();
    }
  }
  flush_hist<MODE>(s);
}

template <typename T, int CONV, int MODE>
cudaError_t launch_typed(const LocalArgs& a, int num_sms, int64_t* launches) {
  const int64_t wn = a.w_hi - a.w_lo;
  if (wn <= 0) return cudaSuccess;
  size_t hist_bytes = MODE == kSmemHist ? (size_t)a.bins * sizeof(int) : 0;
  if (a.view == 3) {
    const size_t smem = 4 * kT3PL * 4 + 256 + hist_bytes;
    auto kern = k_local3<T, CONV, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles_x = (a.n[2] + 31) / 32, tiles_y = (a.n[1] + 7) / 8;
    const int64_t grid_cap = (int64_t)std::max(per_sm, 1) * num_sms;
    int64_t zc = a.zc;
    if (zc <= 0) {
      // enough tiles to keep every resident block busy about four times
      zc = (wn * tiles_x * tiles_y) / (4 * grid_cap);
      zc = std::max<int64_t>(1, std::min<int64_t>(zc, 64));
    }
    const int64_t tiles_z = (wn + zc - 1) / zc;
    const int64_t n_tiles = tiles_x * tiles_y * tiles_z;
    const int64_t grid = a.grid > 0 ? a.grid : std::min(n_tiles, grid_cap);
    kern<<<(unsigned)grid, kThreads, smem, a.stream>>>(a, zc, tiles_x, tiles_y, n_tiles);
    ++*launches;
    return cudaGetLastError();
  }
  constexpr int PL = 34 * 6 * 4;
  const size_t smem = 4 * PL * 4 + 256 + hist_bytes;
  auto kern = k_local4<T, CONV, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles_x = (a.n[3] + 31) / 32, tiles_y = (a.n[2] + 3) / 4,
                tiles_z = (a.n[1] + 1) / 2;
  const int64_t grid_cap = (int64_t)std::max(per_sm, 1) * num_sms;
  int64_t wc = a.zc;
  if (wc <= 0) {
    wc = (wn * tiles_x * tiles_y * tiles_z) / (4 * grid_cap);
    wc = std::max<int64_t>(1, std::min<int64_t>(wc, 64));
  }
  const int64_t tiles_w = (wn + wc - 1) / wc;
  const int64_t n_tiles = tiles_x * tiles_y * tiles_z * tiles_w;
  const int64_t grid = a.grid > 0 ? a.grid : std::min(n_tiles, grid_cap);
  kern<<<(unsigned)grid, kThreads, smem, a.stream>>>(a, wc, tiles_x, tiles_y, tiles_z, n_tiles);
  ++*launches;
  return cudaGetLastError();
}

template <typename T, int CONV>
cudaError_t launch_mode(const LocalArgs& a, int num_sms, int64_t* launches) {
  if (a.pairs != nullptr) return launch_typed<T, CONV, kPairs>(a, num_sms, launches);
  if (a.bins <= kSmemBinsMax) return launch_typed<T, CONV, kSmemHist>(a, num_sms, launches);
  return launch_typed<T, CONV, kGlobalHist>(a, num_sms, launches);
}

template <typename T>
cudaError_t launch_conv(const LocalArgs& a, int num_sms, int64_t* launches) {
  return a.conv == kConvT ? launch_mode<T, kConvT>(a, num_sms, launches)
                          : launch_mode<T, kConvV>(a, num_sms, launches);
}

}  // namespace

cudaError_t launch_local_generic(const LocalArgs& a, int num_sms, int64_t* launches) {
  const int64_t eb = a.dtype == kU8 ? 1 : a.dtype == kU16 ? 2 : 4;
  if (a.row_pitch > 0 && a.row_pitch != a.n[a.view - 1] * eb) return cudaErrorInvalidValue;
  switch (a.dtype) {
    case kU8: return launch_conv<uint8_t>(a, num_sms, launches);
    case kU16: return launch_conv<uint16_t>(a, num_sms, launches);
    case kF32: return launch_conv<float>(a, num_sms, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ecc
