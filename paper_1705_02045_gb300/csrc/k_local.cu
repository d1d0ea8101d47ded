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
#include "ecc_device.cuh"
#include "ecc_internal.h"

#include <algorithm>

namespace ecc {

namespace {

constexpr int kThreads = 256;
enum Mode : int { kSmemHist = 0, kGlobalHist = 1, kPairs = 2 };

// G_2 straight from its definition: sum over delta in {-1,0,1}^2 of
// (-1)^{nz(delta)} times [all bits of the box B_delta set].
__device__ int g2_entry(uint32_t m) {
  int g = 0;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      bool all = true;
      for (int ey = 0; ey <= (dy != 0 ? 1 : 0); ++ey)
        for (int ex = 0; ex <= (dx != 0 ? 1 : 0); ++ex) {
          if (ey == 0 && ex == 0) continue;
          all = all && ((m >> ring_pos(ey * dy, ex * dx)) & 1u);
        }
      if (all) g += ((dy != 0) + (dx != 0)) & 1 ? -1 : 1;
    }
  return g;
}

template <typename T>
__device__ __forceinline__ uint32_t load_key(const T* base, int64_t off, int* err) {
  const T v = base[off];
  if (value_bad(v)) atomicOr(err, kErrValue);
  return value_key(v);
}

// Accumulates one change into the selected output.
template <int MODE>
__device__ __forceinline__ void deposit(bool valid, uint32_t kv, int c, int* hist,
                                        const LocalArgs& a) {
  if (MODE == kPairs) {
    emit_pair(valid && c != 0, kv, c, a.pairs, a.pair_count, a.pair_cap, a.err);
    return;
  }
  if (!valid || c == 0) return;
  if ((int64_t)kv >= a.bins) {
    atomicOr(a.err, kErrValue);
    return;
  }
  if (MODE == kSmemHist)
    atomicAdd(&hist[kv], c);
  else
    atomicAdd(reinterpret_cast<unsigned long long*>(a.vcec) + kv,
              (unsigned long long)(long long)c);
}

template <int MODE>
__device__ void flush_hist(int* hist, const LocalArgs& a) {
  if (MODE != kSmemHist) return;
  __syncthreads();
  for (int64_t b = threadIdx.x; b < a.bins; b += kThreads) {
    const int v = hist[b];
    if (v != 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.vcec) + b,
                (unsigned long long)(long long)v);
  }
}

// ---------------------------------------------------------------------------
// 3D view (z, y, x); tile 32 x 8 in (x, y), marching along z.
// ---------------------------------------------------------------------------
template <typename T, int CONV, int MODE>
__global__ void __launch_bounds__(kThreads)
k_local3(const LocalArgs a, int64_t zc, int64_t tiles_x, int64_t tiles_y, int64_t n_tiles) {
  constexpr int TX = 32, TY = 8, PW = TX + 2, PH = TY + 2, PL = PW * PH;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem);
  int8_t* g2 = reinterpret_cast<int8_t*>(ring + 4 * PL);
  int* hist = reinterpret_cast<int*>(g2 + 256);

  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  g2[tid] = (int8_t)g2_entry(tid);
  if (MODE == kSmemHist)
    for (int64_t b = tid; b < a.bins; b += kThreads) hist[b] = 0;
  __syncthreads();

  const T* img = static_cast<const T*>(a.img);
  const int64_t nz = a.n[0], ny = a.n[1], nx = a.n[2];
  const int64_t plane = ny * nx;

  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t txy = tiles_x * tiles_y;
    const int64_t tz = t / txy, rem = t - tz * txy;
    const int64_t y0 = (rem / tiles_x) * TY, x0 = (rem % tiles_x) * TX;
    const int64_t z0 = a.w_lo + tz * zc, z1 = min(z0 + zc, a.w_hi);

    auto load_plane = [&](int64_t zp) {
      uint32_t* dst = ring + (int)(zp & 3) * PL;
      for (int i = tid; i < PL; i += kThreads) {
        const int ly = i / PW, lx = i - ly * PW;
        const int64_t gy = y0 + ly - 1, gx = x0 + lx - 1;
        uint32_t key = kOutside;
        if (zp >= 0 && zp < nz && gy >= 0 && gy < ny && gx >= 0 && gx < nx) {
          if (zp >= a.w_mem_lo && zp < a.w_mem_hi)
            key = load_key(img, (zp - a.w_mem_lo) * plane + gy * nx + gx, a.err);
          else
            atomicOr(a.err, kErrOverflow);  // plane needed but not resident
        }
        dst[i] = key;
      }
    };

    load_plane(z0 - 1);
    load_plane(z0);
    load_plane(z0 + 1);
    __syncthreads();

    const int64_t gx = x0 + tx, gy = y0 + ty;
    const bool valid = gx < nx && gy < ny;
    for (int64_t z = z0; z < z1; ++z) {
      if (z + 2 <= z1) load_plane(z + 2);
      const uint32_t* pm = ring + (int)((z - 1) & 3) * PL;
      const uint32_t* p0 = ring + (int)(z & 3) * PL;
      const uint32_t* pp = ring + (int)((z + 1) & 3) * PL;
      const int c0 = (ty + 1) * PW + tx + 1;
      const uint32_t kv = p0[c0];
      uint32_t m = 0;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          if (dy == 0 && dx == 0) continue;
          const int o = c0 + dy * PW + dx;
          const int r = ring_pos(dy, dx);
          const bool fwd = dy > 0 || (dy == 0 && dx > 0);
          m |= (fwd ? after<true>(p0[o], kv) : after<false>(p0[o], kv)) << r;
          m |= after<true>(pp[o], kv) << (8 + r);
          m |= after<false>(pm[o], kv) << (16 + r);
        }
      m |= after<true>(pp[c0], kv) << 24;
      m |= after<false>(pm[c0], kv) << 25;
      if (CONV == kConvT) m = ~m & 0x3FFFFFFu;
      const int g = g3_of_mask(m, g2);
      const int c = CONV == kConvV ? -g : g;
      deposit<MODE>(valid, kv, c, hist, a);
      __syncthreads();
    }
  }
  flush_hist<MODE>(hist, a);
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
  int* hist = reinterpret_cast<int*>(g2 + 256);

  const int tid = threadIdx.x, tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
  g2[tid] = (int8_t)g2_entry(tid);
  if (MODE == kSmemHist)
    for (int64_t b = tid; b < a.bins; b += kThreads) hist[b] = 0;
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
      deposit<MODE>(valid, kv, c, hist, a);
      __syncthreads();
    }
  }
  flush_hist<MODE>(hist, a);
}

template <typename T, int CONV, int MODE>
cudaError_t launch_typed(const LocalArgs& a, int num_sms, int64_t* launches) {
  const int64_t wn = a.w_hi - a.w_lo;
  if (wn <= 0) return cudaSuccess;
  size_t hist_bytes = MODE == kSmemHist ? (size_t)a.bins * sizeof(int) : 0;
  if (a.view == 3) {
    constexpr int PL = 34 * 10;
    const size_t smem = 4 * PL * 4 + 256 + hist_bytes;
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
  switch (a.dtype) {
    case kU8: return launch_conv<uint8_t>(a, num_sms, launches);
    case kU16: return launch_conv<uint16_t>(a, num_sms, launches);
    case kF32: return launch_conv<float>(a, num_sms, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ecc
