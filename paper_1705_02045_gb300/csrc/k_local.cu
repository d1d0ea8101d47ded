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
#include "occupancy.h"

#include <algorithm>
#include <type_traits>

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
// 4D view (w, z, y, x); tile 128 x 4 x 2 in (x, y, z), marching along w. Each
// thread owns 4 consecutive voxels in x: the 6 keys of a neighbour row that
// they need (x - 1 .. x + 4) are one 16-byte and one 8-byte shared-memory
// load, so the 80 neighbours of a voxel cost 13.5 loads instead of 80. Halo
// rows hold 130 keys padded to 132 (16-byte aligned rows).
// ---------------------------------------------------------------------------
constexpr int k4TX = 128, k4TY = 4, k4TZ = 2, k4VX = 4;
constexpr int k4PW = 132, k4PH = k4TY + 2, k4PD = k4TZ + 2, k4PL = k4PW * k4PH * k4PD;
static_assert(k4TX / k4VX * k4TY * k4TZ == kThreads, "one thread per 4 voxels");

template <typename T, int CONV, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
k_local4(const LocalArgs a, int64_t wc, int64_t tiles_x, int64_t tiles_y, int64_t tiles_z,
         int64_t n_tiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem);
  int8_t* g2 = reinterpret_cast<int8_t*>(ring + 4 * k4PL);
  Sink s;
  s.bins = a.bins;
  s.vcec = a.vcec;
  s.hist = reinterpret_cast<int*>(g2 + 256);
  s.err = a.err;
  s.pairs = a.pairs;
  s.pair_count = a.pair_count;
  s.pair_cap = a.pair_cap;

  const int tid = threadIdx.x, tx = tid % (k4TX / k4VX), ty = (tid / (k4TX / k4VX)) % k4TY,
            tz = tid / (k4TX / k4VX * k4TY);
  g2[tid] = (int8_t)g2_entry(tid);
  if (MODE == kSmemHist) clear_smem_hist(s);
  __syncthreads();

  const T* img = static_cast<const T*>(a.img);
  const int64_t nw = a.n[0], nz = a.n[1], ny = a.n[2], nx = a.n[3];
  const int64_t vol = nz * ny * nx;
  constexpr int kRowKeys = k4TX + 2;

  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    int64_t r = t;
    const int64_t ix = r % tiles_x; r /= tiles_x;
    const int64_t iy = r % tiles_y; r /= tiles_y;
    const int64_t iz = r % tiles_z; r /= tiles_z;
    const int64_t x0 = ix * k4TX, y0 = iy * k4TY, z0 = iz * k4TZ;
    const int64_t w0 = a.w_lo + r * wc, w1 = min(w0 + wc, a.w_hi);

    // Halo volume wp: 24 rows of 130 keys. Warp v takes rows v, v + 8, v + 16
    // (k4PH * k4PD = 24 = 3 * 8 warps), lane l keys l, l + 32, ... of a row.
    // fetch() issues the global loads into registers; store() writes the keys
    // to the volume's ring slot, so the loads of volume w + 2 are in flight
    // while volume w is evaluated.
    constexpr int kRowsPerWarp = k4PH * k4PD / (kThreads / 32), kKeysPerLane = (kRowKeys + 31) / 32;
    static_assert(kRowsPerWarp * (kThreads / 32) == k4PH * k4PD, "rows split evenly");
    const int warp = tid >> 5, lane = tid & 31;
    // raw values in flight (the key conversion and the NaN / Inf check wait
    // for store(), so the loads do not stall the evaluation of volume w) and
    // a bit per value: inside the image and loaded
    struct Fetched {
      T v[kRowsPerWarp][kKeysPerLane];
      uint32_t in;
    };
    auto fetch = [&](int64_t wp, Fetched& f) {
      const bool wok = wp >= 0 && wp < nw;
      const bool resident = wp >= a.w_mem_lo && wp < a.w_mem_hi;
      if (wok && !resident && tid == 0) atomicOr(a.err, kErrOverflow);
      f.in = 0u;
#pragma unroll
      for (int i = 0; i < kRowsPerWarp; ++i) {
        const int row = warp + i * (kThreads / 32);
        const int lz = row / k4PH, ly = row - lz * k4PH;
        const int64_t gz = z0 + lz - 1, gy = y0 + ly - 1;
        const bool rok = wok && resident && gz >= 0 && gz < nz && gy >= 0 && gy < ny;
        const int64_t base = rok ? (wp - a.w_mem_lo) * vol + (gz * ny + gy) * nx : 0;
#pragma unroll
        for (int k = 0; k < kKeysPerLane; ++k) {
          const int lx = lane + 32 * k;
          const int64_t gx = x0 + lx - 1;
          const bool ok = rok && lx < kRowKeys && gx >= 0 && gx < nx;
          f.v[i][k] = ok ? img[base + gx] : T(0);
          f.in |= (ok ? 1u : 0u) << (i * kKeysPerLane + k);
        }
      }
    };
    auto store = [&](int64_t wp, const Fetched& f) {
      uint32_t* dst = ring + (int)(wp & 3) * k4PL;
#pragma unroll
      for (int i = 0; i < kRowsPerWarp; ++i) {
        const int row = warp + i * (kThreads / 32);
#pragma unroll
        for (int k = 0; k < kKeysPerLane; ++k) {
          const int lx = lane + 32 * k;
          if (lx >= kRowKeys) continue;
          uint32_t key = kFloatRing3<T> ? 0x7F800000u : kOutside;  // +inf / above every key
          if ((f.in >> (i * kKeysPerLane + k)) & 1u) {
            const T v = f.v[i][k];
            if (value_bad(v)) atomicOr(a.err, kErrValue);
            if constexpr (kFloatRing3<T>)
              key = __float_as_uint(v);
            else
              key = value_key(v);
          }
          dst[row * k4PW + lx] = key;
        }
      }
    };
    Fetched kr;
    fetch(w0 - 1, kr);
    store(w0 - 1, kr);
    fetch(w0, kr);
    store(w0, kr);
    fetch(w0 + 1, kr);
    store(w0 + 1, kr);
    __syncthreads();

    const int64_t gx0 = x0 + k4VX * tx, gy = y0 + ty, gz = z0 + tz;
    const bool row_valid = gy < ny && gz < nz;
    // halo index of x = gx0 - 1 in the centre row
    const int c0 = ((tz + 1) * k4PH + ty + 1) * k4PW + k4VX * tx;
    for (int64_t w = w0; w < w1; ++w) {
      const bool next = w + 2 <= w1;
      if (next) fetch(w + 2, kr);
      const uint32_t* vm = ring + (int)((w - 1) & 3) * k4PL;
      const uint32_t* v0 = ring + (int)(w & 3) * k4PL;
      const uint32_t* vp = ring + (int)((w + 1) & 3) * k4PL;
      uint32_t kc[6];
      load6_3(v0 + c0, kc);
      // 26-bit masks (layout of g3_of_mask) of the volumes w, w+1, w-1 for
      // the 4 voxels j (key kc[j + 1]), and the straight neighbours along w
      uint32_t M0[k4VX] = {}, Mp[k4VX] = {}, Mm[k4VX] = {};
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const int o = c0 + (dz * k4PH + dy) * k4PW;
          uint32_t r0[6], rp[6], rm[6];
          load6_3(v0 + o, r0);
          load6_3(vp + o, rp);
          load6_3(vm + o, rm);
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const bool centre = dz == 0 && dy == 0 && dx == 0;
            const int bit = dz == 0 ? (centre ? 0 : ring_pos(dy, dx))
                            : (dy == 0 && dx == 0) ? (dz > 0 ? 24 : 25)
                            : (dz > 0 ? 8 : 16) + ring_pos(dy, dx);
            const bool fwd = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
#pragma unroll
            for (int j = 0; j < k4VX; ++j) {
              const uint32_t kv = kc[j + 1];
              if (centre) continue;
              M0[j] = fwd ? add_after3<T, true>(M0[j], r0[j + 1 + dx], kv, bit)
                          : add_after3<T, false>(M0[j], r0[j + 1 + dx], kv, bit);
              Mp[j] = add_after3<T, true>(Mp[j], rp[j + 1 + dx], kv, bit);
              Mm[j] = add_after3<T, false>(Mm[j], rm[j + 1 + dx], kv, bit);
            }
          }
        }
      // straight neighbours along w (same x, y, z)
      uint32_t kp[6], km[6];
      load6_3(vp + c0, kp);
      load6_3(vm + c0, km);
#pragma unroll
      for (int j = 0; j < k4VX; ++j) {
        const uint32_t kv = kc[j + 1];
        uint32_t m0 = M0[j], mp = Mp[j], mm = Mm[j];
        uint32_t bp = add_after3<T, true>(0u, kp[j + 1], kv, 0);
        uint32_t bm = add_after3<T, false>(0u, km[j + 1], kv, 0);
        if (CONV == kConvT) {
          m0 = ~m0 & 0x3FFFFFFu;
          mp = ~mp & 0x3FFFFFFu;
          mm = ~mm & 0x3FFFFFFu;
          bp ^= 1u;
          bm ^= 1u;
        }
        int g = g3_of_mask(m0, g2);
        if (bp) g -= g3_of_mask(m0 & mp, g2);
        if (bm) g -= g3_of_mask(m0 & mm, g2);
        // (-1)^4 G_4 for V; G_4 of the complement for T
        const uint32_t key = kFloatRing3<T> ? value_key(__uint_as_float(kv)) : kv;
        deposit<MODE>(row_valid && gx0 + j < nx, key, g, s);
      }
      // slot (w + 2) & 3 held volume w - 2, which nobody reads after the
      // previous step's barrier
      if (next) store(w + 2, kr);
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
    int per_sm = 0;
    cudaError_t e = blocks_per_sm(kern, kThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const int64_t tiles_x = (a.n[2] + kT3X - 1) / kT3X, tiles_y = (a.n[1] + kT3Y - 1) / kT3Y;
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
  const size_t smem = 4 * k4PL * 4 + 256 + hist_bytes;
  auto kern = k_local4<T, CONV, MODE>;
  int per_sm = 0;
  cudaError_t e = blocks_per_sm(kern, kThreads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  const int64_t tiles_x = (a.n[3] + k4TX - 1) / k4TX, tiles_y = (a.n[2] + k4TY - 1) / k4TY,
                tiles_z = (a.n[1] + k4TZ - 1) / k4TZ;
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
