// One tile of the generic 3D contribution kernel, shared by the single-image
// kernel (k_local.cu) and the batched persistent kernel (batch.cu).
//
// A block of 256 threads owns a 128 x 8 column tile (x, y) and marches along
// z over planes [z0, z1). Planes z-1 .. z+1 (plus the one-voxel collar in x
// and y, Sec. 3 "Processing one Chunk") sit in a 4-slot ring in shared
// memory; plane z+2 is fetched while plane z is evaluated, one barrier per
// plane.
#pragma once

#include "ecc_device.cuh"
#include "ecc_internal.h"

namespace ecc {

constexpr int kTileThreads = 256;
// 3D tiles: 128 x 8 voxels (x, y), 4 consecutive x voxels per thread; halo
// rows of 130 keys padded to 132 (16-byte aligned rows)
constexpr int kT3X = 128, kT3Y = 8, kT3VX = 4, kT3PW = kT3X + 4, kT3PL = kT3PW * (kT3Y + 2);
enum Mode : int { kSmemHist = 0, kGlobalHist = 1, kPairs = 2 };

// Where the changes go.
struct Sink {
  int64_t bins = 0;
  long long* vcec = nullptr;
  int* hist = nullptr;  // shared memory (kSmemHist)
  int* err = nullptr;
  unsigned long long* pairs = nullptr;
  unsigned long long* pair_count = nullptr;
  int64_t pair_cap = 0;
};

// G_2 straight from its definition: sum over delta in {-1,0,1}^2 of
// (-1)^{nz(delta)} times [all bits of the box B_delta set].
__device__ inline int g2_entry(uint32_t m) {
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

template <int MODE>
__device__ __forceinline__ void deposit(bool valid, uint32_t kv, int c, const Sink& s) {
  if (MODE == kPairs) {
    emit_pair(valid && c != 0, kv, c, s.pairs, s.pair_count, s.pair_cap, s.err);
    return;
  }
  if (!valid || c == 0) return;
  if ((int64_t)kv >= s.bins) {
    atomicOr(s.err, kErrValue);
    return;
  }
  if (MODE == kSmemHist)
    atomicAdd(&s.hist[kv], c);
  else
    atomicAdd(reinterpret_cast<unsigned long long*>(s.vcec) + kv,
              (unsigned long long)(long long)c);
}

// Adds the block histogram to the global int64 VCEC and clears it.
__device__ inline void flush_smem_hist(const Sink& s) {
  __syncthreads();
  for (int64_t b = threadIdx.x; b < s.bins; b += kTileThreads) {
    const int v = s.hist[b];
    if (v != 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(s.vcec) + b,
                (unsigned long long)(long long)v);
      s.hist[b] = 0;
    }
  }
  __syncthreads();
}

__device__ inline void clear_smem_hist(const Sink& s) {
  for (int64_t b = threadIdx.x; b < s.bins; b += kTileThreads) s.hist[b] = 0;
  __syncthreads();
}

// Float images keep their values (as bits) in the halo ring, +inf outside,
// and compare them as floats (same order as the keys: -0 equals +0, NaN is
// rejected), the bit added by an integer multiply-add on the FMA pipe;
// integer images keep their keys and the compare-select-or form.
template <typename T>
constexpr bool kFloatRing3 = sizeof(T) == 4;

template <typename T, bool kForward>
__device__ __forceinline__ uint32_t add_after3(uint32_t m, uint32_t ku, uint32_t kv, int bit) {
  if constexpr (kFloatRing3<T>) {
    uint32_t s;
    if (kForward)
      asm("set.ge.u32.f32 %0, %1, %2;" : "=r"(s) : "f"(__uint_as_float(ku)), "f"(__uint_as_float(kv)));
    else
      asm("set.gt.u32.f32 %0, %1, %2;" : "=r"(s) : "f"(__uint_as_float(ku)), "f"(__uint_as_float(kv)));
    return m - s * (1u << bit);
  } else {
    return m | (after<kForward>(ku, kv) << bit);
  }
}

__device__ __forceinline__ void load6_3(const uint32_t* p, uint32_t k[6]) {
  const uint4 q = *reinterpret_cast<const uint4*>(p);
  const uint2 r = *reinterpret_cast<const uint2*>(p + 4);
  k[0] = q.x;
  k[1] = q.y;
  k[2] = q.z;
  k[3] = q.w;
  k[4] = r.x;
  k[5] = r.y;
}

// One 128 x 8 tile, planes [z0, z1). Each thread owns 4 consecutive x voxels
// of one row: the 6 keys of a neighbour row they need are one 16-byte and one
// 8-byte shared-memory load. Plane z + 2 is fetched into registers while
// plane z is evaluated and stored (converted to keys) afterwards.
template <typename T, int CONV, int MODE>
__device__ void run_tile3(const T* img, int64_t nz, int64_t ny, int64_t nx, int64_t mem_lo,
                          int64_t mem_hi, int64_t x0, int64_t y0, int64_t z0, int64_t z1,
                          uint32_t* ring, const int8_t* g2, const Sink& s) {
  constexpr int PW = kT3PW, PL = kT3PL, kRowKeys = kT3X + 2, kRows = kT3Y + 2;
  constexpr int kWarps = kTileThreads / 32;
  constexpr int kRowsPerWarp = (kRows + kWarps - 1) / kWarps, kKeysPerLane = (kRowKeys + 31) / 32;
  const int tid = threadIdx.x, tx = tid % (kT3X / kT3VX), ty = tid / (kT3X / kT3VX);
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t plane = ny * nx;

  struct Fetched {
    T v[kRowsPerWarp][kKeysPerLane];
    uint32_t in;
  };
  auto fetch = [&](int64_t zp, Fetched& f) {
    const bool zok = zp >= 0 && zp < nz;
    const bool resident = zp >= mem_lo && zp < mem_hi;
    if (zok && !resident && tid == 0) atomicOr(s.err, kErrOverflow);
    f.in = 0u;
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i) {
      const int row = warp + i * kWarps;
      const int64_t gy = y0 + row - 1;
      const bool rok = row < kRows && zok && resident && gy >= 0 && gy < ny;
      const int64_t base = rok ? (zp - mem_lo) * plane + gy * nx : 0;
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
  auto store = [&](int64_t zp, const Fetched& f) {
    uint32_t* dst = ring + (int)(zp & 3) * PL;
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i) {
      const int row = warp + i * kWarps;
      if (row >= kRows) continue;
#pragma unroll
      for (int k = 0; k < kKeysPerLane; ++k) {
        const int lx = lane + 32 * k;
        if (lx >= kRowKeys) continue;
        uint32_t key = kFloatRing3<T> ? 0x7F800000u : kOutside;
        if ((f.in >> (i * kKeysPerLane + k)) & 1u) {
          const T v = f.v[i][k];
          if (value_bad(v)) atomicOr(s.err, kErrValue);
          if constexpr (kFloatRing3<T>)
            key = __float_as_uint((float)v);
          else
            key = value_key(v);
        }
        dst[row * PW + lx] = key;
      }
    }
  };

  Fetched f;
  fetch(z0 - 1, f);
  store(z0 - 1, f);
  fetch(z0, f);
  store(z0, f);
  fetch(z0 + 1, f);
  store(z0 + 1, f);
  __syncthreads();

  const int64_t gx0 = x0 + kT3VX * tx, gy = y0 + ty;
  const bool row_valid = gy < ny;
  const int c0 = (ty + 1) * PW + kT3VX * tx;  // halo index of x = gx0 - 1
  for (int64_t z = z0; z < z1; ++z) {
    const bool next = z + 2 <= z1;
    if (next) fetch(z + 2, f);
    const uint32_t* pm = ring + (int)((z - 1) & 3) * PL;
    const uint32_t* p0 = ring + (int)(z & 3) * PL;
    const uint32_t* pp = ring + (int)((z + 1) & 3) * PL;
    uint32_t kc[6];
    load6_3(p0 + c0, kc);
    uint32_t m[kT3VX] = {};
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int o = c0 + dy * PW;
      uint32_t r0[6], rp[6], rm[6];
      load6_3(p0 + o, r0);
      load6_3(pp + o, rp);
      load6_3(pm + o, rm);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
#pragma unroll
        for (int j = 0; j < kT3VX; ++j) {
          const uint32_t kv = kc[j + 1];
          if (dy == 0 && dx == 0) {
            // straight above / below along z
            m[j] = add_after3<T, true>(m[j], rp[j + 1], kv, 24);
            m[j] = add_after3<T, false>(m[j], rm[j + 1], kv, 25);
            continue;
          }
          const int r = ring_pos(dy, dx);
          const bool fwd = dy > 0 || (dy == 0 && dx > 0);
          m[j] = fwd ? add_after3<T, true>(m[j], r0[j + 1 + dx], kv, r)
                     : add_after3<T, false>(m[j], r0[j + 1 + dx], kv, r);
          m[j] = add_after3<T, true>(m[j], rp[j + 1 + dx], kv, 8 + r);
          m[j] = add_after3<T, false>(m[j], rm[j + 1 + dx], kv, 16 + r);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kT3VX; ++j) {
      uint32_t mj = m[j];
      if (CONV == kConvT) mj = ~mj & 0x3FFFFFFu;
      const int g = g3_of_mask(mj, g2);
      const int c = CONV == kConvV ? -g : g;
      const uint32_t kv = kc[j + 1];
      const uint32_t key = kFloatRing3<T> ? value_key(__uint_as_float(kv)) : kv;
      deposit<MODE>(row_valid && gx0 + j < nx, key, c, s);
    }
    // slot (z + 2) & 3 held plane z - 2, which nobody reads after the
    // previous step's barrier
    if (next) store(z + 2, f);
    __syncthreads();
  }
}

}  // namespace ecc
