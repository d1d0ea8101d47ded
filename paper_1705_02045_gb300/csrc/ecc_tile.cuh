// One tile of the generic 3D contribution kernel, shared by the single-image
// kernel (k_local.cu) and the batched persistent kernel (batch.cu).
//
// A block of 256 threads owns a 32 x 8 column tile (x, y) and marches along z
// over planes [z0, z1). Planes z-1 .. z+1 (plus the one-voxel collar in x and
// y, Sec. 3 "Processing one Chunk") sit in a 4-slot ring in shared memory;
// plane z+2 is loaded while plane z is evaluated, one barrier per plane.
#pragma once

#include "ecc_device.cuh"
#include "ecc_internal.h"

namespace ecc {

constexpr int kTileThreads = 256;
constexpr int kT3X = 32, kT3Y = 8, kT3PW = kT3X + 2, kT3PL = kT3PW * (kT3Y + 2);
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

template <typename T, int CONV, int MODE>
__device__ void run_tile3(const T* img, int64_t nz, int64_t ny, int64_t nx, int64_t mem_lo,
                          int64_t mem_hi, int64_t x0, int64_t y0, int64_t z0, int64_t z1,
                          uint32_t* ring, const int8_t* g2, const Sink& s) {
  constexpr int TX = kT3X, PW = kT3PW, PL = kT3PL;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int64_t plane = ny * nx;

  auto load_plane = [&](int64_t zp) {
    uint32_t* dst = ring + (int)(zp & 3) * PL;
    for (int i = tid; i < PL; i += kTileThreads) {
      const int ly = i / PW, lx = i - ly * PW;
      const int64_t gy = y0 + ly - 1, gx = x0 + lx - 1;
      uint32_t key = kOutside;
      if (zp >= 0 && zp < nz && gy >= 0 && gy < ny && gx >= 0 && gx < nx) {
        if (zp >= mem_lo && zp < mem_hi)
          key = load_key(img, (zp - mem_lo) * plane + gy * nx + gx, s.err);
        else
          atomicOr(s.err, kErrOverflow);  // plane needed but not resident
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
    deposit<MODE>(valid, kv, c, s);
    __syncthreads();
  }
}

}  // namespace ecc
