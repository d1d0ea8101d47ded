// Device-side building blocks shared by the contribution kernels.
//
// The per-voxel change of Algorithm 1 (Sec. 3, "Tracking the Changes"):
// voxel v introduces the face c of its cell iff every other voxel w containing
// c comes after v in the order (f(w), index(w)); the change is the sum over
// introduced faces of (-1)^dim. Faces of v's cell are indexed by
// delta in {-1,0,1}^d (delta_k = 0: interval along k; +-1: the upper/lower
// endpoint), dim = #zeros(delta); the voxels containing face delta, other than
// v, are the box B_delta = {v + e : e_k in {0, delta_k}} minus v. With the
// "after" bits M of the 3^d - 1 neighbours (a voxel outside the image counts
// as +inf, i.e. after),
//     change_V(v) = (-1)^d G_d(M),   G_d(M) = sum_delta (-1)^{nz(delta)} prod_{B_delta} M.
// The dual-complex convention T (lower star: cells are boxes of voxel centres
// entering at their max) gives change_T(v) = G_d(~M'), M' = "precedes and
// inside" = NOT after, i.e. the same G on the complemented bits.
//
// G factorises along the marching axis: splitting delta = (delta', delta_0),
//     G_d(M) = G_{d-1}(m0) - b+ G_{d-1}(m0 & m+) - b- G_{d-1}(m0 & m-),
// with m0 the in-plane bits, m+- the bits of the planes above/below at the same
// in-plane offsets, and b+- the straight up/down bits. G_2 is a 256-entry
// table over the 8 in-plane bits; G_3 is three lookups, G_4 nine.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ecc_internal.h"

namespace ecc {

// Key of a voxel outside the image: compares above every valid key.
constexpr uint32_t kOutside = 0xFFFFFFFFu;

// Order-preserving keys: comparisons of keys equal comparisons of values.
__device__ __forceinline__ uint32_t value_key(uint8_t v) { return v; }
__device__ __forceinline__ uint32_t value_key(uint16_t v) { return v; }
// IEEE-754 binary32 -> uint32 whose unsigned order is the float order; -0.0
// maps like +0.0 (one value). Finite inputs map below 0xFF800000 < kOutside.
__device__ __forceinline__ uint32_t value_key(float v) {
  uint32_t b = __float_as_uint(v);
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ bool value_bad(uint8_t) { return false; }
__device__ __forceinline__ bool value_bad(uint16_t) { return false; }
__device__ __forceinline__ bool value_bad(float v) {
  return (__float_as_uint(v) & 0x7F800000u) == 0x7F800000u;  // Inf or NaN
}

// In-plane ring position of offset (dy, dx) != (0, 0): row-major over the
// 3x3 neighbourhood with the centre skipped.
__host__ __device__ constexpr int ring_pos(int dy, int dx) {
  return (dy + 1) * 3 + (dx + 1) - ((dy + 1) * 3 + (dx + 1) > 4 ? 1 : 0);
}

// "u after v" for a neighbour at a lexicographically positive offset (u has
// the larger linear index: ties go to u being after) or a negative one.
template <bool kForward>
__device__ __forceinline__ uint32_t after(uint32_t ku, uint32_t kv) {
  return kForward ? (ku >= kv ? 1u : 0u) : (ku > kv ? 1u : 0u);
}

// 26-bit 3D neighbourhood mask layout used by the 3D and 4D kernels:
//   bits 0..7   in-plane ring (dz = 0), ring_pos(dy, dx)
//   bits 8..15  ring of the plane above (dz = +1)
//   bits 16..23 ring of the plane below (dz = -1)
//   bit 24      straight above, bit 25 straight below.
__device__ __forceinline__ int g3_of_mask(uint32_t m, const int8_t* g2) {
  const uint32_t m0 = m & 0xFFu;
  int g = g2[m0];
  g -= ((m >> 24) & 1u) ? g2[m0 & ((m >> 8) & 0xFFu)] : 0;
  g -= ((m >> 25) & 1u) ? g2[m0 & ((m >> 16) & 0xFFu)] : 0;
  return g;
}

// Warp-aggregated append of (key, contribution) pairs. Every lane of the warp
// must call it (active mask = full warp at the call site).
__device__ __forceinline__ void emit_pair(bool has, uint32_t key, int c,
                                          unsigned long long* pairs,
                                          unsigned long long* count, int64_t cap,
                                          int* err) {
  const unsigned full = 0xFFFFFFFFu;
  const unsigned ballot = __ballot_sync(full, has);
  if (ballot == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(ballot) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(ballot));
  base = __shfl_sync(full, base, leader);
  if (has) {
    const unsigned long long slot = base + __popc(ballot & ((1u << lane) - 1u));
    if ((int64_t)slot < cap) {
      pairs[slot] = ((unsigned long long)key << 32) | (uint32_t)c;
    } else {
      atomicOr(err, kErrOverflow);
    }
  }
}

}  // namespace ecc
