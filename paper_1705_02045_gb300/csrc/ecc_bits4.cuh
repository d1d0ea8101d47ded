// Bit-sliced contribution kernel for 4D images (integer values or float32
// keys), marching along the slowest axis w.
//
// The quantity is that of Algorithm 1 (Sec. 3): per voxel the signed count of
// the faces it introduces, at its gray value. As in the 3D bit-sliced kernels
// a lane holds 32 voxels of one row as bit planes (float32 values as their
// order-preserving 32-bit keys, 32 planes), each unordered neighbour pair is
// compared once by a borrow chain, and voxels outside the image count as +inf
// (the infinite collar of Sec. 4) through outside masks. In 4D a voxel has 80
// neighbours: 40 later in the linear order, 13 of them in its own volume w
// and 27 in volume w + 1. The change is evaluated through the factorisation
// along w,
//     G_4(M) = G_3(m0) - b+ G_3(m0 & m+) - b- G_3(m0 & m-),
// with m0 the 26 after-bits in the own volume, m+- those of volumes w +- 1 at
// the same 3D offsets and b+- the straight w neighbours; each G_3 is 13 - N
// with N the 26-term count of the 3D kernels.
//
// Layout: a block holds 13 consecutive z-slices of one 30 x 30 (y, x) tile,
// 11 own slices and the z-collar slice below and above them, in 12 warps: a
// warp per own slice and one for both collar slices. A warp holds 32 rows of
// a slice (lanes 0 and 31 the y-collar) and a lane one 32-voxel word (bits 0
// and 31 the x-collar), as in the warp-column layout of the 3D kernel. The
// block marches along w; the bit planes of every slice's rows in volumes w
// and w + 1 sit in shared memory (double-buffered by volume parity), rows
// y +- 1 of a slice come by warp shuffles. The collar warp advances only the
// borrow chains the own slices next to the collar slices read.
// Comparison words travel to the later voxel's row through shared memory:
// those with slice z + 1 within the step, those with volume w + 1 to the next
// step. Two block barriers per step.
#pragma once

#include <type_traits>

#include "ecc_bitsw.cuh"
#include "ecc_device.cuh"

namespace ecc {

constexpr int k4ZB = 11;             // own z-slices per block
constexpr int k4Slices = k4ZB + 2;   // with the collar slice below and above
constexpr int k4Warps = k4ZB + 1;    // a warp per own slice, one for both collar slices

// Slices: z = tz * k4ZB - 1 + slice. Warps 0 .. k4ZB - 1 hold the own slices
// 1 .. k4ZB, warp k4ZB the collar slices 0 and k4ZB + 1. The SM's four
// schedulers take warps by index mod 4: three of them run three own warps,
// the fourth two own warps and the lighter collar warp.

struct Bits4Img {
  const unsigned char* img;  // volume w_mem_lo
  int64_t n[4];              // w, z, y, x
  int64_t w_mem_lo, w_mem_hi;
  int64_t bins;
  long long* vcec;
  int* err;
  unsigned long long* pairs;  // float images: (key << 32 | change)
  unsigned long long* pair_count;
  int64_t pair_cap;
};

struct Bits4Geo {
  int64_t tiles_x, tiles_y, tiles_z, cols;
};

inline Bits4Geo bits4_geo(int64_t nz, int64_t ny, int64_t nx) {
  Bits4Geo g{};
  g.tiles_x = (nx + kWcOwn - 1) / kWcOwn;
  g.tiles_y = (ny + kWcOwn - 1) / kWcOwn;
  g.tiles_z = (nz + k4ZB - 1) / k4ZB;
  g.cols = g.tiles_x * g.tiles_y * g.tiles_z;
  return g;
}

// Pairs a warp gathers in shared memory before appending them to the global
// list (one atomic on its counter per flush).
constexpr int k4PairBuf = 64;

// Shared-memory words of one block: planes of both volumes for every slice,
// the in-volume exports to slice z + 1, the cross exports of two steps.
template <int NB>
constexpr size_t bits4_smem_words() {
  return (size_t)2 * k4Slices * NB * 32 + (size_t)k4Slices * 9 * 32 + (size_t)2 * k4Slices * 27 * 32;
}

namespace b4 {

// 32 x 32 bit transpose: afterwards A[k] bit j = bit k of the original A[j].
// The 16- and 8-bit stages exchange half-words and bytes with one byte
// permutation per output word; the 4-, 2- and 1-bit stages are delta swaps.
__device__ __forceinline__ void transpose32(uint32_t A[32]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t a = A[j], b = A[j | 16];
    A[j] = __byte_perm(a, b, 0x5410);       // low halves of a and b
    A[j | 16] = __byte_perm(a, b, 0x7632);  // high halves
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (j & 8) continue;
    const uint32_t a = A[j], b = A[j | 8];
    A[j] = __byte_perm(a, b, 0x6240);      // bytes 0, 2 of a and b
    A[j | 8] = __byte_perm(a, b, 0x7351);  // bytes 1, 3
  }
  const uint32_t M[3] = {0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int s = 4 >> st;
    const uint32_t m = M[st];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j & s) continue;
      const uint32_t a = A[j], b = A[j | s];
      A[j] = (a & m) | ((b << s) & ~m);
      A[j | s] = ((a >> s) & m) | (b & ~m);
    }
  }
}

// Words [0, 32) of the 32 float32 values starting at voxel x0 (may be -1) of
// a row; voxels outside [0, nx) read as 0. fast: the row starts on a 16-byte
// boundary (16-byte loads; the in-chunk offset is the same in every lane).
__device__ __forceinline__ void load_window4(const unsigned char* row, int64_t x0, int64_t nx,
                                             bool fast, uint32_t* raw) {
  const int64_t vb0 = (x0 < 0 ? 0 : x0) * 4, vb1 = (x0 + 32 < nx ? x0 + 32 : nx) * 4;
  const int64_t s = x0 * 4;
  if (fast) {
    const int64_t a = s & ~int64_t(15);
    const int q = (int)((s - a) >> 2);
    uint32_t w[36];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const int64_t cb = a + 16 * c;
      if (cb + 16 > vb0 && cb < vb1) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + cb));
        w[4 * c] = v.x;
        w[4 * c + 1] = v.y;
        w[4 * c + 2] = v.z;
        w[4 * c + 3] = v.w;
      } else {
        w[4 * c] = w[4 * c + 1] = w[4 * c + 2] = w[4 * c + 3] = 0u;
      }
    }
    // the window's first element is word q of the chunks: one of four unrolled
    // selections
    switch (q) {
#define ECC_B4_SELECT(Q)                                                  \
  case Q:                                                                 \
    _Pragma("unroll") for (int i = 0; i < 32; ++i) raw[i] = w[i + Q];     \
    break;
      ECC_B4_SELECT(0)
      ECC_B4_SELECT(1)
      ECC_B4_SELECT(2)
      ECC_B4_SELECT(3)
#undef ECC_B4_SELECT
    }
  } else {
    // element-aligned words
    const uint32_t* p = reinterpret_cast<const uint32_t*>(row);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int64_t x = x0 + i;
      raw[i] = (x >= 0 && x < nx) ? __ldg(p + x) : 0u;
    }
  }
}

// Bit-sliced 26-term count of the 3D kernels over the neighbour words
// w[dz+1][dy+1][dx+1] (centre unused): faces, complemented edge triples and
// vertex 7-boxes; G_3(w) = 13 - N. n[0..4]: the bit planes of N.
__device__ __forceinline__ void count26(const uint32_t (&w)[3][3][3], uint32_t n[5]) {
  using namespace bits;
  auto W = [&](int dz, int dy, int dx) -> uint32_t { return w[dz + 1][dy + 1][dx + 1]; };
  uint32_t tm[26];
  int t = 0;
  tm[t++] = W(0, 0, 1);
  tm[t++] = W(0, 0, -1);
  tm[t++] = W(0, 1, 0);
  tm[t++] = W(0, -1, 0);
  tm[t++] = W(1, 0, 0);
  tm[t++] = W(-1, 0, 0);
  uint32_t Exy[2][2];
#pragma unroll
  for (int sx = 0; sx < 2; ++sx)
#pragma unroll
    for (int sy = 0; sy < 2; ++sy) {
      const int dx = sx ? 1 : -1, dy = sy ? 1 : -1;
      Exy[sx][sy] = W(0, 0, dx) & W(0, dy, 0) & W(0, dy, dx);
      tm[t++] = ~Exy[sx][sy];
    }
#pragma unroll
  for (int sx = 0; sx < 2; ++sx)
#pragma unroll
    for (int sz = 0; sz < 2; ++sz) {
      const int dx = sx ? 1 : -1, dz = sz ? 1 : -1;
      tm[t++] = ~(W(0, 0, dx) & W(dz, 0, 0) & W(dz, 0, dx));
    }
#pragma unroll
  for (int sy = 0; sy < 2; ++sy)
#pragma unroll
    for (int sz = 0; sz < 2; ++sz) {
      const int dy = sy ? 1 : -1, dz = sz ? 1 : -1;
      tm[t++] = ~(W(0, dy, 0) & W(dz, 0, 0) & W(dz, dy, 0));
    }
#pragma unroll
  for (int sx = 0; sx < 2; ++sx)
#pragma unroll
    for (int sy = 0; sy < 2; ++sy)
#pragma unroll
      for (int sz = 0; sz < 2; ++sz) {
        const int dx = sx ? 1 : -1, dy = sy ? 1 : -1, dz = sz ? 1 : -1;
        tm[t++] = Exy[sx][sy] & W(dz, 0, 0) & W(dz, 0, dx) & W(dz, dy, 0) & W(dz, dy, dx);
      }
  uint32_t s[8], c[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) fa(tm[3 * i], tm[3 * i + 1], tm[3 * i + 2], s[i], c[i]);
  uint32_t a0, a1, a2, d0, d1, d2, b0, e0, e1;
  fa(s[0], s[1], s[2], a0, d0);
  fa(s[3], s[4], s[5], a1, d1);
  fa(s[6], s[7], tm[24], a2, d2);
  fa(a0, a1, a2, b0, e0);
  ha(b0, tm[25], n[0], e1);
  uint32_t f0, f1, f2, f3, q0, q1, q2, q3, h0, i0, i1;
  fa(c[0], c[1], c[2], f0, q0);
  fa(c[3], c[4], c[5], f1, q1);
  fa(c[6], c[7], d0, f2, q2);
  fa(d1, d2, e0, f3, q3);
  fa(f0, f1, f2, h0, i0);
  fa(f3, e1, h0, n[1], i1);
  uint32_t j0, k0, j1, k1, k2;
  fa(q0, q1, q2, j0, k0);
  fa(q3, i0, i1, j1, k1);
  ha(j0, j1, n[2], k2);
  fa(k0, k1, k2, n[3], n[4]);
}

// Bit-sliced sum of two numbers of `bits` planes (LSB first), one more plane out.
template <int BITS>
__device__ __forceinline__ void add_planes(const uint32_t* a, const uint32_t* b, uint32_t* s) {
  uint32_t carry = 0u;
#pragma unroll
  for (int i = 0; i < BITS; ++i) {
    const uint32_t x = a[i] ^ b[i];
    s[i] = x ^ carry;
    carry = (a[i] & b[i]) | (carry & x);
  }
  s[BITS] = carry;
}

}  // namespace b4

// Deposit modes of the 4D kernel.
enum Bits4Mode : int { k4Smem = 0, k4Global = 1, k4Pairs = 2 };

// Borrow-chain groups of one bit plane (bits4_span): the comparisons with
// slice z - 1 in volume w + 1 (A), with slice z + 1 in volumes w and w + 1 (B),
// and those within the own slice (row x + 1, row y + 1, volume w + 1) (C). An
// own slice advances all three, the collar slice below only B (its words with
// slice z + 1 are the ones the first own slice reads), the one above only A.
enum : int { k4GroupA = 1, k4GroupB = 2, k4GroupC = 4 };

// Planes [w0, w1) of the block's column unit (tx, ty, tz). All threads of the
// block call it; blockDim.x = 32 * k4Warps. sm: bits4_smem_words<NB>() words;
// hist: the shared histogram (k4Smem) or the warps' pair buffers (k4Pairs,
// k4Warps x k4PairBuf 8-byte entries; flushed before return).
template <int NB, int CONV, int MODE>
__device__ void bits4_span(const Bits4Img& im, int64_t tx, int64_t ty, int64_t tz, int64_t w0,
                           int64_t w1, bool fast, uint32_t* sm, int* hist) {
  using namespace bits;
  constexpr int EB = NB == 32 ? 4 : NB <= 8 ? 1 : 2;
  constexpr int RAW = 8 * EB;
  const unsigned FULL = 0xFFFFFFFFu, ALL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const bool collar = wi == k4ZB;  // the warp of both collar slices
  const int sl = collar ? 0 : wi + 1;  // own slice (the collar warp: slice 0 first)
  constexpr int kTop = k4ZB + 1;       // the collar slice above
  const int64_t nw = im.n[0], nz = im.n[1], ny = im.n[2], nx = im.n[3];
  const int64_t y = ty * kWcOwn - 1 + lane, x0 = tx * kWcOwn - 1;
  const int64_t z = tz * k4ZB - 1 + sl;
  bool vy[3], vz[3];
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    vy[d + 1] = y + d >= 0 && y + d < ny;
    vz[d + 1] = z + d >= 0 && z + d < nz;
  }
  uint32_t xin;
  {
    const int64_t lo = x0 < 0 ? -x0 : 0, hi = nx - x0 >= 32 ? 32 : nx - x0;
    xin = (hi >= 32 ? FULL : ((1u << hi) - 1u)) & (FULL << lo);
  }
  const bool own = !collar && lane >= 1 && lane <= kWcOwn && vy[1] && vz[1];
  const uint32_t dep = own ? (xin & 0x7FFFFFFEu) : 0u;
  const uint32_t xo = ~xin;
  const uint32_t cx[3] = {xo >> 1, xo, xo << 1};
  const size_t row_bytes = (size_t)nx * EB;
  const int ip = sl + 1, imn = sl > 0 ? sl - 1 : sl;
  // k4Pairs: this warp's pair buffer and its fill (the same in every lane)
  unsigned long long* pbuf = reinterpret_cast<unsigned long long*>(hist) + wi * k4PairBuf;
  int pfill = 0;
  auto flush_pairs = [&]() {
    if (pfill == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(im.pair_count, (unsigned long long)pfill);
    base = __shfl_sync(FULL, base, 0);
    for (int i = lane; i < pfill; i += 32) {
      const unsigned long long slot = base + (unsigned long long)i;
      if ((int64_t)slot < im.pair_cap)
        im.pairs[slot] = pbuf[i];
      else
        atomicOr(im.err, kErrOverflow);
    }
    __syncwarp();
    pfill = 0;
  };

  uint32_t* SP = sm;                                  // [2][k4Slices][NB][32]
  uint32_t* GI = SP + 2 * k4Slices * NB * 32;         // [k4Slices][9][32]
  uint32_t* GC = GI + k4Slices * 9 * 32;              // [2][k4Slices][27][32]
  auto sp_at = [&](int64_t wv, int slice, int k) -> uint32_t* {
    return SP + (((int)(wv & 1) * k4Slices + slice) * NB + k) * 32;
  };
  auto gc_at = [&](int64_t wv, int slice, int dz, int dy, int dx) -> uint32_t* {
    return GC + (((int)(wv & 1) * k4Slices + slice) * 27 + (dz + 1) * 9 + (dy + 1) * 3 + dx + 1) * 32;
  };
  // this lane's row of slice s in volume wp
  auto row_ptr_s = [&](int s, int64_t wp) {
    const int64_t zs = tz * k4ZB - 1 + s;
    return im.img + (((size_t)(wp - im.w_mem_lo) * (size_t)nz + (size_t)zs) * (size_t)ny +
                     (size_t)y) * row_bytes;
  };
  auto row_in = [&](int s, int64_t wp) {
    const int64_t zs = tz * k4ZB - 1 + s;
    return vy[1] && zs >= 0 && zs < nz && wp >= 0 && wp < nw;
  };
  auto load_raw_s = [&](int s, int64_t wp, uint32_t* raw) {
    if (!row_in(s, wp)) return;
    if (wp < im.w_mem_lo || wp >= im.w_mem_hi) {
      atomicOr(im.err, kErrOverflow);
      return;
    }
    if constexpr (EB == 4)
      b4::load_window4(row_ptr_s(s, wp), x0, nx, fast, raw);
    else
      wc::load_window<EB>(row_ptr_s(s, wp), x0, nx, fast, raw);
  };
  // the row's bytes into L2 (its first and last byte: at most 32 voxels + 2,
  // two 128-byte lines for 4-byte values)
  auto prefetch_row_s = [&](int s, int64_t wp) {
    if (!row_in(s, wp) || wp < im.w_mem_lo || wp >= im.w_mem_hi) return;
    const int64_t xa = x0 < 0 ? 0 : x0, xb = (x0 + 32 < nx ? x0 + 32 : nx) - 1;
    const unsigned char* row = row_ptr_s(s, wp);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + xa * EB));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + xb * EB));
  };
  // bit planes of a loaded row of slice s; value checks on the voxels inside
  // the image. Rows outside the image keep whatever planes they get: every
  // comparison with them is replaced through the outside masks.
  auto make_planes_s = [&](int s, int64_t wp, uint32_t* raw, uint32_t* P) {
    const uint32_t inside = row_in(s, wp) ? xin : 0u;
    if constexpr (EB == 4) {
      // order-preserving keys: -0.0 as +0.0, negative values complemented,
      // the sign bit set on the others
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const uint32_t b = raw[i] == 0x80000000u ? 0u : raw[i];
        raw[i] = b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
      }
      b4::transpose32(raw);
      // Inf / NaN (exponent all ones), tested on the key planes: a value of
      // either sign keeps its exponent bits in key bits 23..30, complemented
      // when negative (key bit 31 clear)
      uint32_t e1 = raw[23], e0 = raw[23];
#pragma unroll
      for (int k = 24; k <= 30; ++k) {
        e1 &= raw[k];
        e0 |= raw[k];
      }
      if (((e1 & raw[31]) | (~e0 & ~raw[31])) & inside) atomicOr(im.err, kErrValue);
#pragma unroll
      for (int k = 0; k < 32; ++k) P[k] = raw[k];
    } else if constexpr (EB == 1) {
      transpose8(raw, P);
    } else {
      uint32_t lo[8], hi[8], ph[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        lo[j] = __byte_perm(raw[2 * j], raw[2 * j + 1], 0x6420);
        hi[j] = __byte_perm(raw[2 * j], raw[2 * j + 1], 0x7531);
      }
      transpose8(lo, P);
      transpose8(hi, ph);
      uint32_t extra = 0;
#pragma unroll
      for (int k = 8; k < 16; ++k) {
        if (k < NB) P[k] = ph[k - 8];
        else extra |= ph[k - 8];
      }
      if (extra & inside) atomicOr(im.err, kErrValue);
    }
  };

  uint32_t raw[RAW];
#pragma unroll
  for (int i = 0; i < RAW; ++i) raw[i] = 0u;
  uint32_t Y[NB];  // planes of the volume loaded ahead
  const int64_t ws = w0 == 0 ? w0 : w0 - 1;
  auto prime = [&](int s) {
    load_raw_s(s, ws, raw);
    make_planes_s(s, ws, raw, Y);
#pragma unroll
    for (int k = 0; k < NB; ++k) sp_at(ws, s, k)[lane] = Y[k];
    load_raw_s(s, ws + 1, raw);
    make_planes_s(s, ws + 1, raw, Y);
#pragma unroll
    for (int k = 0; k < NB; ++k) sp_at(ws + 1, s, k)[lane] = Y[k];
    if (w0 == 0) {
      // no volume below the first: its exports are zero (every neighbour
      // there is outside, i.e. after)
#pragma unroll
      for (int e = 0; e < 27; ++e) GC[(((int)((ws - 1) & 1) * k4Slices + s) * 27 + e) * 32 + lane] = 0u;
    }
  };
  prime(sl);
  if (collar) prime(kTop);
  // chains the collar warp does not advance keep these values
  uint32_t bx = 0u, by[3] = {0u, 0u, 0u}, bz[3][3] = {}, bw[3][3][3] = {};
  __syncthreads();

  for (int64_t w = ws; w < w1; ++w) {
    const bool more = w + 2 <= w1;
    // volume w + 2 comes to L2 now and to registers after the comparisons
    if (more) {
      prefetch_row_s(sl, w + 2);
      if (collar) prefetch_row_s(kTop, w + 2);
    }
    // ---- the forward comparisons, bit plane by bit plane
    // Each chain starts at 0 (no borrow) and takes the planes LSB first; the
    // plane loop is unrolled only partly, the planes coming from shared memory.
    constexpr int kUnroll = NB % 8 == 0 ? 8 : NB % 7 == 0 ? 7 : 1;
    // sc: the slice whose rows are compared; s_lo, s_hi: the slices below
    // and above it
    auto advance = [&](auto groups, int sc, int s_lo, int s_hi) {
      constexpr int G = decltype(groups)::value;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if constexpr ((G & k4GroupC) != 0) by[i] = 0u;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if constexpr ((G & k4GroupA) != 0) bw[0][i][j] = 0u;
          if constexpr ((G & k4GroupB) != 0) bz[i][j] = bw[2][i][j] = 0u;
          if constexpr ((G & k4GroupC) != 0) bw[1][i][j] = 0u;
        }
      }
      if constexpr ((G & k4GroupC) != 0) bx = 0u;
#pragma unroll kUnroll
      for (int k = 0; k < NB; ++k) {
        const uint32_t c = sp_at(w, sc, k)[lane];
        const uint32_t C[3] = {c >> 1, c, c << 1};  // [dx+1]: C[i + 1], C[i], C[i - 1]
        // borrow of n - cc through this plane: [n < cc] over the planes so far
        auto chain = [&](uint32_t& b, uint32_t n, uint32_t cc) {
          const uint32_t nn = ~n;
          b = (nn & cc) | (nn & b) | (cc & b);
        };
        auto rows = [&](uint32_t q, uint32_t (&r)[3]) {
          r[0] = __shfl_up_sync(FULL, q, 1);
          r[1] = q;
          r[2] = __shfl_down_sync(FULL, q, 1);
        };
        if constexpr ((G & k4GroupA) != 0) {
          uint32_t r[3];
          rows(sp_at(w + 1, s_lo, k)[lane], r);
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) chain(bw[0][dy][dx], r[dy], C[dx]);
        }
        if constexpr ((G & k4GroupB) != 0) {
          uint32_t r[3], q[3];
          rows(sp_at(w, s_hi, k)[lane], r);
          rows(sp_at(w + 1, s_hi, k)[lane], q);
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
              chain(bz[dy][dx], r[dy], C[dx]);
              chain(bw[2][dy][dx], q[dy], C[dx]);
            }
        }
        if constexpr ((G & k4GroupC) != 0) {
          const uint32_t ny1 = __shfl_down_sync(FULL, c, 1);
          uint32_t r[3];
          rows(sp_at(w + 1, sc, k)[lane], r);
          chain(bx, c, C[2]);
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            chain(by[dx], ny1, C[dx]);
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) chain(bw[1][dy][dx], r[dy], C[dx]);
          }
        }
      }
    };
    if (!collar) {
      advance(std::integral_constant<int, k4GroupA | k4GroupB | k4GroupC>{}, sl, imn, ip);
    } else {
      advance(std::integral_constant<int, k4GroupB>{}, 0, 0, 1);
      advance(std::integral_constant<int, k4GroupA>{}, kTop, k4ZB, kTop);
    }
    if (more) load_raw_s(sl, w + 2, raw);
    const bool w_in = w >= 0 && w < nw, w1_in = w + 1 >= 0 && w + 1 < nw;
    const bool c_in = vy[1] && vz[1] && w_in;
    const uint32_t co[3] = {c_in ? cx[0] : ALL, c_in ? cx[1] : ALL, c_in ? cx[2] : ALL};
    const uint32_t Gx = gcmp(bx, co[2], c_in ? xo : ALL);
    uint32_t Gy[3], Gz[3][3], Gw[3][3][3];
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      Gy[dx] = gcmp(by[dx], co[dx], (vy[2] && vz[1] && w_in) ? xo : ALL);
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        Gz[dy][dx] = gcmp(bz[dy][dx], co[dx], (vy[dy] && vz[2] && w_in) ? xo : ALL);
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
          Gw[dz][dy][dx] = gcmp(bw[dz][dy][dx], co[dx], (vy[dy] && vz[dz] && w1_in) ? xo : ALL);
      }
    }
    // ---- exports: to slice z + 1 (this step) and to volume w + 1 (next step),
    // the words some own slice reads
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) GI[((sl * 9) + dy * 3 + dx) * 32 + lane] = Gz[dy][dx];
    if (!collar) {
#pragma unroll
      for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) gc_at(w, sl, dz - 1, dy - 1, dx - 1)[lane] = Gw[dz][dy][dx];
    } else {
      // slice 0: its words with slice 1 of volume w + 1; the top collar
      // slice: its words with the slice below it in volume w + 1, under that
      // slice's own outside masks
      const int64_t zt = tz * k4ZB - 1 + kTop;
      const bool vzt0 = zt - 1 >= 0 && zt - 1 < nz, vzt1 = zt >= 0 && zt < nz;
      const bool ct_in = vy[1] && vzt1 && w_in;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          gc_at(w, 0, 1, dy - 1, dx - 1)[lane] = Gw[2][dy][dx];
          gc_at(w, kTop, -1, dy - 1, dx - 1)[lane] =
              gcmp(bw[0][dy][dx], ct_in ? cx[dx] : ALL, (vy[dy] && vzt0 && w1_in) ? xo : ALL);
        }
    }
    uint32_t Gydn[3];  // row y - 1's (0, 0, +1, dx) words
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) Gydn[dx] = __shfl_up_sync(FULL, Gy[dx], 1);
    // the planes of volume w + 2, stored once every warp is done with volume w
    if (more) make_planes_s(sl, w + 2, raw, Y);
    if (more && collar) load_raw_s(kTop, w + 2, raw);
    __syncthreads();
    if (more) {
#pragma unroll
      for (int k = 0; k < NB; ++k) sp_at(w + 2, sl, k)[lane] = Y[k];
      if (collar) {
        make_planes_s(kTop, w + 2, raw, Y);
#pragma unroll
        for (int k = 0; k < NB; ++k) sp_at(w + 2, kTop, k)[lane] = Y[k];
      }
    }
    // ---- the change evaluation and deposits
    uint32_t nzm = 0u;
    uint32_t D[8];  // the change as 8-bit two's complement planes
    if (w >= w0 && dep) {
      uint32_t A[5], Bp[5], Bm[5], bp = 0u, bm = 0u;
      auto sh = [](uint32_t g, int dx) -> uint32_t { return dx > 0 ? g >> 1 : dx < 0 ? g << 1 : g; };
      auto gen = [](uint32_t v) -> uint32_t { return CONV == kConvV ? v : ~v; };
      uint32_t w0b[3][3][3], t[3][3][3];
      // in-volume after-bits; the words this warp exported are read back from
      // shared memory rather than kept in registers across the barrier
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          w0b[2][dy + 1][dx + 1] = gen(sh(GI[((sl * 9) + (dy + 1) * 3 + (dx + 1)) * 32 + lane], dx));
          w0b[0][dy + 1][dx + 1] =
              gen(~GI[((imn * 9) + (1 - dy) * 3 + (1 - dx)) * 32 + ((lane + dy) & 31)]);
        }
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        w0b[1][2][dx + 1] = gen(sh(Gy[dx + 1], dx));
        w0b[1][0][dx + 1] = gen(~Gydn[1 - dx]);
      }
      w0b[1][1][2] = gen(sh(Gx, 1));
      w0b[1][1][0] = gen(~Gx);
      w0b[1][1][1] = 0u;
      b4::count26(w0b, A);
      // volume w + 1
#pragma unroll
      for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx)
            t[dz][dy][dx] = w0b[dz][dy][dx] & gen(sh(gc_at(w, sl, dz - 1, dy - 1, dx - 1)[lane], dx - 1));
      bp = gen(gc_at(w, sl, 0, 0, 0)[lane]);
      b4::count26(t, Bp);
      // volume w - 1: the words volume w - 1 exported last step, complemented
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const int sn = dz < 0 ? imn : dz > 0 ? ip : sl;
            t[dz + 1][dy + 1][dx + 1] =
                w0b[dz + 1][dy + 1][dx + 1] &
                gen(~gc_at(w - 1, sn, -dz, -dy, -dx)[(lane + dy) & 31]);
          }
      bm = gen(~gc_at(w - 1, sl, 0, 0, 0)[lane]);
      b4::count26(t, Bm);
      // change = (13 + bp Bp + bm Bm) - (A + 13 bp + 13 bm); zero where both
      // sides agree plane by plane
      uint32_t L1[6], L[7], R1[6], R[7];
      const uint32_t c13p[5] = {bp, 0u, bp, bp, 0u}, c13m[6] = {bm, 0u, bm, bm, 0u, 0u};
      b4::add_planes<5>(A, c13p, L1);
      b4::add_planes<6>(L1, c13m, L);
      uint32_t xp[5], xm[5];
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        xp[b] = Bp[b] & bp;
        xm[b] = Bm[b] & bm;
      }
      b4::add_planes<5>(xp, xm, R1);
      const uint32_t c13[6] = {ALL, 0u, ALL, ALL, 0u, 0u};
      b4::add_planes<6>(R1, c13, R);
      // D = R - L = R + ~L + 1 over 8 planes (L, R < 128)
      uint32_t carry = ALL, any = 0u;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const uint32_t lb = b < 7 ? ~L[b] : ALL, rb = b < 7 ? R[b] : 0u;
        const uint32_t x = rb ^ lb;
        D[b] = x ^ carry;
        carry = (rb & lb) | (carry & x);
        any |= D[b];
      }
      nzm = any & dep;
    }
    // deposits: one voxel per lane and round (the pair append is warp-wide)
    const unsigned char* rowz = row_ptr_s(sl, w);
    while (__any_sync(FULL, nzm != 0u)) {
      const bool has = nzm != 0u;
      int j = 0;
      int change = 0;
      uint32_t key = 0u;
      if (has) {
        j = __ffs(nzm) - 1;
        nzm &= nzm - 1;
        int v = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) v |= (int)((D[b] >> j) & 1u) << b;
        change = (int)(signed char)v;
        // the voxel's value (x0 + j >= 0: own bits are 1..30)
        const unsigned char* vp = rowz + (size_t)(x0 + j) * EB;
        if constexpr (EB == 4)
          key = value_key(__ldg(reinterpret_cast<const float*>(vp)));
        else if constexpr (EB == 2)
          key = __ldg(reinterpret_cast<const unsigned short*>(vp));
        else
          key = __ldg(vp);
      }
      if constexpr (MODE == k4Pairs) {
        // into the warp's buffer (every lane with a voxel has a non-zero change)
        const unsigned ballot = __ballot_sync(FULL, has);
        const int n = __popc(ballot);
        if (pfill + n > k4PairBuf) flush_pairs();
        if (has)
          pbuf[pfill + __popc(ballot & ((1u << lane) - 1u))] =
              ((unsigned long long)key << 32) | (uint32_t)change;
        __syncwarp();
        pfill += n;
      } else if (has && change != 0) {
        const uint32_t v = key & ((1u << (NB < 32 ? NB : 31)) - 1u);
        if (MODE == k4Smem)
          atomicAdd(&hist[v], change);
        else
          atomicAdd(reinterpret_cast<unsigned long long*>(im.vcec) + v,
                    (unsigned long long)(long long)change);
      }
    }
    __syncthreads();
  }
  if constexpr (MODE == k4Pairs) flush_pairs();
}

}  // namespace ecc
