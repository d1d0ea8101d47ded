// Bit-sliced contribution code for 1-3D integer images, shared by the
// single-image kernel (k_bits.cu) and the batched persistent kernel
// (batch.cu).
//
// Same quantity as the generic kernel (Algorithm 1 of Sec. 3: per voxel, the
// signed count of the faces it introduces, added to the VCEC at its gray
// value), computed 32 voxels at a time:
//
// * A lane holds 32 consecutive voxels of one row as bit planes: plane k bit j
//   = bit k of voxel x0 + j.
// * "N >= C" for 32 voxel pairs is a borrow chain over the planes, one
//   three-input logic op per plane. Voxels outside the image count as +inf
//   (the infinite collar of the paper's Sec. 4): per-row and x-edge masks
//   override the comparison in the same final logic op.
// * Each unordered neighbour pair is compared once: for the 13 neighbour
//   offsets d that come later in the linear order, G_d[i] = [f(N_i) >= f(C_{i-dx})]
//   is indexed by the later voxel. The earlier voxel reads its "neighbour
//   after me" bit as G_d shifted by dx; the later voxel reads NOT G_d
//   ("after" is strict in that direction: ties go to the larger index).
// * With the 26 after-bits M, change_V = -G_3(M) and change_T = G_3(~M),
//   G_3 = 1 - sum(face bits) + sum(edge triples) - sum(vertex 7-boxes). Both are
//   N - 13 with N = popcount of 26 terms (faces; complemented or plain edge
//   triples; plain or complemented vertex boxes), evaluated by a carry-save
//   adder tree on whole words.
//
// Layout: a row group of L lanes covers a whole row (L = the power of two
// >= nx / 32), or, for rows wider than 1024, a warp covers 1024 voxels of
// which the middle 960 are its own (lanes 0 and 31 supply the x-collar). A
// block holds consecutive rows (the first and the last row are the y-collar,
// both in its first warp) and marches along z over a span of planes.
// y-neighbour planes and the exported comparison words go through shared
// memory, x-neighbour bits through warp shuffles.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ecc_internal.h"

namespace ecc {

struct BitsGeo {
  int L;       // lanes per row group (power of two)
  int R;       // row groups per warp (32 / L)
  int RB;      // rows per block, including the two collar rows
  int modeB;   // 1: warps overlap in x by one lane on each side
  int64_t tiles_x, tiles_y, tiles_z, n_tiles, zc;
};

struct BitsImg {
  const unsigned char* img;  // plane w_mem_lo of the image
  int64_t n[3];              // z, y, x
  int64_t row_pitch;         // bytes between rows (rows may start at any byte)
  int64_t w_lo, w_hi;        // planes processed
  int64_t w_mem_lo, w_mem_hi;  // planes resident at img
  int64_t bins;
  long long* vcec;
  int* err;
  long long* curve;    // non-null: the last block writes the curve, zeroes vcec and *done
  unsigned int* done;  // blocks finished (starts at 0)
};

enum BitsHist : int { kBitsSmem = 0, kBitsGlobal = 1 };
constexpr int kBitsG0Rec = 3, kBitsG1Rec = 7;

// Geometry for an image (z-range of wn planes) with W warps per block.
inline BitsGeo bits_geo(int64_t nx, int64_t ny, int64_t wn, int W, int64_t zc) {
  BitsGeo g{};
  const int64_t segs = (nx + 31) / 32;
  if (segs <= 32) {
    int L = 1;
    while (L < segs) L <<= 1;
    g.L = L;
    g.R = 32 / L;
    g.modeB = 0;
    g.tiles_x = 1;
  } else {
    g.L = 32;
    g.R = 1;
    g.modeB = 1;
    g.tiles_x = (nx + 959) / 960;
  }
  g.RB = W * g.R;
  g.tiles_y = (ny + (g.RB - 2) - 1) / (g.RB - 2);
  g.zc = zc > 0 ? zc : std::max<int64_t>(wn, 1);
  g.tiles_z = (wn + g.zc - 1) / g.zc;
  g.n_tiles = g.tiles_x * g.tiles_y * g.tiles_z;
  return g;
}

namespace bits {

__device__ __forceinline__ void fa(uint32_t a, uint32_t b, uint32_t c, uint32_t& s, uint32_t& co) {
  s = a ^ b ^ c;
  co = (a & b) | (c & (a ^ b));
}
__device__ __forceinline__ void ha(uint32_t a, uint32_t b, uint32_t& s, uint32_t& co) {
  s = a ^ b;
  co = a & b;
}

// Bytes -> bit planes. u[j] holds bytes 4j..4j+3 (voxel order); afterwards
// p[k] bit v = bit k of byte v, v = 0..31.
__device__ __forceinline__ void transpose8(const uint32_t u[8], uint32_t p[8]) {
  uint32_t t[8];
  {
    // two 4x4 byte transposes: t[i] holds bytes i, i+8, i+16, i+24 (i < 8)
    const uint32_t a = __byte_perm(u[0], u[2], 0x5140), b = __byte_perm(u[0], u[2], 0x7362);
    const uint32_t c = __byte_perm(u[4], u[6], 0x5140), d = __byte_perm(u[4], u[6], 0x7362);
    t[0] = __byte_perm(a, c, 0x5410);
    t[1] = __byte_perm(a, c, 0x7632);
    t[2] = __byte_perm(b, d, 0x5410);
    t[3] = __byte_perm(b, d, 0x7632);
    const uint32_t e = __byte_perm(u[1], u[3], 0x5140), f = __byte_perm(u[1], u[3], 0x7362);
    const uint32_t g = __byte_perm(u[5], u[7], 0x5140), h = __byte_perm(u[5], u[7], 0x7362);
    t[4] = __byte_perm(e, g, 0x5410);
    t[5] = __byte_perm(e, g, 0x7632);
    t[6] = __byte_perm(f, h, 0x5410);
    t[7] = __byte_perm(f, h, 0x7632);
  }
  // three delta swaps: register index bit s <-> bit s of the position in a byte
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int s = 1 << st;
    const uint32_t M = st == 0 ? 0x55555555u : st == 1 ? 0x33333333u : 0x0F0F0F0Fu;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (r & s) continue;
      const uint32_t a = t[r], b = t[r | s];
      t[r] = (a & M) | ((b << s) & ~M);
      t[r | s] = ((a >> s) & M) | (b & ~M);
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] = t[k];
}

// Bit planes -> bytes, the inverse of transpose8: the three swaps (each an
// involution, and they commute) and then the byte transposes (involutions).
__device__ __forceinline__ void untranspose8(const uint32_t p[8], uint32_t u[8]) {
  uint32_t t[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) t[k] = p[k];
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int s = 1 << st;
    const uint32_t M = st == 0 ? 0x55555555u : st == 1 ? 0x33333333u : 0x0F0F0F0Fu;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (r & s) continue;
      const uint32_t a = t[r], b = t[r | s];
      t[r] = (a & M) | ((b << s) & ~M);
      t[r | s] = ((a >> s) & M) | (b & ~M);
    }
  }
  {
    const uint32_t a = __byte_perm(t[0], t[1], 0x5140), b = __byte_perm(t[0], t[1], 0x7362);
    const uint32_t c = __byte_perm(t[2], t[3], 0x5140), d = __byte_perm(t[2], t[3], 0x7362);
    u[0] = __byte_perm(a, c, 0x5410);
    u[2] = __byte_perm(a, c, 0x7632);
    u[4] = __byte_perm(b, d, 0x5410);
    u[6] = __byte_perm(b, d, 0x7632);
    const uint32_t e = __byte_perm(t[4], t[5], 0x5140), f = __byte_perm(t[4], t[5], 0x7362);
    const uint32_t g = __byte_perm(t[6], t[7], 0x5140), h = __byte_perm(t[6], t[7], 0x7362);
    u[1] = __byte_perm(e, g, 0x5410);
    u[3] = __byte_perm(e, g, 0x7632);
    u[5] = __byte_perm(f, h, 0x5410);
    u[7] = __byte_perm(f, h, 0x7632);
  }
}

// Borrow out of N - C on 32 voxel pairs (planes LSB first): 1 where N < C.
template <int NB>
__device__ __forceinline__ uint32_t borrow(const uint32_t* N, const uint32_t* C) {
  uint32_t b = C[0] & ~N[0];
#pragma unroll
  for (int k = 1; k < NB; ++k) {
    const uint32_t n = ~N[k], c = C[k];
    b = (n & c) | (n & b) | (c & b);
  }
  return b;
}

// [N >= C] with voxels outside the image as +inf: 1 where N is outside
// (nout), else 0 where C is outside (cout), else no borrow. One logic op.
__device__ __forceinline__ uint32_t gcmp(uint32_t b, uint32_t cout, uint32_t nout) {
  return (~b & ~cout) | nout;
}

}  // namespace bits

// The deposit of a word with many non-zero changes (noisy data): per-voxel N
// as bytes by the inverse transpose, the row's raw values re-read (an L2
// hit) from rp (the word's first voxel; left0 voxels of the row from there),
// and an unrolled deposit with constant byte offsets. Out of line, so that
// the common path of smooth data keeps its code small.
template <int NB, int EB, int HM>
__device__ __noinline__ void deposit_dense(uint32_t n0, uint32_t n1, uint32_t n2, uint32_t n3,
                                           uint32_t n4, uint32_t nzm, const unsigned char* rp,
                                           int64_t left0, int* hist, long long* vcec) {
  constexpr int RAW = 8 * EB;
  const uint32_t pn[8] = {n0, n1, n2, n3, n4, 0u, 0u, 0u};
  uint32_t nbyte[8];
  bits::untranspose8(pn, nbyte);
  // two halves of 16 voxels keep fewer raw words live
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    uint32_t rz[RAW / 2];
    const uintptr_t pa = reinterpret_cast<uintptr_t>(rp) + (uintptr_t)(hf * 16 * EB);
    const uint32_t* q = reinterpret_cast<const uint32_t*>(pa & ~uintptr_t(3));
    const uint32_t sh8 = (uint32_t)(pa & 3u) * 8u;
    uint32_t w[RAW / 2 + 1];
    const int64_t left = left0 - hf * 16;
    const int64_t bytes = (left >= 16 ? 16 : (left > 0 ? left : 0)) * EB + (int64_t)(pa & 3u);
#pragma unroll
    for (int i = 0; i <= RAW / 2; ++i) w[i] = 4 * i < bytes ? __ldg(q + i) : 0u;
#pragma unroll
    for (int i = 0; i < RAW / 2; ++i) rz[i] = __funnelshift_r(w[i], w[i + 1], sh8);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int j = hf * 16 + jj;
      if ((nzm >> j) & 1u) {
        const int N = (int)((nbyte[j >> 2] >> ((j & 3) * 8)) & 31u);
        uint32_t v = EB == 1 ? (rz[jj >> 2] >> ((jj & 3) * 8)) & 0xFFu
                             : (rz[jj >> 1] >> ((jj & 1) * 16)) & 0xFFFFu;
        v &= (1u << NB) - 1u;
        if (HM == kBitsSmem)
          atomicAdd(&hist[v], N - 13);
        else
          atomicAdd(reinterpret_cast<unsigned long long*>(vcec) + v,
                    (unsigned long long)(long long)(N - 13));
      }
    }
  }
}

// Planes [z0, z1) of the row column (tx, ty) of geometry geo, one image. All
// threads of the block call it; blockDim.x = 32 * (geo.RB / geo.R). pl/g0/g1
// are the shared exchange arrays (record strides pl_rec (odd, >= NB + 1), 3,
// 7), hist the shared histogram (kBitsSmem).
template <int NB, int CONV, int HM>
__device__ void bits_span(const BitsImg& im, const BitsGeo& geo, int64_t tx, int64_t ty,
                          int64_t z0, int64_t z1, uint32_t* pl, uint32_t* g0, uint32_t* g1,
                          int pl_rec, int* hist) {
  using namespace bits;
  constexpr int NP = NB;                // value planes
  constexpr int EB = NB <= 8 ? 1 : 2;   // bytes per voxel
  constexpr int RAW = 8 * EB;           // raw 32-bit words per lane and row
  const int L = geo.L, RB = geo.RB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / L, l = lane - grp * L;
  // row within the block, 0..RB-1: the two collar rows (0 and RB-1) share the
  // first warp (row groups 0 and 1), so the other warps hold own rows only
  // and the collar warp skips what collar rows do not need
  const int slot = warp * geo.R + grp;
  const int br = slot == 0 ? 0 : slot == 1 ? RB - 1 : slot - 1;
  const int my = br * L + l;
  const int up = (br + 1 < RB ? br + 1 : br) * L + l;  // clamped neighbour rows
  const int dn = (br > 0 ? br - 1 : br) * L + l;
  const int64_t nz = im.n[0], ny = im.n[1], nx = im.n[2];
  const size_t row_bytes = (size_t)im.row_pitch;
  const unsigned FULL = 0xFFFFFFFFu;

  const int64_t y = ty * (RB - 2) - 1 + br;
  const int64_t x0 = (geo.modeB ? tx * 960 - 32 : 0) + 32 * (int64_t)l;
  const bool row_in = y >= 0 && y < ny;
  uint32_t xin = 0;  // bits whose x lies inside the image
  if (x0 < nx && x0 + 32 > 0) {
    const int64_t lo = x0 < 0 ? -x0 : 0, hi = nx - x0 >= 32 ? 32 : nx - x0;
    xin = (hi >= 32 ? FULL : ((1u << hi) - 1u)) & (FULL << lo);
  }
  const bool own_lane = (geo.modeB ? (l >= 1 && l <= 30) : true) && x0 >= 0 && x0 < nx;
  const bool own_row = br >= 1 && br <= RB - 2 && row_in;
  const uint32_t dep = (own_lane && own_row) ? xin : 0u;
  const bool aligned16 =
      ((reinterpret_cast<uintptr_t>(im.img) | (uintptr_t)row_bytes) & 15u) == 0;
  const uint32_t edgeL = x0 == 0 ? 1u : 0u;
  const uint32_t edgeR = x0 + 32 >= nx ? 0x80000000u : 0u;

  // outside masks: xo = bits outside the image in x; cx[dx+1] = outside bits
  // of the centre row shifted by dx (C'[i] = C[i - dx])
  const uint32_t xo = ~xin;
  const uint32_t cx[3] = {(xo >> 1) | edgeR, xo, (xo << 1) | edgeL};
  const int64_t yup = y + 1, ydn = y - 1;
  const bool up_in = yup >= 0 && yup < ny, dn_in = ydn >= 0 && ydn < ny;

  // raw words of plane zp for this lane's 32 voxels (unchanged where not
  // loaded: those voxels are outside and masked)
  auto load_raw = [&](int64_t zp, uint32_t* raw) {
    if (!row_in || zp < 0 || zp >= nz || x0 < 0 || x0 >= nx) return;
    if (zp < im.w_mem_lo || zp >= im.w_mem_hi) {
      atomicOr(im.err, kErrOverflow);
      return;
    }
    const unsigned char* p =
        im.img + ((size_t)(zp - im.w_mem_lo) * ny + (size_t)y) * row_bytes + (size_t)x0 * EB;
    if (aligned16) {
#pragma unroll
      for (int c = 0; c < RAW / 4; ++c) {
        if (x0 + c * (16 / EB) < nx) {
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + c);
          raw[4 * c] = v.x;
          raw[4 * c + 1] = v.y;
          raw[4 * c + 2] = v.z;
          raw[4 * c + 3] = v.w;
        }
      }
    } else {
      // rows at any byte alignment: aligned 4-byte words, funnel-shifted;
      // only words holding at least one byte of this row's voxels are read
      const uintptr_t pa = reinterpret_cast<uintptr_t>(p);
      const uint32_t* q = reinterpret_cast<const uint32_t*>(pa & ~uintptr_t(3));
      const uint32_t sh = (uint32_t)(pa & 3u) * 8u;
      const int64_t bytes = (nx - x0 >= 32 ? 32 : nx - x0) * EB + (int64_t)(pa & 3u);
      uint32_t w[RAW + 1];
#pragma unroll
      for (int j = 0; j <= RAW; ++j) w[j] = 4 * j < bytes ? __ldg(q + j) : 0u;
#pragma unroll
      for (int i = 0; i < RAW; ++i) raw[i] = __funnelshift_r(w[i], w[i + 1], sh);
    }
  };
  // planes of the lane's row at plane zp from its raw words
  auto make_planes = [&](int64_t zp, const uint32_t* raw, uint32_t* P) {
    const uint32_t inside = (row_in && zp >= 0 && zp < nz) ? xin : 0u;
    if (EB == 1) {
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
    (void)inside;
  };

  uint32_t raw[RAW] = {};
  uint32_t Pz[NP], Ryp[NP], Pn[NP], Pup[NP], Pdn[NP];
  uint32_t Gp[3] = {0u, 0u, 0u};  // own G_(1,0,dx) of the previous step

  // prologue: the own row and the row above at the first plane zs. A tile at
  // z0 = 0 has no plane below: its "previous step" exports are zero (the
  // plane below is outside, every neighbour there comes after), so it starts
  // at zs = z0; otherwise one priming step at z0 - 1 computes them.
  const int64_t zs = z0 == 0 ? z0 : z0 - 1;
  if (z0 == 0) {
    uint32_t* g1z = g1 + (int)((z0 - 1) & 1) * RB * L * kBitsG1Rec;
#pragma unroll
    for (int i = 0; i < 6; ++i) g1z[my * kBitsG1Rec + i] = 0u;
  }
  load_raw(zs, raw);
  make_planes(zs, raw, Pz);
#pragma unroll
  for (int k = 0; k < NP; ++k) pl[my * pl_rec + k] = Pz[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NP; ++k) Ryp[k] = pl[up * pl_rec + k];
  load_raw(zs + 1, raw);
  __syncthreads();

  for (int64_t z = zs; z < z1; ++z) {
    // planes of z + 1 (prefetched one step ago); prefetch z + 2
    make_planes(z + 1, raw, Pn);
    if (z + 2 <= z1) load_raw(z + 2, raw);
    // exchange the planes of z + 1; read the previous step's exports
#pragma unroll
    for (int k = 0; k < NP; ++k) pl[my * pl_rec + k] = Pn[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      Pup[k] = pl[up * pl_rec + k];
      Pdn[k] = pl[dn * pl_rec + k];
    }
    const uint32_t* g1p = g1 + (int)((z - 1) & 1) * RB * L * kBitsG1Rec;
    uint32_t Gdn1[3], Gup1[3];  // prev G_(1,+1,.) of row br-1, G_(1,-1,.) of row br+1
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Gdn1[i] = g1p[dn * kBitsG1Rec + i];
      Gup1[i] = g1p[up * kBitsG1Rec + 3 + i];
    }
    // centre row shifted for dx = +1 (C[i-1]) and dx = -1 (C[i+1]). Full-warp
    // shuffles: a lane at a row-group boundary is at an image x-edge, where
    // the shifted-in bit is masked as outside (cx, edgeL/edgeR).
    uint32_t Cl[NP], Cr[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const uint32_t left = __shfl_up_sync(FULL, Pz[k], 1);
      const uint32_t right = __shfl_down_sync(FULL, Pz[k], 1);
      Cl[k] = __funnelshift_l(left, Pz[k], 1);
      Cr[k] = __funnelshift_r(Pz[k], right, 1);
    }
    // outside masks of this step's rows
    const bool z_in = z >= 0 && z < nz, z1_in = z + 1 < nz;
    const uint32_t ALL = 0xFFFFFFFFu;
    const bool c_in = row_in && z_in;
    const uint32_t co[3] = {c_in ? cx[0] : ALL, c_in ? cx[1] : ALL, c_in ? cx[2] : ALL};
    const uint32_t no_z = c_in ? xo : ALL;                  // own row at z
    const uint32_t no_yp = (up_in && z_in) ? xo : ALL;      // row y+1 at z
    const uint32_t no1[3] = {(dn_in && z1_in) ? xo : ALL, (row_in && z1_in) ? xo : ALL,
                             (up_in && z1_in) ? xo : ALL};  // rows y-1..y+1 at z+1
    // the 13 forward comparisons, indexed by the later voxel
    const uint32_t G001 = gcmp(borrow<NB>(Pz, Cl), co[2], no_z);
    uint32_t G01[3], G1[3][3];  // [dx+1], [dy+1][dx+1]
    G01[0] = gcmp(borrow<NB>(Ryp, Cr), co[0], no_yp);
    G01[1] = gcmp(borrow<NB>(Ryp, Pz), co[1], no_yp);
    G01[2] = gcmp(borrow<NB>(Ryp, Cl), co[2], no_yp);
    G1[0][0] = gcmp(borrow<NB>(Pdn, Cr), co[0], no1[0]);
    G1[0][1] = gcmp(borrow<NB>(Pdn, Pz), co[1], no1[0]);
    G1[0][2] = gcmp(borrow<NB>(Pdn, Cl), co[2], no1[0]);
    G1[1][0] = gcmp(borrow<NB>(Pn, Cr), co[0], no1[1]);
    G1[1][1] = gcmp(borrow<NB>(Pn, Pz), co[1], no1[1]);
    G1[1][2] = gcmp(borrow<NB>(Pn, Cl), co[2], no1[1]);
    G1[2][0] = gcmp(borrow<NB>(Pup, Cr), co[0], no1[2]);
    G1[2][1] = gcmp(borrow<NB>(Pup, Pz), co[1], no1[2]);
    G1[2][2] = gcmp(borrow<NB>(Pup, Cl), co[2], no1[2]);
    // exports
    uint32_t* g1w = g1 + (int)(z & 1) * RB * L * kBitsG1Rec;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g0[my * kBitsG0Rec + i] = G01[i];
      g1w[my * kBitsG1Rec + i] = G1[2][i];
      g1w[my * kBitsG1Rec + 3 + i] = G1[0][i];
    }
    __syncthreads();
    // the change evaluation, where a lane of the warp deposits (never in the
    // collar warp or on a priming plane); warp-uniform, so the shuffles in it
    // see the whole warp
    if (__any_sync(FULL, z >= z0 && dep != 0u)) {
    uint32_t G01dn[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) G01dn[i] = g0[dn * kBitsG0Rec + i];

    // forward after-bits are G shifted by dx (x-neighbour bit by shuffle)
    auto sh = [&](uint32_t g, int dx) -> uint32_t {
      if (dx == 1) {
        const uint32_t r = __shfl_down_sync(FULL, g, 1);
        return __funnelshift_r(g, r, 1) | edgeR;
      }
      if (dx == -1) {
        const uint32_t q = __shfl_up_sync(FULL, g, 1);
        return __funnelshift_l(q, g, 1) | edgeL;
      }
      return g;
    };
    // after-bits of the 26 neighbours: x+-1; (0,+-1,dx); (+-1,dy,dx)
    const uint32_t xp = sh(G001, 1), xm = ~G001;
    uint32_t a0p[3], a0m[3], ap[3][3], am[3][3];
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      a0p[dx + 1] = sh(G01[dx + 1], dx);
      a0m[dx + 1] = ~G01dn[1 - dx];
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) ap[dy + 1][dx + 1] = sh(G1[dy + 1][dx + 1], dx);
      am[1][dx + 1] = ~Gp[1 - dx];
      am[0][dx + 1] = ~Gdn1[1 - dx];  // neighbour (-1,-1,dx): delta (1,+1,-dx) of row br-1
      am[2][dx + 1] = ~Gup1[1 - dx];  // neighbour (-1,+1,dx): delta (1,-1,-dx) of row br+1
    }

    if (z >= z0 && dep) {
      // b(dz, dy, dx): after-bits (V) or their complement (T)
      auto b = [&](int dz, int dy, int dx) -> uint32_t {
        uint32_t v;
        if (dz == 0) {
          if (dy == 0) v = dx > 0 ? xp : xm;
          else v = dy > 0 ? a0p[dx + 1] : a0m[dx + 1];
        } else {
          v = dz > 0 ? ap[dy + 1][dx + 1] : am[dy + 1][dx + 1];
        }
        return CONV == kConvV ? v : ~v;
      };
      uint32_t tm[26];
      int n = 0;
      tm[n++] = xp; tm[n++] = xm; tm[n++] = a0p[1]; tm[n++] = a0m[1];
      tm[n++] = ap[1][1]; tm[n++] = am[1][1];
      uint32_t Exy[2][2];
#pragma unroll
      for (int sx = 0; sx < 2; ++sx)
#pragma unroll
        for (int sy = 0; sy < 2; ++sy) {
          const int dx = sx ? 1 : -1, dy = sy ? 1 : -1;
          Exy[sx][sy] = b(0, 0, dx) & b(0, dy, 0) & b(0, dy, dx);
          tm[n++] = CONV == kConvV ? ~Exy[sx][sy] : Exy[sx][sy];
        }
#pragma unroll
      for (int sx = 0; sx < 2; ++sx)
#pragma unroll
        for (int sz = 0; sz < 2; ++sz) {
          const int dx = sx ? 1 : -1, dz = sz ? 1 : -1;
          const uint32_t e = b(0, 0, dx) & b(dz, 0, 0) & b(dz, 0, dx);
          tm[n++] = CONV == kConvV ? ~e : e;
        }
#pragma unroll
      for (int sy = 0; sy < 2; ++sy)
#pragma unroll
        for (int sz = 0; sz < 2; ++sz) {
          const int dy = sy ? 1 : -1, dz = sz ? 1 : -1;
          const uint32_t e = b(0, dy, 0) & b(dz, 0, 0) & b(dz, dy, 0);
          tm[n++] = CONV == kConvV ? ~e : e;
        }
#pragma unroll
      for (int sx = 0; sx < 2; ++sx)
#pragma unroll
        for (int sy = 0; sy < 2; ++sy)
#pragma unroll
          for (int sz = 0; sz < 2; ++sz) {
            const int dx = sx ? 1 : -1, dy = sy ? 1 : -1, dz = sz ? 1 : -1;
            const uint32_t v7 =
                Exy[sx][sy] & b(dz, 0, 0) & b(dz, 0, dx) & b(dz, dy, 0) & b(dz, dy, dx);
            tm[n++] = CONV == kConvV ? v7 : ~v7;
          }
      // popcount of the 26 terms, bit-sliced: n0..n4
      uint32_t s[8], c[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) fa(tm[3 * i], tm[3 * i + 1], tm[3 * i + 2], s[i], c[i]);
      uint32_t a0, a1, a2, d0, d1, d2, b0, e0, n0, e1;
      fa(s[0], s[1], s[2], a0, d0);
      fa(s[3], s[4], s[5], a1, d1);
      fa(s[6], s[7], tm[24], a2, d2);
      fa(a0, a1, a2, b0, e0);
      ha(b0, tm[25], n0, e1);
      uint32_t f0, f1, f2, f3, q0, q1, q2, q3, h0, i0, n1, i1;
      fa(c[0], c[1], c[2], f0, q0);
      fa(c[3], c[4], c[5], f1, q1);
      fa(c[6], c[7], d0, f2, q2);
      fa(d1, d2, e0, f3, q3);
      fa(f0, f1, f2, h0, i0);
      fa(f3, e1, h0, n1, i1);
      uint32_t j0, k0, j1, k1, n2, k2, n3, n4;
      fa(q0, q1, q2, j0, k0);
      fa(q3, i0, i1, j1, k1);
      ha(j0, j1, n2, k2);
      fa(k0, k1, k2, n3, n4);
      // change = N - 13; zero iff N == 0b01101
      const uint32_t eq13 = ~n4 & n3 & n2 & ~n1 & n0;
      uint32_t nzm = ~eq13 & dep;
      // bins = 2^NB here; a value with bits above NB has already set the
      // value error (make_planes), so masking only keeps its (discarded)
      // deposit inside the histogram
      auto deposit = [&](uint32_t v, int c) {
        v &= (1u << NB) - 1u;
        if (HM == kBitsSmem) {
          atomicAdd(&hist[v], c);
        } else {
          atomicAdd(reinterpret_cast<unsigned long long*>(im.vcec) + v,
                    (unsigned long long)(long long)c);
        }
      };
      if (__popc(nzm) >= 8) {
        // many non-zero changes (noisy data): the unrolled deposit, out of line
        const unsigned char* rp = im.img + ((size_t)(z - im.w_mem_lo) * ny + (size_t)y) * row_bytes +
                                  (size_t)x0 * EB;
        deposit_dense<NB, EB, HM>(n0, n1, n2, n3, n4, nzm, rp, nx - x0, hist, im.vcec);
        nzm = 0;
      }
      while (nzm) {
        const int j = __ffs(nzm) - 1;
        nzm &= nzm - 1;
        const int N = (int)(((n0 >> j) & 1u) | (((n1 >> j) & 1u) << 1) | (((n2 >> j) & 1u) << 2) |
                            (((n3 >> j) & 1u) << 3) | (((n4 >> j) & 1u) << 4));
        // its gray value: the row was read from global memory two steps ago
        const unsigned char* vp = im.img +
            ((size_t)(z - im.w_mem_lo) * ny + (size_t)y) * row_bytes + (size_t)(x0 + j) * EB;
        const uint32_t v = EB == 1 ? (uint32_t)__ldg(vp)
                                   : (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(vp));
        deposit(v, N - 13);
      }
    }
    }  // any lane deposits
#pragma unroll
    for (int i = 0; i < 3; ++i) Gp[i] = G1[1][i];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      Pz[k] = Pn[k];
      Ryp[k] = Pup[k];
    }
  }
  __syncthreads();
}

// Tile t of geometry geo: row column t mod (tiles_x * tiles_y), planes
// [w_lo + tz * zc, + zc) with tz = t / (tiles_x * tiles_y).
template <int NB, int CONV, int HM>
__device__ __forceinline__ void bits_tile(const BitsImg& im, const BitsGeo& geo, int64_t t,
                                          uint32_t* pl, uint32_t* g0, uint32_t* g1, int pl_rec,
                                          int* hist) {
  const int64_t txy = geo.tiles_x * geo.tiles_y;
  const int64_t tz = t / txy, rem = t - tz * txy;
  const int64_t ty = rem / geo.tiles_x, tx = rem - ty * geo.tiles_x;
  const int64_t z0 = im.w_lo + tz * geo.zc, z1 = min(z0 + geo.zc, im.w_hi);
  bits_span<NB, CONV, HM>(im, geo, tx, ty, z0, z1, pl, g0, g1, pl_rec, hist);
}

}  // namespace ecc
