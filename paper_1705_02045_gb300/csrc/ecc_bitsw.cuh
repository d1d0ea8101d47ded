// Warp-column layout of the bit-sliced contribution kernel for 1-3D integer
// images (single-image launches, k_bits.cu).
//
// The quantity and the per-word arithmetic are those of ecc_bits.cuh
// (Algorithm 1 of Sec. 3: per voxel the signed count of the faces it
// introduces, added to the VCEC at its gray value; 32 voxels per lane as bit
// planes, each unordered neighbour pair compared once by a borrow chain, the
// change as N - 13 from a carry-save count of 26 terms). What differs is who
// holds which voxels:
//
// * A warp owns a column of 32 consecutive rows (one lane per row) of one
//   32-voxel word each, marching along z. Lanes 0 and 31 hold the rows below
//   and above the warp's 30 own rows, and bits 0 and 31 of every word the
//   voxels left and right of its 30 own voxels (the one-voxel collar of
//   Sec. 3, "Processing one Chunk", in y and x). Tiles step by 30 in x and y.
// * Every exchange between neighbouring rows is a warp shuffle, every x
//   neighbour an in-word shift, and the previous plane's comparison words stay
//   in the lane's registers: there is no shared-memory exchange and no block
//   barrier in the z-march. Warps of a block share only the shared-memory
//   histogram.
// * Collar bits and lanes compute garbage in the positions that their own
//   missing neighbours would feed; no own voxel (bits 1..30 of lanes 1..30)
//   reads such a position.
//
// Voxels outside the image count as +inf (the infinite collar of Sec. 4), by
// the same outside masks as the row-group layout.
#pragma once

#include "ecc_bits.cuh"

namespace ecc {

constexpr int kWcOwn = 30;  // own rows per warp and own voxels per word

struct WcGeo {
  int64_t tiles_x, tiles_y, cols;
};

inline WcGeo wc_geo(int64_t nx, int64_t ny) {
  WcGeo g{};
  g.tiles_x = (nx + kWcOwn - 1) / kWcOwn;
  g.tiles_y = (ny + kWcOwn - 1) / kWcOwn;
  g.cols = g.tiles_x * g.tiles_y;
  return g;
}

namespace wc {

// Words [0, RAW) of the 32-voxel window starting at voxel x0 (may be -1) of
// a row: word i holds bytes 4i..4i+3 of the window. Only memory holding at
// least one byte of the row's voxels [max(x0, 0), min(x0 + 32, nx)) is read;
// the rest of the window reads as zero. fast: the row starts on a 16-byte
// boundary (16-byte loads, the in-chunk offset the same for every lane of the
// warp); otherwise aligned 4-byte words.
template <int EB>
__device__ __forceinline__ void load_window(const unsigned char* row, int64_t x0, int64_t nx,
                                            bool fast, uint32_t* raw) {
  constexpr int RAW = 8 * EB;
  const int64_t vb0 = (x0 < 0 ? 0 : x0) * EB;
  const int64_t vb1 = (x0 + 32 < nx ? x0 + 32 : nx) * EB;
  const int64_t s = x0 * EB;
  if (fast) {
    const int64_t a = s & ~int64_t(15);
    const int o = (int)(s - a);
    uint32_t w[RAW + 4];
#pragma unroll
    for (int c = 0; c <= RAW / 4; ++c) {
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
    const uint32_t sh = 8u * (uint32_t)(o & 3);
    // o >> 2 is the same in every lane: one of four unrolled extractions
    switch (o >> 2) {
#define ECC_WC_EXTRACT(q)                                                              \
  case q:                                                                              \
    _Pragma("unroll") for (int i = 0; i < RAW; ++i) raw[i] =                           \
        __funnelshift_r(w[i + q], w[i + q + 1], sh);                                   \
    break;
      ECC_WC_EXTRACT(0)
      ECC_WC_EXTRACT(1)
      ECC_WC_EXTRACT(2)
      ECC_WC_EXTRACT(3)
#undef ECC_WC_EXTRACT
    }
  } else {
    const uintptr_t pa = reinterpret_cast<uintptr_t>(row) + (uintptr_t)s;
    const uintptr_t qa = pa & ~uintptr_t(3);
    const uint32_t sh = 8u * (uint32_t)(pa & 3u);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(row) + (uintptr_t)vb0;
    const uintptr_t hi = reinterpret_cast<uintptr_t>(row) + (uintptr_t)vb1;
    uint32_t w[RAW + 1];
#pragma unroll
    for (int j = 0; j <= RAW; ++j) {
      const uintptr_t wa = qa + 4 * (uintptr_t)j;
      w[j] = (wa + 4 > lo && wa < hi) ? __ldg(reinterpret_cast<const uint32_t*>(wa)) : 0u;
    }
#pragma unroll
    for (int i = 0; i < RAW; ++i) raw[i] = __funnelshift_r(w[i], w[i + 1], sh);
  }
}

}  // namespace wc

// Planes [z0, z1) of the warp column (tx, ty). Called by all 32 lanes of a
// warp (other warps of the block are independent). hist: the block's shared
// histogram (kBitsSmem). fast: rows start on 16-byte boundaries.
template <int NB, int CONV, int HM>
__device__ void bitsw_span(const BitsImg& im, int64_t tx, int64_t ty, int64_t z0, int64_t z1,
                           bool fast, int* hist) {
  using namespace bits;
  constexpr int NP = NB;
  constexpr int EB = NB <= 8 ? 1 : 2;
  constexpr int RAW = 8 * EB;
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xFFFFFFFFu;
  const int64_t nz = im.n[0], ny = im.n[1], nx = im.n[2];
  const size_t pitch = (size_t)im.row_pitch;

  const int64_t y = ty * kWcOwn - 1 + lane;
  const int64_t x0 = tx * kWcOwn - 1;  // < nx - 1: the tile holds an own voxel
  const bool row_in = y >= 0 && y < ny;
  uint32_t xin;  // bits whose x lies inside the image
  {
    const int64_t lo = x0 < 0 ? -x0 : 0, hi = nx - x0 >= 32 ? 32 : nx - x0;
    xin = (hi >= 32 ? FULL : ((1u << hi) - 1u)) & (FULL << lo);
  }
  const bool own_lane = lane >= 1 && lane <= kWcOwn;
  const uint32_t dep = (own_lane && row_in) ? (xin & 0x7FFFFFFEu) : 0u;
  // outside masks: xo = bits outside in x; cx[dx+1] = outside bits of the
  // centre row shifted by dx (C'[i] = C[i - dx]); the bit shifted in at the
  // word's end only feeds collar positions
  const uint32_t xo = ~xin;
  const uint32_t cx[3] = {xo >> 1, xo, xo << 1};
  const bool up_in = y + 1 >= 0 && y + 1 < ny, dn_in = y - 1 >= 0 && y - 1 < ny;

  auto row_ptr = [&](int64_t zp) {
    return im.img + ((size_t)(zp - im.w_mem_lo) * (size_t)ny + (size_t)y) * pitch;
  };
  // raw words of plane zp for this lane's 32 voxels (unchanged where not
  // loaded: those voxels are outside and masked)
  auto load_raw = [&](int64_t zp, uint32_t* raw) {
    if (!row_in || zp < 0 || zp >= nz) return;
    if (zp < im.w_mem_lo || zp >= im.w_mem_hi) {
      atomicOr(im.err, kErrOverflow);
      return;
    }
    wc::load_window<EB>(row_ptr(zp), x0, nx, fast, raw);
  };
  auto make_planes = [&](int64_t zp, const uint32_t* raw, uint32_t* P) {
    if (EB == 1) {
      transpose8(raw, P);
    } else {
      const uint32_t inside = (row_in && zp >= 0 && zp < nz) ? xin : 0u;
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

  // One step of the z-march at plane z: Pz / Ryp hold the own row and row
  // y + 1 at z, Gp this lane's comparison words G_(1,dy,dx) of the previous
  // step ([dy+1][dx+1]); the step fills Pn / Pup (own row and row y + 1 at
  // z + 1) and G1 (this step's words), which the march copies back.
  auto step = [&](int64_t z, const uint32_t(&Pz)[NP], const uint32_t(&Ryp)[NP],
                  uint32_t(&Pn)[NP], uint32_t(&Pup)[NP], const uint32_t(&Gp)[3][3],
                  uint32_t(&G1)[3][3]) {
    // planes of z + 1 (loaded one step ago); load z + 2
    make_planes(z + 1, raw, Pn);
    if (z + 2 <= z1) load_raw(z + 2, raw);
    uint32_t Pdn[NP];
    // rows y - 1 and y + 1 at z + 1 (lanes 0 and 31 get their own row: only
    // collar results depend on it)
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      Pup[k] = __shfl_down_sync(FULL, Pn[k], 1);
      Pdn[k] = __shfl_up_sync(FULL, Pn[k], 1);
    }
    // centre row shifted for dx = +1 (C[i-1]) and dx = -1 (C[i+1])
    uint32_t Cl[NP], Cr[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      Cl[k] = Pz[k] << 1;
      Cr[k] = Pz[k] >> 1;
    }
    const bool z_in = z >= 0 && z < nz, z1_in = z + 1 < nz;
    const uint32_t ALL = 0xFFFFFFFFu;
    const bool c_in = row_in && z_in;
    const uint32_t co[3] = {c_in ? cx[0] : ALL, c_in ? cx[1] : ALL, c_in ? cx[2] : ALL};
    const uint32_t no_z = c_in ? xo : ALL;
    const uint32_t no_yp = (up_in && z_in) ? xo : ALL;
    const uint32_t no1[3] = {(dn_in && z1_in) ? xo : ALL, (row_in && z1_in) ? xo : ALL,
                             (up_in && z1_in) ? xo : ALL};
    // the 13 forward comparisons, indexed by the later voxel
    const uint32_t G001 = gcmp(borrow<NB>(Pz, Cl), co[2], no_z);
    uint32_t G01[3];
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
    // the earlier voxels' words, from the neighbouring lanes: G_(0,+1,.) of
    // row y - 1 (this step), G_(1,+1,.) of row y - 1 and G_(1,-1,.) of row
    // y + 1 (previous step)
    uint32_t G01dn[3], Gdn1[3], Gup1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      G01dn[i] = __shfl_up_sync(FULL, G01[i], 1);
      Gdn1[i] = __shfl_up_sync(FULL, Gp[2][i], 1);
      Gup1[i] = __shfl_down_sync(FULL, Gp[0][i], 1);
    }
    if (__any_sync(FULL, z >= z0 && dep != 0u) && z >= z0 && dep) {
      // forward after-bits: G shifted by dx within the word
      auto sh = [](uint32_t g, int dx) -> uint32_t {
        return dx > 0 ? g >> 1 : dx < 0 ? g << 1 : g;
      };
      const uint32_t xp = sh(G001, 1), xm = ~G001;
      uint32_t a0p[3], a0m[3], ap[3][3], am[3][3];
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        a0p[dx + 1] = sh(G01[dx + 1], dx);
        a0m[dx + 1] = ~G01dn[1 - dx];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) ap[dy + 1][dx + 1] = sh(G1[dy + 1][dx + 1], dx);
        am[1][dx + 1] = ~Gp[1][1 - dx];
        am[0][dx + 1] = ~Gdn1[1 - dx];  // neighbour (-1,-1,dx): delta (1,+1,-dx) of row y-1
        am[2][dx + 1] = ~Gup1[1 - dx];  // neighbour (-1,+1,dx): delta (1,-1,-dx) of row y+1
      }
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
      auto deposit = [&](uint32_t v, int cval) {
        v &= (1u << NB) - 1u;
        if (HM == kBitsSmem) {
          atomicAdd(&hist[v], cval);
        } else {
          atomicAdd(reinterpret_cast<unsigned long long*>(im.vcec) + v,
                    (unsigned long long)(long long)cval);
        }
      };
      const unsigned char* rowz = row_ptr(z);
      if (__popc(nzm) >= 8) {
        // many non-zero changes (noisy data): per-voxel N as bytes by the
        // inverse transpose, the row's raw values re-read (an L1/L2 hit), and
        // a fully unrolled deposit with constant offsets
        const uint32_t pn[8] = {n0, n1, n2, n3, n4, 0u, 0u, 0u};
        uint32_t nbyte[8];
        untranspose8(pn, nbyte);
        uint32_t rz[RAW];
        wc::load_window<EB>(rowz, x0, nx, fast, rz);
#pragma unroll
        for (int j = 1; j <= kWcOwn; ++j) {
          if ((nzm >> j) & 1u) {
            const int N = (int)((nbyte[j >> 2] >> ((j & 3) * 8)) & 31u);
            const uint32_t v = EB == 1 ? (rz[j >> 2] >> ((j & 3) * 8)) & 0xFFu
                                       : (rz[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
            deposit(v, N - 13);
          }
        }
        nzm = 0;
      }
      while (nzm) {
        const int j = __ffs(nzm) - 1;
        nzm &= nzm - 1;
        const int N = (int)(((n0 >> j) & 1u) | (((n1 >> j) & 1u) << 1) | (((n2 >> j) & 1u) << 2) |
                            (((n3 >> j) & 1u) << 3) | (((n4 >> j) & 1u) << 4));
        // its gray value (read from global memory two steps ago); j >= 1, so
        // x0 + j >= 0
        const unsigned char* vp = rowz + (size_t)(x0 + j) * EB;
        const uint32_t v = EB == 1 ? (uint32_t)__ldg(vp)
                                   : (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(vp));
        deposit(v, N - 13);
      }
    }
  };

  uint32_t PA[NP], RA[NP], PB[NP], RB[NP];
  // a tile at z0 = 0 has no plane below (outside: every neighbour there comes
  // after, so the previous words are zero); otherwise one priming step at
  // z0 - 1 computes them
  uint32_t GA[3][3], GB[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) GA[i][j] = 0u;
  const int64_t zs = z0 == 0 ? z0 : z0 - 1;
  load_raw(zs, raw);
  make_planes(zs, raw, PA);
#pragma unroll
  for (int k = 0; k < NP; ++k) RA[k] = __shfl_down_sync(FULL, PA[k], 1);
  load_raw(zs + 1, raw);
  // (a z-march unrolled by two, the register sets trading roles instead of
  // being copied, measured much slower: two inlined copies of the step)
  for (int64_t z = zs; z < z1; ++z) {
    step(z, PA, RA, PB, RB, GA, GB);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      PA[k] = PB[k];
      RA[k] = RB[k];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) GA[i][j] = GB[i][j];
  }
}

}  // namespace ecc
