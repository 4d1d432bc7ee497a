// 8 x 8-cell blocks of the gasket (internal): a block (BX, BY) with BX & BY
// == 0 holds the 27 members (i, j), i & j == 0, of a level-3 gasket and meets
// the rest of the gasket through four links only: (0,0) to (0,7) of the block
// above and to (7,0) of the block left, (7,0) to (0,0) of the block right,
// (0,7) to (0,0) of the block below.  Its member cells lie in 12 of its 16
// 16-byte row chunks (columns 0-3 of every row, 4-7 of rows 0-3); a row of 8
// floats is one 32-byte sector.
#pragma once

#include "dfloat.cuh"
#include "gasket.cuh"

namespace fractal {
namespace {

constexpr int kB = 8;

__host__ __device__ constexpr bool amem(int i, int j) { return i >= 0 && j >= 0 && i < kB && j < kB && (i & j) == 0; }

__device__ __forceinline__ bool ablock(int gx, int gy, int nblk) {
  return (unsigned)gx < (unsigned)nblk && (unsigned)gy < (unsigned)nblk && (gx & gy) == 0;
}

// Four consecutive values of a row, 16-byte accesses.
__device__ __forceinline__ void ld4(const float* p, float* v) {
  const float4 c = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = c.x;
  v[1] = c.y;
  v[2] = c.z;
  v[3] = c.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
  const double2 c0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 c1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = c0.x;
  v[1] = c0.y;
  v[2] = c1.x;
  v[3] = c1.y;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

__device__ __forceinline__ float ldg1(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldg1(const double* p) { return __ldg(p); }

// The block's member values (0 at non-members) from a row-major n x n array.
template <typename T>
__device__ __forceinline__ void load_block(T (&v)[kB * kB], const T* __restrict__ p, int n) {
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    ld4(p + (size_t)j * n, &v[j * kB]);
    if (j < 4) {
      ld4(p + (size_t)j * n + 4, &v[j * kB + 4]);
    } else {
#pragma unroll
      for (int i = 4; i < kB; ++i) v[j * kB + i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < kB; ++i)
      if (!amem(i, j)) v[j * kB + i] = T(0);
  }
}

template <typename T>
__device__ __forceinline__ void store_block(T* __restrict__ p, int n, const T (&v)[kB * kB]) {
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    st4(p + (size_t)j * n, &v[j * kB]);
    st4(p + (size_t)j * n + 4, &v[j * kB + 4]);
  }
}

// Neighbour cells at the ports: up (0,-1), left (-1,0), right (8,0), down
// (0,8) relative to the block origin; 0 where that block is not a member
// (or outside the array).
template <typename T>
struct Ports {
  T up, lf, rt, dn;
};

template <typename T>
__device__ __forceinline__ Ports<T> load_ports(const T* __restrict__ base, int n, bool hu, bool hl, bool hr, bool hd) {
  Ports<T> q;
  q.up = hu ? ldg1(base - n) : T(0);
  q.lf = hl ? ldg1(base - 1) : T(0);
  q.rt = hr ? ldg1(base + kB) : T(0);
  q.dn = hd ? ldg1(base + (size_t)kB * n) : T(0);
  return q;
}

// Visit the member neighbours of member cell (i, j): f(u there, kappa there,
// x there) for three fields u, kappa, x of the block and its ports.
template <typename T, typename F>
__device__ __forceinline__ void for_neighbours(int i, int j, const T (&u)[kB * kB], const float (&k)[kB * kB],
                                               const T (&x)[kB * kB], const Ports<T>& pu, const Ports<float>& pk,
                                               const Ports<T>& px, bool hu, bool hl, bool hr, bool hd, F f) {
  if (amem(i, j - 1)) f(u[(j - 1) * kB + i], k[(j - 1) * kB + i], x[(j - 1) * kB + i]);
  if (amem(i - 1, j)) f(u[j * kB + i - 1], k[j * kB + i - 1], x[j * kB + i - 1]);
  if (amem(i + 1, j)) f(u[j * kB + i + 1], k[j * kB + i + 1], x[j * kB + i + 1]);
  if (amem(i, j + 1)) f(u[(j + 1) * kB + i], k[(j + 1) * kB + i], x[(j + 1) * kB + i]);
  if (i == 0 && j == 0) {
    if (hu) f(pu.up, pk.up, px.up);
    if (hl) f(pu.lf, pk.lf, px.lf);
  }
  if (i == kB - 1 && j == 0 && hr) f(pu.rt, pk.rt, px.rt);
  if (i == 0 && j == kB - 1 && hd) f(pu.dn, pk.dn, px.dn);
}

// This thread's block and whether it and its four neighbour blocks are members.
struct BlockPos {
  bool active;
  bool hu, hl, hr, hd;
  size_t base;  // element index of the block origin
};

template <int MODE>
__device__ __forceinline__ bool block_pos(const Geo& g, int L, BlockPos& b) {
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return false;  // whole CTA: BB slot off the gasket
  int nb = 1, lw = 1;
  for (int i = 0; i < L; ++i) nb *= 3;
  for (int i = 0; i < (L + 1) / 2; ++i) lw *= 3;
  b.active = false;
  const int t = threadIdx.x;
  if (t >= nb) return true;
  int bx, by;
  lambda_scalar((uint32_t)(t % lw), (uint32_t)(t / lw), L, bx, by);
  const int GX = (sx << L) + bx, GY = (sy << L) + by, nblk = g.n / kB;
  b.active = true;
  b.hu = ablock(GX, GY - 1, nblk);
  b.hl = ablock(GX - 1, GY, nblk);
  b.hr = ablock(GX + 1, GY, nblk);
  b.hd = ablock(GX, GY + 1, nblk);
  b.base = (size_t)GY * kB * (size_t)g.n + (size_t)GX * kB;
  return true;
}

// Member 4-degree of cell (i, j) inside the block (its links to other blocks
// are added at the ports).
__host__ __device__ constexpr int bdeg(int i, int j) {
  return (amem(i - 1, j) ? 1 : 0) + (amem(i + 1, j) ? 1 : 0) + (amem(i, j - 1) ? 1 : 0) + (amem(i, j + 1) ? 1 : 0);
}

// Sum of a cell's neighbour values, in a fixed order, with no leading 0 + x.
struct NbSum {
  float s = 0.f;
  bool any = false;
  __device__ __forceinline__ void add(float v) {
    s = any ? s + v : v;
    any = true;
  }
};

// One step of the 27 members of a block: u' = u + a * (sum of member
// neighbours - degree * u).  Non-member neighbours hold no value and are not
// summed; vu, vl, vr, vd are the neighbour values at the ports (0 where the
// neighbour is not a staged member) and d0, dr, dd the ports' degrees.
//
// The 27 members and 26 links of a block form a tree; bparent names each
// member's parent in it (the left neighbour if that is a member, else the
// one above), and these parent links are all 26 links.  The update runs in
// place, children before parents (anti-diagonals from the far corner): a
// cell's old value joins its parent's neighbour sum before the cell is
// overwritten, and the parent is still old when the cell is updated, so no
// second copy of the block is needed.
__host__ __device__ constexpr int bparent(int i, int j) {
  return (i > 0 && amem(i - 1, j)) ? j * kB + i - 1 : (j - 1) * kB + i;
}

__device__ __forceinline__ void block_step(float (&u)[kB * kB], float a, float vu, float vl, float vr, float vd,
                                           float d0, float dr, float dd) {
  NbSum acc[kB * kB];  // children's old values, per cell
#pragma unroll
  for (int s = 2 * (kB - 1); s >= 0; --s) {
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int i = s - j;
      if (i < 0 || i >= kB || !amem(i, j)) continue;
      const int q = j * kB + i;
      NbSum nb = acc[q];
      float d = (float)bdeg(i, j);
      if (q != 0) nb.add(u[bparent(i, j)]);
      if (i == 0 && j == 0) {
        nb.add(vu);
        nb.add(vl);
        d = d0;
      }
      if (i == kB - 1 && j == 0) {
        nb.add(vr);
        d = dr;
      }
      if (i == 0 && j == kB - 1) {
        nb.add(vd);
        d = dd;
      }
      const float c = u[q];
      if (q != 0) acc[bparent(i, j)].add(c);
      u[q] = fmaf(a, fmaf(-d, c, nb.s), c);
    }
  }
}

// The same step for two blocks at once, one in .x and one in .y of every
// value: each operation is a paired FP32 instruction (two IEEE
// round-to-nearest operations, the same results as the scalar form).
// nd0, ndr, ndd: the ports' degrees, negated.
struct NbSum2 {
  float2 s = make_float2(0.f, 0.f);
  bool any = false;
  __device__ __forceinline__ void add(float2 v) {
    s = any ? __fadd2_rn(s, v) : v;
    any = true;
  }
};

__device__ __forceinline__ void block_step2(float2 (&u)[kB * kB], float2 a, float2 vu, float2 vl, float2 vr, float2 vd,
                                            float2 nd0, float2 ndr, float2 ndd) {
  NbSum2 acc[kB * kB];  // children's old values, per cell
#pragma unroll
  for (int s = 2 * (kB - 1); s >= 0; --s) {
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int i = s - j;
      if (i < 0 || i >= kB || !amem(i, j)) continue;
      const int q = j * kB + i;
      NbSum2 nb = acc[q];
      const float dn = -(float)bdeg(i, j);
      float2 nd = make_float2(dn, dn);
      if (q != 0) nb.add(u[bparent(i, j)]);
      if (i == 0 && j == 0) {
        nb.add(vu);
        nb.add(vl);
        nd = nd0;
      }
      if (i == kB - 1 && j == 0) {
        nb.add(vr);
        nd = ndr;
      }
      if (i == 0 && j == kB - 1) {
        nb.add(vd);
        nd = ndd;
      }
      const float2 c = u[q];
      if (q != 0) acc[bparent(i, j)].add(c);
      u[q] = __ffma2_rn(a, __ffma2_rn(nd, c, nb.s), c);
    }
  }
}

// A 16-byte chunk of row j starting at column i0 with its non-members zeroed.
__device__ __forceinline__ float4 mask_chunk(float4 v, int i0, int j) {
  v.x = amem(i0 + 0, j) ? v.x : 0.f;
  v.y = amem(i0 + 1, j) ? v.y : 0.f;
  v.z = amem(i0 + 2, j) ? v.z : 0.f;
  v.w = amem(i0 + 3, j) ? v.w : 0.f;
  return v;
}

// Rank of the member slot (x, y) among the member slots (x & y == 0) of the
// 2^L x 2^L box in row-major order (the BB enumeration, compacted).  Rows
// above contribute sum_{y' < y} 2^(L - popc(y')); the row itself the x' < x
// with x' & y == 0.  Both by the bits from the top, O(L).
__device__ __forceinline__ int bb_rank(int x, int y, int L) {
  int above = 0, pref = 1, p3 = 1;
  for (int i = 0; i < L; ++i) p3 *= 3;
  for (int i = L - 1; i >= 0; --i) {
    p3 /= 3;  // 3^i
    if ((y >> i) & 1) {
      above += pref * 2 * p3;
    } else {
      pref *= 2;
    }
  }
  int within = 0;
  for (int i = L - 1; i >= 0; --i) {
    if ((x >> i) & 1) {
      within += 1 << (i - __popc(y & ((1 << i) - 1)));
      if ((y >> i) & 1) break;
    }
  }
  return above + within;
}

}  // namespace
}  // namespace fractal
