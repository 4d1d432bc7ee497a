// Device side of the block-space map and the per-tile workloads on the
// embedded Sierpinski gasket (cell (x, y) is a member iff (x & y) == 0).
//
// Structure of every kernel in this library:
//   1. CTA -> super-tile.  The grid is the Lemma-2 orthotope of the gasket at
//      level R = r_b - m.  In lambda mode each warp evaluates lambda(omega)
//      (Theorem 1, Sec. 6.1) for omega = blockIdx with one lane per scale
//      level and a warp ballot as the sum of the Delta terms; in BB mode the
//      map is the identity over the 2^R x 2^R bounding box and non-member
//      super-tiles exit at once.
//   2. Super-tile -> tiles.  A super-tile of side T = rho * 2^m holds 3^m
//      member tiles of rho x rho cells, enumerated by applying lambda again at
//      level m ("further unrolling", Sec. 5.1); in BB mode all 4^m tile slots
//      are visited and non-member ones discarded.
//   3. Tile -> cells.  Each tile is a bounding sub-box (Sec. 5.3): every cell
//      is loaded and stored with vector accesses, and membership is the
//      arithmetic test (x & y) == 0, evaluated for a whole row segment at once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fractal {

enum : int { kLambda = 0, kBB = 1 };

// Launch geometry shared by host and device (passed by value).
struct Geo {
  int32_t n;      // embedding side 2^k
  int32_t m;      // tile levels unrolled inside one CTA
  int32_t R;      // levels mapped by the grid: r_b - m
  int32_t T;      // super-tile side in cells: rho << m
  int32_t slots;  // tile slots per CTA: 3^m (lambda) or 4^m (BB)
  int32_t lw;     // width of the level-m packed grid: 3^ceil(m/2)
  int32_t tiles;  // member tiles of a member super-tile: 3^m
};

constexpr uint32_t kNoTile = 0xffffffffu;

// Loads a thread keeps in flight at once in a staging pass; launches size the
// CTA so that one pass covers the whole super-tile.
constexpr int kIPT = 4;

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

__host__ __device__ inline int tab_words(int slots) { return (slots + 3) & ~3; }

// ---------------------------------------------------------------------------
// Membership
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool is_member(int gx, int gy, int n) {
  return (unsigned)gx < (unsigned)n && (unsigned)gy < (unsigned)n && (gx & gy) == 0;
}

// Bits i of a 32-cell row segment with (i & t) == 0, t < 32: the in-tile test
// of Sec. 6.1 evaluated for a whole row (bit i clears when i shares a bit
// with t).
__device__ __forceinline__ uint32_t row_pattern(uint32_t t) {
  uint32_t m = 0xffffffffu;
  m &= (t & 1u) ? 0x55555555u : 0xffffffffu;
  m &= (t & 2u) ? 0x33333333u : 0xffffffffu;
  m &= (t & 4u) ? 0x0f0f0f0fu : 0xffffffffu;
  m &= (t & 8u) ? 0x00ff00ffu : 0xffffffffu;
  m &= (t & 16u) ? 0x0000ffffu : 0xffffffffu;
  return m;
}

template <int W>
__device__ __forceinline__ uint32_t low_bits() {
  return W >= 32 ? 0xffffffffu : ((1u << W) - 1u);
}

// Membership bits of the W cells (gx0 .. gx0+W-1, gy); gx0 must be a
// multiple of W inside the array (callers check), so
// (gx0 + i) & gy == (gx0 & gy) | (i & gy).
template <int W>
__device__ __forceinline__ uint32_t chunk_members(int gx0, int gy, int n) {
  if ((unsigned)gy >= (unsigned)n || (gx0 & gy) != 0) return 0u;
  return row_pattern((uint32_t)gy & (uint32_t)(W - 1)) & low_bits<W>();
}

// ---------------------------------------------------------------------------
// lambda(omega), Theorem 1 / Sec. 6.1, in the (x & y) == 0 orientation
// ---------------------------------------------------------------------------

// Warp-collective.  Lane mu-1 (mu = 1..levels) extracts the replica index
//   beta_mu = digit ceil(mu/2)-1, base 3, of omega_x (odd mu) or omega_y (even mu),
// takes the replica offset from the arithmetic hash tau = (beta/2, beta - beta/2),
// flips tau_y (the paper's gasket is this one mirrored in y), and the ballot
// adds Delta^mu = tau^mu * 2^(mu-1): every level owns its own bit, so the sum
// is the ballot word.  All 32 lanes must call it with the same arguments.
__device__ __forceinline__ void warp_lambda(uint32_t wx, uint32_t wy, int levels, int& bx, int& by) {
  const unsigned lane = threadIdx.x & 31u;
  uint32_t v = (lane & 1u) ? wy : wx;  // mu = lane + 1
  const unsigned j = lane >> 1;        // ceil(mu/2) - 1
#pragma unroll
  for (unsigned i = 0; i < 8; ++i) {
    if (i < j) v /= 3u;
  }
  const uint32_t beta = v % 3u;
  const uint32_t tx = beta >> 1;
  const uint32_t ty = beta - (beta >> 1);
  const bool on = lane < (unsigned)levels;
  bx = (int)__ballot_sync(0xffffffffu, on && tx != 0u);
  by = (int)__ballot_sync(0xffffffffu, on && ty == 0u);
}

// Per-thread form of the same map (used for the few levels unrolled inside a
// CTA).  Digits of omega_x feed odd mu, digits of omega_y even mu.
__device__ __forceinline__ void lambda_scalar(uint32_t wx, uint32_t wy, int levels, int& bx, int& by) {
  uint32_t x = 0, y = 0;
  for (int mu = 1; mu <= levels; ++mu) {
    uint32_t beta;
    if (mu & 1) {
      beta = wx % 3u;
      wx /= 3u;
    } else {
      beta = wy % 3u;
      wy /= 3u;
    }
    const uint32_t tx = beta >> 1;
    const uint32_t ty = beta - (beta >> 1);
    x |= tx << (mu - 1);
    y |= (1u - ty) << (mu - 1);
  }
  bx = (int)x;
  by = (int)y;
}

// Step 1: this CTA's super-tile.  Returns false (whole CTA) for a BB block
// off the gasket.
template <int MODE>
__device__ __forceinline__ bool cta_supertile(const Geo& g, int& sx, int& sy) {
  if (MODE == kLambda) {
    warp_lambda(blockIdx.x, blockIdx.y, g.R, sx, sy);
    return true;
  }
  sx = (int)blockIdx.x;
  sy = (int)blockIdx.y;
  return (sx & sy) == 0;
}

// Inverse of the level-m map: tile (ux, uy) of a member super-tile (ux & uy
// == 0) -> its index j = omega_y * lw + omega_x in the level-m packed grid.
// Per level mu the bit pair (x, y) gives the replica index (flipped table H:
// (0,1) -> 0, (0,0) -> 1, (1,0) -> 2), a base-3 digit of omega_x (odd mu) or
// omega_y (even mu).
__device__ __forceinline__ int lambda_inverse(int ux, int uy, int levels, int lw) {
  int wx = 0, wy = 0, px = 1, py = 1;
  for (int mu = 1; mu <= levels; ++mu) {
    const int bx = (ux >> (mu - 1)) & 1, by = (uy >> (mu - 1)) & 1;
    const int beta = bx ? 2 : (by ? 0 : 1);
    if (mu & 1) {
      wx += beta * px;
      px *= 3;
    } else {
      wy += beta * py;
      py *= 3;
    }
  }
  return wy * lw + wx;
}

// Step 2: slot table in shared memory, entry = ux | uy << 16 (tile offsets
// inside the super-tile) or kNoTile for a discarded BB slot.
template <int MODE>
__device__ __forceinline__ void build_slot_table(uint32_t* tab, const Geo& g) {
  for (int j = threadIdx.x; j < g.slots; j += blockDim.x) {
    int ux, uy;
    if (MODE == kLambda) {
      lambda_scalar((uint32_t)(j % g.lw), (uint32_t)(j / g.lw), g.m, ux, uy);
      tab[j] = (uint32_t)ux | ((uint32_t)uy << 16);
    } else {
      ux = j & ((1 << g.m) - 1);
      uy = j >> g.m;
      tab[j] = (ux & uy) ? kNoTile : ((uint32_t)ux | ((uint32_t)uy << 16));
    }
  }
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (warp trees, then warp 0 over the warps).
template <typename V>
__device__ __forceinline__ V block_sum(V v, V* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    V t = lane < nw ? red[lane] : V(0);
    t = warp_sum(t);
    return t;
  }
  return V(0);
}

__device__ __forceinline__ int64_t cta_id() { return (int64_t)blockIdx.y * gridDim.x + blockIdx.x; }

// ---------------------------------------------------------------------------
// uint8 rows <-> bit rows
// ---------------------------------------------------------------------------

// 4 bytes -> 4 bits (byte b nonzero -> bit b).  Bit 7 of each byte of t is
// set iff the byte is nonzero; the multiply gathers bits 7, 15, 23, 31 into
// bits 28..31 (the partial products are distinct single bits below 28, so
// nothing carries into the top nibble).
__device__ __forceinline__ uint32_t nz4(uint32_t w) {
  const uint32_t t = (((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u;
  return (t * 0x00204081u) >> 28;
}

// 4 bits -> 4 bytes of 0/1 (bit b -> byte b); partial products are distinct
// single bits, so the mask picks exactly bits 0, 8, 16, 24.
__device__ __forceinline__ uint32_t spread4(uint32_t b) {
  return ((b & 0xfu) * 0x00204081u) & 0x01010101u;
}

// B3/S23 on a 32-cell row segment, bit-sliced: up/mid/dn are the rows above,
// at and below the segment as 34-bit windows (bit 0 = the cell left of the
// segment, bits 1..32 = its cells, bit 33 = the cell right of it).  The eight
// neighbour planes are summed with full adders into the count's bits 0..2
// (a count of 8 wraps to 0, which is neither 2 nor 3); a cell is alive next
// if the count is 3, or 2 and it is alive now.
__device__ __forceinline__ uint32_t life_rule32(uint64_t up, uint64_t mid, uint64_t dn) {
  const uint32_t a = (uint32_t)up, b = (uint32_t)(up >> 1), c = (uint32_t)(up >> 2);
  const uint32_t d = (uint32_t)mid, e = (uint32_t)(mid >> 2);
  const uint32_t f = (uint32_t)dn, g = (uint32_t)(dn >> 1), h = (uint32_t)(dn >> 2);
  const uint32_t self = (uint32_t)(mid >> 1);
  const uint32_t s1 = a ^ b ^ c, c1 = (a & b) | (c & (a ^ b));
  const uint32_t s2 = d ^ e ^ f, c2 = (d & e) | (f & (d ^ e));
  const uint32_t s3 = g ^ h, c3 = g & h;
  const uint32_t bit0 = s1 ^ s2 ^ s3, c4 = (s1 & s2) | (s3 & (s1 ^ s2));
  const uint32_t t1 = c1 ^ c2 ^ c3, c5 = (c1 & c2) | (c3 & (c1 ^ c2));
  const uint32_t bit1 = t1 ^ c4, c6 = t1 & c4;
  const uint32_t bit2 = c5 ^ c6;
  return bit1 & ~bit2 & (bit0 | self);
}

template <int W>
__device__ __forceinline__ uint32_t load_alive_bits(const uint8_t* __restrict__ p) {
  if constexpr (W == 32) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(p) + 1);
    return nz4(a.x) | nz4(a.y) << 4 | nz4(a.z) << 8 | nz4(a.w) << 12 | nz4(b.x) << 16 |
           nz4(b.y) << 20 | nz4(b.z) << 24 | nz4(b.w) << 28;
  } else if constexpr (W == 16) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    return nz4(a.x) | nz4(a.y) << 4 | nz4(a.z) << 8 | nz4(a.w) << 12;
  } else if constexpr (W == 8) {
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
    return nz4(a.x) | nz4(a.y) << 4;
  } else if constexpr (W == 4) {
    return nz4(__ldg(reinterpret_cast<const uint32_t*>(p)));
  } else if constexpr (W == 2) {
    const uint32_t v = __ldg(reinterpret_cast<const unsigned short*>(p));
    return (v & 0xffu ? 1u : 0u) | (v >> 8 ? 2u : 0u);
  } else {
    return __ldg(p) ? 1u : 0u;
  }
}

// Store W cells: byte i = ((bits >> i) & 1) * value.
template <int W>
__device__ __forceinline__ void store_state_bytes(uint8_t* __restrict__ p, uint32_t bits, uint32_t value) {
  if constexpr (W >= 16) {
#pragma unroll
    for (int h = 0; h < W / 16; ++h) {
      const uint32_t b = bits >> (16 * h);
      uint4 v;
      v.x = spread4(b) * value;
      v.y = spread4(b >> 4) * value;
      v.z = spread4(b >> 8) * value;
      v.w = spread4(b >> 12) * value;
      reinterpret_cast<uint4*>(p)[h] = v;
    }
  } else if constexpr (W == 8) {
    uint2 v;
    v.x = spread4(bits) * value;
    v.y = spread4(bits >> 4) * value;
    *reinterpret_cast<uint2*>(p) = v;
  } else if constexpr (W == 4) {
    *reinterpret_cast<uint32_t*>(p) = spread4(bits) * value;
  } else if constexpr (W == 2) {
    *reinterpret_cast<unsigned short*>(p) =
        (unsigned short)(((bits & 1u) * value) | (((bits >> 1) & 1u) * value) << 8);
  } else {
    *p = (uint8_t)((bits & 1u) * value);
  }
}

// ---------------------------------------------------------------------------
// float rows
// ---------------------------------------------------------------------------

template <int W>
struct FVec {
  float v[W];
};

template <int W>
__device__ __forceinline__ FVec<W> load_f(const float* __restrict__ p, bool global) {
  FVec<W> r;
  if constexpr (W == 4) {
    const float4 t = global ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (W == 2) {
    const float2 t = global ? __ldg(reinterpret_cast<const float2*>(p)) : *reinterpret_cast<const float2*>(p);
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    r.v[0] = global ? __ldg(p) : *p;
  }
  return r;
}

template <int W>
__device__ __forceinline__ void store_f(float* __restrict__ p, const FVec<W>& r) {
  if constexpr (W == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else if constexpr (W == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
  } else {
    *p = r.v[0];
  }
}

// ---------------------------------------------------------------------------
// Super-tile ring: the 4T+4 cells around the super-tile.  Only ring cells
// that are members AND touch a member of the super-tile are ever needed.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void ring_cell(int it, int T, int& lx, int& ly) {
  if (it < T + 2) {
    lx = it - 1; ly = -1;
  } else if (it < 2 * T + 4) {
    lx = it - (T + 2) - 1; ly = T;
  } else if (it < 3 * T + 4) {
    lx = -1; ly = it - (2 * T + 4);
  } else {
    lx = T; ly = it - (3 * T + 4);
  }
}

// Does ring cell (lx, ly) (global (gx, gy)) have a Moore neighbour that is a
// member inside the super-tile [0,T)^2?
__device__ __forceinline__ bool ring_needed(int lx, int ly, int gx, int gy, int T, int n) {
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int qx = lx + dx, qy = ly + dy;
      if ((dx | dy) != 0 && qx >= 0 && qx < T && qy >= 0 && qy < T && is_member(gx + dx, gy + dy, n))
        return true;
    }
  }
  return false;
}

}  // namespace fractal
