// TMA-staged step kernels (sm_103a): one elected warp issues a 2-D tensor
// copy (cp.async.bulk.tensor) per member tile of the CTA's super-tile into
// dense shared-memory tiles, completing on one mbarrier; the CTA then updates
// the tiles from shared memory and writes them back with vector stores.
//
// Halo.  With membership (x & y) == 0, a member tile's member cells touch
// only a handful of cells outside the tile (all of them at in-tile offsets
// whose low bits are zero, so each is a member iff its tile is):
//   von Neumann (diffusion): (0,-1), (-1,0), (rho,0), (0,rho);
//   Moore (automaton):       those four and (rho,-1), (rho,1), (-1,rho), (1,rho).
// Each comes from a neighbouring tile of the same super-tile (shared memory),
// or, for the super-tile's own border, from the matching cell of the
// super-tile's ring, which is prefetched before the wait.
#include "launch.h"
#include "tma.cuh"

namespace fractal {

// TMA writes each tile to a 128-byte aligned shared-memory slot.
__host__ __device__ constexpr int tile_stride(int tile_bytes) { return (tile_bytes + 127) & ~127; }

// Shared-memory layout of the TMA kernels; host and device compute it alike.
struct TmaLayout {
  int bar, tab, inv, ring, tiles, total;
  __host__ __device__ TmaLayout(const Geo& g, int tile_bytes) {
    const int nt = g.tiles;          // member tiles per CTA (3^m)
    const int side = 1 << g.m;       // tile slots per super-tile side
    bar = 0;
    tab = 16;
    inv = tab + ((nt * 4 + 15) & ~15);
    ring = inv + ((side * side * 2 + 15) & ~15);
    tiles = (ring + 8 * 4 + 127) & ~127;
    total = tiles + nt * tile_stride(tile_bytes);
  }
};

int tma_smem_bytes(const Geo& g, int tile_bytes) { return TmaLayout(g, tile_bytes).total; }

namespace {

// Member tiles of the super-tile in the launch's order (lambda: further
// unrolling; BB: row-major scan of all 4^m slots keeping members), and the
// inverse map (local tile -> index, -1 for a non-member tile).
template <int MODE>
__device__ __forceinline__ void build_tables(uint32_t* tab, int16_t* inv, const Geo& g) {
  const int side = 1 << g.m;
  for (int j = threadIdx.x; j < side * side; j += blockDim.x) inv[j] = -1;
  __syncthreads();
  if (MODE == kLambda) {
    for (int j = threadIdx.x; j < g.tiles; j += blockDim.x) {
      int ux, uy;
      lambda_scalar((uint32_t)(j % g.lw), (uint32_t)(j / g.lw), g.m, ux, uy);
      tab[j] = (uint32_t)ux | ((uint32_t)uy << 16);
      inv[uy * side + ux] = (int16_t)j;
    }
  } else {
    // slot j = (ux, uy) row-major; its rank among member slots is the number
    // of member slots before it (discarding the others, as the BB launch does)
    for (int j = threadIdx.x; j < side * side; j += blockDim.x) {
      const int ux = j & (side - 1), uy = j >> g.m;
      if (ux & uy) continue;
      int rank = 0;
      for (int q = 0; q < j; ++q) rank += ((q & (side - 1)) & (q >> g.m)) == 0;
      tab[rank] = (uint32_t)ux | ((uint32_t)uy << 16);
      inv[j] = (int16_t)rank;
    }
  }
}

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) diffusion_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                            const float* __restrict__ in, float* __restrict__ out,
                                                            float a, Geo g, int* err) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int MBH = RHO < 4 ? RHO : 4;                  // micro-block: 4 columns x MBH rows
  constexpr int MBX = RHO / 4;                            // micro-blocks per tile row
  constexpr int LOG_MBT = ilog2c(MBX * (RHO / MBH));      // micro-blocks per tile (log)
  constexpr int TILE = RHO * RHO;                         // floats
  constexpr int TS = tile_stride(TILE * 4) / 4;           // slot stride (floats)
  extern __shared__ __align__(128) unsigned char sm[];

  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const TmaLayout L(g, TILE * 4);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm + L.tab);
  int16_t* inv = reinterpret_cast<int16_t*>(sm + L.inv);
  float* ring = reinterpret_cast<float*>(sm + L.ring);
  float* tiles = reinterpret_cast<float*>(sm + L.tiles);
  const int n = g.n, T = g.T, side = 1 << g.m;
  const int ox = sx * T, oy = sy * T;

  if (threadIdx.x == 0) {
    prefetch_tensormap(&tin);
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  build_tables<MODE>(tab, inv, g);
  __syncthreads();

  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (uint32_t)(g.tiles * TILE * 4));
    __syncwarp();
    for (int c = threadIdx.x; c < g.tiles; c += 32) {
      const uint32_t e = tab[c];
      tma_load_2d(tiles + c * TS, &tin, ox + (int)(e & 0xffffu) * RHO, oy + (int)(e >> 16) * RHO, bar);
    }
    // super-tile ring for the von Neumann halo: (0,-1), (-1,0), (T,0), (0,T)
    if (threadIdx.x < 4) {
      const int r = threadIdx.x;
      const int lx = r == 1 ? -1 : (r == 2 ? T : 0);
      const int ly = r == 0 ? -1 : (r == 3 ? T : 0);
      const int gx = ox + lx, gy = oy + ly;
      float v = 0.0f;
      if (is_member(gx, gy, n)) v = __ldg(in + (size_t)gy * n + gx);
      ring[r] = v;
      ring[4 + r] = is_member(gx, gy, n) ? 1.0f : 0.0f;
    }
  }
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0, err, kErrTmaTimeout)) {
    mbar_wait_bounded(bar, 0, err, kErrDrainTimeout);
    return;
  }

  const int items = g.tiles << LOG_MBT;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it >> LOG_MBT;
    const int mb = it & ((1 << LOG_MBT) - 1);
    const uint32_t e = tab[c];
    const int ux = (int)(e & 0xffffu), uy = (int)(e >> 16);
    const int tx0 = (mb % MBX) * 4, ty0 = (mb / MBX) * MBH;
    const float* tile = tiles + c * TS;

    // The four cells outside the tile (value, member flag).
    float ev_up = 0.f, ev_lf = 0.f, ev_rt = 0.f, ev_dn = 0.f;
    bool ef_up = false, ef_lf = false, ef_rt = false, ef_dn = false;
    if (ty0 == 0 && tx0 == 0) {
      if (uy > 0) {
        const int q = inv[(uy - 1) * side + ux];
        if (q >= 0) { ev_up = tiles[q * TS + (RHO - 1) * RHO]; ef_up = true; }
      } else if (ux == 0) {
        ev_up = ring[0]; ef_up = ring[4] != 0.f;
      }
      if (ux > 0) {
        const int q = inv[uy * side + ux - 1];
        if (q >= 0) { ev_lf = tiles[q * TS + RHO - 1]; ef_lf = true; }
      } else if (uy == 0) {
        ev_lf = ring[1]; ef_lf = ring[5] != 0.f;
      }
    }
    if (ty0 == 0 && tx0 + 4 == RHO) {
      if (ux + 1 < side) {
        const int q = inv[uy * side + ux + 1];
        if (q >= 0) { ev_rt = tiles[q * TS]; ef_rt = true; }
      } else if (uy == 0) {
        ev_rt = ring[2]; ef_rt = ring[6] != 0.f;
      }
    }
    if (tx0 == 0 && ty0 + MBH == RHO) {
      if (uy + 1 < side) {
        const int q = inv[(uy + 1) * side + ux];
        if (q >= 0) { ev_dn = tiles[q * TS]; ef_dn = true; }
      } else if (ux == 0) {
        ev_dn = ring[3]; ef_dn = ring[7] != 0.f;
      }
    }

    float* gout = out + (size_t)(oy + uy * RHO) * n + ox + ux * RHO + tx0;
#pragma unroll
    for (int r = 0; r < MBH; ++r) {
      const int ty = ty0 + r;
      const float4 cur = *reinterpret_cast<const float4*>(tile + ty * RHO + tx0);
      float4 up = make_float4(ev_up, 0.f, 0.f, 0.f), dn = make_float4(ev_dn, 0.f, 0.f, 0.f);
      uint32_t mu = ef_up ? 1u : 0u, md = ef_dn ? 1u : 0u;
      if (ty > 0) {
        up = *reinterpret_cast<const float4*>(tile + (ty - 1) * RHO + tx0);
        mu = row_pattern((uint32_t)(ty - 1)) >> tx0;
      }
      if (ty < RHO - 1) {
        dn = *reinterpret_cast<const float4*>(tile + (ty + 1) * RHO + tx0);
        md = row_pattern((uint32_t)(ty + 1)) >> tx0;
      }
      const uint32_t pm = row_pattern((uint32_t)ty);
      const uint32_t mm = pm >> tx0;
      // left of column tx0 and right of column tx0+3
      float lf = ev_lf, rt = ev_rt;
      bool ml = (ty == 0) && ef_lf, mr = (ty == 0) && ef_rt;
      if (tx0 > 0) { lf = tile[ty * RHO + tx0 - 1]; ml = (pm >> (tx0 - 1)) & 1u; }
      if (tx0 + 4 < RHO) { rt = tile[ty * RHO + tx0 + 4]; mr = (pm >> (tx0 + 4)) & 1u; }
      const float cv[4] = {cur.x, cur.y, cur.z, cur.w};
      const float uv[4] = {up.x, up.y, up.z, up.w};
      const float dv[4] = {dn.x, dn.y, dn.z, dn.w};
      float res[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float u = cv[i];
        const bool hl = i == 0 ? ml : ((mm >> (i - 1)) & 1u) != 0u;
        const bool hr = i == 3 ? mr : ((mm >> (i + 1)) & 1u) != 0u;
        const float vl = i == 0 ? lf : cv[i > 0 ? i - 1 : 0];
        const float vr = i == 3 ? rt : cv[i < 3 ? i + 1 : 0];
        // N4 in the order up, left, right, down; absent neighbours carry no flux
        float s = ((mu >> i) & 1u) ? uv[i] - u : 0.0f;
        s += hl ? vl - u : 0.0f;
        s += hr ? vr - u : 0.0f;
        s += ((md >> i) & 1u) ? dv[i] - u : 0.0f;
        res[i] = ((mm >> i) & 1u) ? fmaf(a, s, u) : 0.0f;
      }
      *reinterpret_cast<float4*>(gout + (size_t)ty * n) = make_float4(res[0], res[1], res[2], res[3]);
    }
  }
}

// Bits of a uint8 tile row (nonzero -> 1).
template <int RHO>
__device__ __forceinline__ uint32_t row_bits(const uint8_t* p) {
  if constexpr (RHO == 32) {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const uint4 b = *reinterpret_cast<const uint4*>(p + 16);
    return nz4(a.x) | nz4(a.y) << 4 | nz4(a.z) << 8 | nz4(a.w) << 12 | nz4(b.x) << 16 | nz4(b.y) << 20 |
           nz4(b.z) << 24 | nz4(b.w) << 28;
  } else {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    return nz4(a.x) | nz4(a.y) << 4 | nz4(a.z) << 8 | nz4(a.w) << 12;
  }
}

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

// Alive bit of a cell outside tile (ux, uy): a neighbouring tile's cell
// (tile offsets dx, dy in {-1,0,1}; in-tile cell (cx, cy)), or the matching
// super-tile ring entry when the neighbour tile lies outside the super-tile.
template <int RHO>
__device__ __forceinline__ uint32_t ext_bit(const uint8_t* tiles, const int16_t* inv, const uint8_t* ring, int side,
                                            int ux, int uy, int dx, int dy, int cx, int cy) {
  const int vx = ux + dx, vy = uy + dy;
  if (vx >= 0 && vx < side && vy >= 0 && vy < side) {
    const int q = inv[vy * side + vx];
    return q >= 0 ? (tiles[q * RHO * RHO + cy * RHO + cx] != 0 ? 1u : 0u) : 0u;
  }
  // local super-tile coordinates of the cell
  const int T = RHO * side;
  const int lx = vx * RHO + cx, ly = vy * RHO + cy;
  int r = -1;
  if (lx == -1 && ly == 0) r = 0;
  else if (lx == -1 && ly == T) r = 1;
  else if (lx == 0 && ly == -1) r = 2;
  else if (lx == T && ly == -1) r = 3;
  else if (lx == T && ly == 0) r = 4;
  else if (lx == T && ly == 1) r = 5;
  else if (lx == 0 && ly == T) r = 6;
  else if (lx == 1 && ly == T) r = 7;
  return r >= 0 ? ring[r] : 0u;  // no other cell outside the super-tile can touch a member
}

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(1024) ca_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                      const uint8_t* __restrict__ in, uint8_t* __restrict__ out, Geo g,
                                                      int* err) {
  constexpr int RHO = 1 << LOG_RHO;  // 16 or 32: one lane per tile row
  constexpr int TILE = RHO * RHO;    // bytes
  static_assert(tile_stride(TILE) == TILE, "uint8 tiles of 16x16 or 32x32 bytes are 128-byte multiples");
  extern __shared__ __align__(128) unsigned char sm[];

  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const TmaLayout L(g, TILE);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm + L.tab);
  int16_t* inv = reinterpret_cast<int16_t*>(sm + L.inv);
  uint8_t* ring = reinterpret_cast<uint8_t*>(sm + L.ring);
  uint8_t* tiles = sm + L.tiles;
  const int n = g.n, T = g.T, side = 1 << g.m;
  const int ox = sx * T, oy = sy * T;

  if (threadIdx.x == 0) {
    prefetch_tensormap(&tin);
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  build_tables<MODE>(tab, inv, g);
  __syncthreads();

  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (uint32_t)(g.tiles * TILE));
    __syncwarp();
    for (int c = threadIdx.x; c < g.tiles; c += 32) {
      const uint32_t e = tab[c];
      tma_load_2d(tiles + c * TILE, &tin, ox + (int)(e & 0xffffu) * RHO, oy + (int)(e >> 16) * RHO, bar);
    }
    // the eight super-tile ring cells a member can touch (Moore halo)
    if (threadIdx.x < 8) {
      const int r = threadIdx.x;  // ring order: (-1,0) (-1,T) (0,-1) (T,-1) (T,0) (T,1) (0,T) (1,T)
      const int lx = r < 2 ? -1 : (r == 2 || r == 6) ? 0 : (r == 7 ? 1 : T);
      const int ly = r == 0 ? 0 : (r == 2 || r == 3) ? -1 : (r == 4 ? 0 : (r == 5 ? 1 : T));
      const int gx = ox + lx, gy = oy + ly;
      ring[r] = (is_member(gx, gy, n) && in[(size_t)gy * n + gx] != 0) ? 1 : 0;
    }
  }
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0, err, kErrTmaTimeout)) {
    mbar_wait_bounded(bar, 0, err, kErrDrainTimeout);
    return;
  }

  // One lane per tile row; groups of RHO lanes are one tile.  The loop runs
  // whole warps (the shuffles need every lane), padding lanes store nothing.
  const int rows = g.tiles * RHO;
  const int rows_padded = (rows + 31) & ~31;
  const int lane = threadIdx.x & 31;
  for (int it = threadIdx.x; it < rows_padded; it += blockDim.x) {
    const bool live = it < rows;
    const int c = live ? it / RHO : 0;
    const int r = it & (RHO - 1);
    const uint32_t e = tab[c];
    const int ux = (int)(e & 0xffffu), uy = (int)(e >> 16);
    const uint8_t* tile = tiles + c * TILE;
    const uint32_t pm = row_pattern((uint32_t)r) & low_bits<RHO>();
    const uint32_t bits = row_bits<RHO>(tile + r * RHO) & pm;
    // own-row window: bit 0 = cell -1, bits 1..RHO = the row, bit RHO+1 = cell RHO
    uint64_t own = (uint64_t)bits << 1;
    if (r == 0) {
      own |= ext_bit<RHO>(tiles, inv, ring, side, ux, uy, -1, 0, RHO - 1, 0);
      own |= (uint64_t)ext_bit<RHO>(tiles, inv, ring, side, ux, uy, 1, 0, 0, 0) << (RHO + 1);
    } else if (r == 1) {
      own |= (uint64_t)ext_bit<RHO>(tiles, inv, ring, side, ux, uy, 1, 0, 0, 1) << (RHO + 1);
    }
    uint64_t up = __shfl_up_sync(0xffffffffu, own, 1, RHO);
    uint64_t dn = __shfl_down_sync(0xffffffffu, own, 1, RHO);
    if (r == 0) {
      up = ((uint64_t)ext_bit<RHO>(tiles, inv, ring, side, ux, uy, 0, -1, 0, RHO - 1) << 1) |
           ((uint64_t)ext_bit<RHO>(tiles, inv, ring, side, ux, uy, 1, -1, 0, RHO - 1) << (RHO + 1));
    }
    if (r == RHO - 1) {
      dn = (uint64_t)ext_bit<RHO>(tiles, inv, ring, side, ux, uy, -1, 1, RHO - 1, 0) |
           ((uint64_t)ext_bit<RHO>(tiles, inv, ring, side, ux, uy, 0, 1, 0, 0) << 1) |
           ((uint64_t)ext_bit<RHO>(tiles, inv, ring, side, ux, uy, 0, 1, 1, 0) << 2);
    }
    const uint32_t next = life_rule32(up, own, dn) & pm;
    uint8_t* gtile = out + (size_t)(oy + uy * RHO) * n + ox + ux * RHO;
    if constexpr (RHO == 32) {
      // lanes 2q, 2q+1 store the halves of rows q and q + 16 (whole sectors)
      const int h = lane & 1;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int q = (lane >> 1) + 16 * j;
        const uint32_t b = __shfl_sync(0xffffffffu, next, q);
        if (live) store_state_bytes<16>(gtile + (size_t)q * n + 16 * h, b >> (16 * h), 1u);
      }
    } else {
      if (live) store_state_bytes<16>(gtile + (size_t)r * n, next, 1u);
    }
  }
}

template <int MODE, int LOG_RHO>
cudaError_t go_diff(const Launch& L, const CUtensorMap& map, const float* in, float* out, float a, int* err,
                    cudaStream_t s) {
  auto* k = diffusion_tma_kernel<MODE, LOG_RHO>;
  cudaError_t e = allow_smem((const void*)k, L.smem);
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, L.smem, s>>>(map, in, out, a, L.geo, err);
  return cudaGetLastError();
}

template <int MODE, int LOG_RHO>
cudaError_t go_ca(const Launch& L, const CUtensorMap& map, const uint8_t* in, uint8_t* out, int* err,
                  cudaStream_t s) {
  auto* k = ca_tma_kernel<MODE, LOG_RHO>;
  cudaError_t e = allow_smem((const void*)k, L.smem);
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, L.smem, s>>>(map, in, out, L.geo, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_diffusion_tma(int mode, int log_rho, const Launch& L, const CUtensorMap& map, const float* in,
                                 float* out, float a, int* err, cudaStream_t s) {
  switch (mode * 8 + log_rho) {
    case 0 * 8 + 2: return go_diff<kLambda, 2>(L, map, in, out, a, err, s);
    case 0 * 8 + 3: return go_diff<kLambda, 3>(L, map, in, out, a, err, s);
    case 0 * 8 + 4: return go_diff<kLambda, 4>(L, map, in, out, a, err, s);
    case 0 * 8 + 5: return go_diff<kLambda, 5>(L, map, in, out, a, err, s);
    case 1 * 8 + 2: return go_diff<kBB, 2>(L, map, in, out, a, err, s);
    case 1 * 8 + 3: return go_diff<kBB, 3>(L, map, in, out, a, err, s);
    case 1 * 8 + 4: return go_diff<kBB, 4>(L, map, in, out, a, err, s);
    case 1 * 8 + 5: return go_diff<kBB, 5>(L, map, in, out, a, err, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ca_tma(int mode, int log_rho, const Launch& L, const CUtensorMap& map, const uint8_t* in,
                          uint8_t* out, int* err, cudaStream_t s) {
  switch (mode * 8 + log_rho) {
    case 0 * 8 + 4: return go_ca<kLambda, 4>(L, map, in, out, err, s);
    case 0 * 8 + 5: return go_ca<kLambda, 5>(L, map, in, out, err, s);
    case 1 * 8 + 4: return go_ca<kBB, 4>(L, map, in, out, err, s);
    case 1 * 8 + 5: return go_ca<kBB, 5>(L, map, in, out, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fractal
