// TMA-staged step kernels (sm_103a): one elected warp issues a 2-D tensor
// copy (cp.async.bulk.tensor) per member tile of the CTA's super-tile into
// dense shared-memory tiles, plus one 16-byte box per super-tile ring cell,
// all completing on one mbarrier; the CTA then updates the tiles from shared
// memory and writes them back with vector stores.
//
// Halo.  With membership (x & y) == 0, a member tile's member cells touch
// only a handful of cells outside the tile (all of them at in-tile offsets
// whose low bits are zero, so each is a member iff its tile is):
//   von Neumann (diffusion): (0,-1), (-1,0), (rho,0), (0,rho);
//   Moore (automaton):       those four and (rho,-1), (rho,1), (-1,rho), (1,rho).
// The same holds one level up for the super-tile of side T, so its ring holds
// at most these 4 (resp. 8) cells, loaded as 16-byte TMA boxes (coordinates
// outside the array read as zero).  Everything else comes from neighbouring
// tiles in shared memory.
#include "launch.h"
#include "tma.cuh"

namespace fractal {

// TMA writes each tile and ring box to a 128-byte aligned shared-memory slot.
__host__ __device__ constexpr int tile_stride(int tile_bytes) { return (tile_bytes + 127) & ~127; }

constexpr int kRingSlot = 128;  // bytes per ring box slot (the box itself is 16 bytes)

// Shared-memory layout of the TMA kernels; host and device compute it alike.
struct TmaLayout {
  int bar, sxy, tab, inv, halo, ring, tiles, total;
  __host__ __device__ TmaLayout(const Geo& g, int tile_bytes, int rings) {
    const int side = 1 << g.m;
    bar = 0;
    sxy = 8;
    tab = 16;
    inv = tab + ((g.tiles * 4 + 15) & ~15);
    halo = inv + ((side * side * 2 + 15) & ~15);  // per tile: 4 floats + flag word, or 1 word of bits
    ring = (halo + g.tiles * 20 + 127) & ~127;
    tiles = ring + rings * kRingSlot;
    total = tiles + g.tiles * tile_stride(tile_bytes);
  }
};

namespace {

// Member tiles of the super-tile in launch order and the inverse map (local
// tile -> index, -1 for a non-member tile), one pass over the 4^m slots.
// lambda: the level-m map's order (index = omega_y * lw + omega_x);
// BB: row-major scan keeping members, as a bounding-box launch discards.
template <int MODE>
__device__ __forceinline__ void build_tables(uint32_t* tab, int16_t* inv, const Geo& g) {
  const int side = 1 << g.m;
  for (int j = threadIdx.x; j < side * side; j += blockDim.x) {
    const int ux = j & (side - 1), uy = j >> g.m;
    if (ux & uy) {
      inv[j] = -1;
      continue;
    }
    int rank;
    if (MODE == kLambda) {
      rank = lambda_inverse(ux, uy, g.m, g.lw);
    } else {
      rank = 0;
      for (int q = 0; q < j; ++q) rank += ((q & (side - 1)) & (q >> g.m)) == 0;
    }
    tab[rank] = (uint32_t)ux | ((uint32_t)uy << 16);
    inv[j] = (int16_t)rank;
  }
}

// Prologue shared by both kernels: CTA -> super-tile (lambda by warp 0, BB by
// identity), barrier init, tables.  Returns false for a discarded BB block.
template <int MODE>
__device__ __forceinline__ bool tma_prologue(const Geo& g, uint64_t* bar, int* sxy, uint32_t* tab, int16_t* inv,
                                             const CUtensorMap* t0, const CUtensorMap* t1, int& sx, int& sy) {
  if (MODE == kBB) {
    sx = (int)blockIdx.x;
    sy = (int)blockIdx.y;
    if (sx & sy) return false;
  }
  if (threadIdx.x < 32) {
    if (MODE == kLambda) {
      warp_lambda(blockIdx.x, blockIdx.y, g.R, sx, sy);
      if (threadIdx.x == 0) {
        sxy[0] = sx;
        sxy[1] = sy;
      }
    }
    if (threadIdx.x == 0) {
      prefetch_tensormap(t0);
      prefetch_tensormap(t1);
      mbar_init(bar, 1);
      fence_barrier_init();
    }
  }
  build_tables<MODE>(tab, inv, g);
  __syncthreads();
  if (MODE == kLambda) {
    sx = sxy[0];
    sy = sxy[1];
  }
  return true;
}

// Halo cell k of a square of side S (tile or super-tile), relative to its
// corner.  Moore order: (-1,0) (S,0) (S,1) (0,-1) (S,-1) (-1,S) (0,S) (1,S);
// von Neumann order: (0,-1) (-1,0) (S,0) (0,S).
__device__ __forceinline__ void moore_halo(int k, int S, int& x, int& y) {
  x = (k == 0 || k == 5) ? -1 : ((k == 3 || k == 6) ? 0 : (k == 7 ? 1 : S));
  y = (k == 0 || k == 1) ? 0 : (k == 2 ? 1 : ((k == 3 || k == 4) ? -1 : S));
}

__device__ __forceinline__ void vn_halo(int k, int S, int& x, int& y) {
  x = k == 1 ? -1 : (k == 2 ? S : 0);
  y = k == 0 ? -1 : (k == 3 ? S : 0);
}

// Global x of a ring box holding cell gx (16-byte aligned, may be negative).
template <int RB>
__device__ __forceinline__ int box_x(int gx) {
  return gx >= 0 ? (gx & ~(RB - 1)) : -RB;
}

// Warp 0: expect the bytes, then one TMA per member tile and per ring cell
// (RINGS = 8: Moore halo of the super-tile, 4: von Neumann).
template <int RHO, int E, int RINGS>
__device__ __forceinline__ void tma_issue(uint64_t* bar, const uint32_t* tab, unsigned char* tiles,
                                          unsigned char* rings, const CUtensorMap* tin, const CUtensorMap* tring,
                                          const Geo& g, int ox, int oy) {
  constexpr int TS = tile_stride(RHO * RHO * E);
  constexpr int RB = 16 / E;  // ring box width in elements
  const int lane = threadIdx.x;
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(g.tiles * RHO * RHO * E + RINGS * 16));
  __syncwarp();
  for (int c = lane; c < g.tiles; c += 32) {
    const uint32_t e = tab[c];
    tma_load_2d(tiles + c * TS, tin, ox + (int)(e & 0xffffu) * RHO, oy + (int)(e >> 16) * RHO, bar);
  }
  if (lane < RINGS) {
    int lx, ly;
    if (RINGS == 8) moore_halo(lane, g.T, lx, ly);
    else vn_halo(lane, g.T, lx, ly);
    const int gx = ox + lx, gy = oy + ly;
    tma_load_2d(rings + lane * kRingSlot, tring, box_x<RB>(gx), gy, bar);
  }
}

// ------------------------------------------------------------- diffusion ----

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(256, 4) diffusion_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                            const __grid_constant__ CUtensorMap tring,
                                                            float* __restrict__ out, float a, Geo g, int* err) {
  constexpr int RHO = 1 << LOG_RHO;                       // >= 4
  constexpr int MBX = RHO / 4;                            // float4s per tile row
  constexpr int LOG_Q = 2 * LOG_RHO - 2;                  // float4s per tile (log)
  constexpr int TILE = RHO * RHO;                         // floats
  constexpr int TS = tile_stride(TILE * 4) / 4;           // slot stride (floats)
  constexpr int RB = 4;                                   // ring box: 4 floats
  extern __shared__ __align__(128) unsigned char sm[];

  const TmaLayout L(g, TILE * 4, 4);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);
  int* sxy = reinterpret_cast<int*>(sm + L.sxy);
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm + L.tab);
  int16_t* inv = reinterpret_cast<int16_t*>(sm + L.inv);
  const float* ring = reinterpret_cast<const float*>(sm + L.ring);
  float* tiles = reinterpret_cast<float*>(sm + L.tiles);
  int sx, sy;
  if (!tma_prologue<MODE>(g, bar, sxy, tab, inv, &tin, &tring, sx, sy)) return;
  const int n = g.n, T = g.T, side = 1 << g.m;
  const int ox = sx * T, oy = sy * T;
  // super-tile ring cells of the von Neumann halo: (0,-1), (-1,0), (T,0), (0,T)
  if (threadIdx.x < 32)
    tma_issue<RHO, 4, 4>(bar, tab, reinterpret_cast<unsigned char*>(tiles), sm + L.ring, &tin, &tring, g, ox, oy);
  if (!mbar_wait_bounded(bar, 0, err, kErrTmaTimeout)) {
    mbar_wait_bounded(bar, 0, err, kErrDrainTimeout);
    return;
  }

  // Halo pre-pass: the four cells outside each tile, (0,-1) (-1,0) (rho,0)
  // (0,rho), from the neighbouring tile's corner cell or the super-tile ring;
  // absent cells get value 0 and flag 0.
  float* hv = reinterpret_cast<float*>(sm + L.halo);                     // [tiles][4]
  uint32_t* hf = reinterpret_cast<uint32_t*>(sm + L.halo + g.tiles * 16);  // [tiles] flag bits
  for (int t = threadIdx.x; t < g.tiles * 4; t += blockDim.x) {
    const int c = t >> 2, k = t & 3;
    const uint32_t e = tab[c];
    const int ux = (int)(e & 0xffffu), uy = (int)(e >> 16);
    int hx, hy;
    vn_halo(k, RHO, hx, hy);
    const int dx = hx < 0 ? -1 : (hx >= RHO ? 1 : 0), dy = hy < 0 ? -1 : (hy >= RHO ? 1 : 0);
    const int vx = ux + dx, vy = uy + dy;
    float v = 0.f;
    bool f = false;
    if (vx >= 0 && vx < side && vy >= 0 && vy < side) {
      const int q = inv[vy * side + vx];
      if (q >= 0) {
        v = tiles[q * TS + (hy - dy * RHO) * RHO + (hx - dx * RHO)];
        f = true;
      }
    } else {
      // outside the super-tile: the super-tile's halo cell of the same index or no member
      int rx, ry;
      vn_halo(k, T, rx, ry);
      const int lx = ux * RHO + hx, ly = uy * RHO + hy;
      if (lx == rx && ly == ry) {
        const int gx = ox + lx, gy = oy + ly;
        f = is_member(gx, gy, n);
        if (f) v = ring[k * (kRingSlot / 4) + gx - box_x<RB>(gx)];
      }
    }
    hv[t] = v;
    reinterpret_cast<uint8_t*>(hf)[t] = f ? 1 : 0;
  }
  __syncthreads();

  // One thread per 4-column strip of a tile, walking all RHO rows; the S =
  // RHO/4 strips of a tile are adjacent lanes (horizontal neighbours by
  // shuffle).  Tiles start their walk at different rows so that the 8 lanes
  // of a 128-bit shared-memory phase read 8 different bank groups.  Whole
  // warps run every iteration (shuffles); padding lanes store nothing.
  constexpr int S = RHO / 4;
  constexpr int LOG_S = LOG_RHO - 2;
  const int lane = threadIdx.x & 31;
  const int strip = lane & (S - 1);
  const int tx0 = strip * 4;
  const int rot = (lane >> LOG_S) & ((8 >> LOG_S) > 1 ? (8 >> LOG_S) - 1 : 0) & (RHO - 1);
  const int items = g.tiles * S;
  const int items_padded = (items + 31) & ~31;
  for (int it = threadIdx.x; it < items_padded; it += blockDim.x) {
    const bool live = it < items;
    const int c = live ? (it >> LOG_S) : 0;
    const uint32_t e = tab[c];
    const int ux = (int)(e & 0xffffu), uy = (int)(e >> 16);
    const float* tile = tiles + c * TS;
    const uint32_t hfl = reinterpret_cast<const uint32_t*>(hf)[c];  // byte k = flag of halo k
    const float ev_up = hv[c * 4 + 0], ev_lf = hv[c * 4 + 1], ev_rt = hv[c * 4 + 2], ev_dn = hv[c * 4 + 3];
    const bool ef_up = (hfl & 0xffu) != 0u, ef_lf = (hfl & 0xff00u) != 0u;
    const bool ef_rt = (hfl & 0xff0000u) != 0u, ef_dn = (hfl & 0xff000000u) != 0u;
    float* gtile = out + (size_t)(oy + uy * RHO) * n + ox + ux * RHO + tx0;
#pragma unroll 2
    for (int st = 0; st < RHO; ++st) {
      const int ty = (st + rot) & (RHO - 1);
      const float4 cur = *reinterpret_cast<const float4*>(tile + ty * RHO + tx0);
      float4 up = *reinterpret_cast<const float4*>(tile + (ty > 0 ? ty - 1 : 0) * RHO + tx0);
      float4 dn = *reinterpret_cast<const float4*>(tile + (ty < RHO - 1 ? ty + 1 : RHO - 1) * RHO + tx0);
      const uint32_t pm = row_pattern((uint32_t)ty);
      uint32_t mu, md;
      if (ty > 0) {
        mu = row_pattern((uint32_t)(ty - 1)) >> tx0;
      } else {
        up = make_float4(ev_up, 0.f, 0.f, 0.f);
        mu = (strip == 0 && ef_up) ? 1u : 0u;
      }
      if (ty < RHO - 1) {
        md = row_pattern((uint32_t)(ty + 1)) >> tx0;
      } else {
        dn = make_float4(ev_dn, 0.f, 0.f, 0.f);
        md = (strip == 0 && ef_dn) ? 1u : 0u;
      }
      const uint32_t mm = pm >> tx0;
      // horizontal neighbours across strips
      float lf = __shfl_up_sync(0xffffffffu, cur.w, 1, S);
      float rt = __shfl_down_sync(0xffffffffu, cur.x, 1, S);
      bool ml, mr;
      if (strip > 0) {
        ml = (pm >> (tx0 - 1)) & 1u;
      } else {
        lf = ev_lf;
        ml = ty == 0 && ef_lf;
      }
      if (strip < S - 1) {
        mr = (pm >> (tx0 + 4)) & 1u;
      } else {
        rt = ev_rt;
        mr = ty == 0 && ef_rt;
      }
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
        float acc = ((mu >> i) & 1u) ? uv[i] - u : 0.0f;
        acc += hl ? vl - u : 0.0f;
        acc += hr ? vr - u : 0.0f;
        acc += ((md >> i) & 1u) ? dv[i] - u : 0.0f;
        res[i] = ((mm >> i) & 1u) ? fmaf(a, acc, u) : 0.0f;
      }
      if (live) *reinterpret_cast<float4*>(gtile + (size_t)ty * n) = make_float4(res[0], res[1], res[2], res[3]);
    }
  }
}

// ------------------------------------------------------------- automaton ----

__device__ __forceinline__ uint32_t nz_half(uint4 v) {
  return nz4(v.x) | nz4(v.y) << 4 | nz4(v.z) << 8 | nz4(v.w) << 12;
}

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512, 4) ca_tma_kernel(const __grid_constant__ CUtensorMap tin,
                                                      const __grid_constant__ CUtensorMap tring,
                                                      uint8_t* __restrict__ out, Geo g, int* err) {
  constexpr int RHO = 1 << LOG_RHO;  // 16 or 32: one lane per tile row
  constexpr int TILE = RHO * RHO;    // bytes
  static_assert(tile_stride(TILE) == TILE, "uint8 tiles of 16x16 or 32x32 bytes are 128-byte multiples");
  constexpr int RB = 16;             // ring box: 16 bytes
  extern __shared__ __align__(128) unsigned char sm[];

  const TmaLayout L(g, TILE, 8);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);
  int* sxy = reinterpret_cast<int*>(sm + L.sxy);
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm + L.tab);
  int16_t* inv = reinterpret_cast<int16_t*>(sm + L.inv);
  const uint8_t* ring = sm + L.ring;
  uint8_t* tiles = sm + L.tiles;
  int sx, sy;
  if (!tma_prologue<MODE>(g, bar, sxy, tab, inv, &tin, &tring, sx, sy)) return;
  const int n = g.n, T = g.T, side = 1 << g.m;
  const int ox = sx * T, oy = sy * T;
  // the eight super-tile ring cells a member can touch (Moore halo)
  if (threadIdx.x < 32) tma_issue<RHO, 1, 8>(bar, tab, tiles, sm + L.ring, &tin, &tring, g, ox, oy);
  if (!mbar_wait_bounded(bar, 0, err, kErrTmaTimeout)) {
    mbar_wait_bounded(bar, 0, err, kErrDrainTimeout);
    return;
  }

  // Halo pre-pass: alive bit of each of the 8 Moore halo cells of every
  // tile, (-1,0) (R,0) (R,1) (0,-1) (R,-1) (-1,R) (0,R) (1,R) with R = rho,
  // from the neighbouring tile or the super-tile ring (absent cells: 0).
  uint8_t* hb = sm + L.halo;  // [tiles][8]
  for (int t = threadIdx.x; t < g.tiles * 8; t += blockDim.x) {
    const int c = t >> 3, k = t & 7;
    const uint32_t e = tab[c];
    const int ux = (int)(e & 0xffffu), uy = (int)(e >> 16);
    int hx, hy;
    moore_halo(k, RHO, hx, hy);
    const int dx = hx < 0 ? -1 : (hx >= RHO ? 1 : 0), dy = hy < 0 ? -1 : (hy >= RHO ? 1 : 0);
    const int vx = ux + dx, vy = uy + dy;
    uint8_t bit = 0;
    if (vx >= 0 && vx < side && vy >= 0 && vy < side) {
      const int q = inv[vy * side + vx];
      if (q >= 0) bit = tiles[q * TILE + (hy - dy * RHO) * RHO + (hx - dx * RHO)] != 0;
    } else {
      // Outside the super-tile the cell is the super-tile's halo cell of the
      // same index or no member at all (no other cell outside the
      // super-tile neighbours one of its members).
      int rx, ry;
      moore_halo(k, T, rx, ry);
      const int lx = ux * RHO + hx, ly = uy * RHO + hy;
      if (lx == rx && ly == ry) {
        const int gx = ox + lx, gy = oy + ly;
        bit = is_member(gx, gy, n) && ring[k * kRingSlot + gx - box_x<RB>(gx)] != 0;
      }
    }
    hb[t] = bit;
  }
  __syncthreads();

  // One lane per tile row; groups of RHO lanes are one tile.  The loop runs
  // whole warps (the shuffles need every lane); padding lanes compute on tile
  // 0 and store nothing.
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
    const uint2 hw = *reinterpret_cast<const uint2*>(hb + c * 8);
    const uint32_t halo = nz4(hw.x) | (nz4(hw.y) << 4);

    // this row's bits; the two 16-byte halves are read in an order that
    // spreads a 128-bit shared-memory phase over all bank groups
    const uint32_t pm = row_pattern((uint32_t)r) & low_bits<RHO>();
    uint32_t bits;
    if constexpr (RHO == 32) {
      const int h0 = (r >> 2) & 1;
      const uint4 p = *reinterpret_cast<const uint4*>(tile + r * RHO + 16 * h0);
      const uint4 q = *reinterpret_cast<const uint4*>(tile + r * RHO + 16 * (1 - h0));
      const uint32_t bp = nz_half(p), bq = nz_half(q);
      bits = h0 ? (bq | bp << 16) : (bp | bq << 16);
    } else {
      bits = nz_half(*reinterpret_cast<const uint4*>(tile + r * RHO));
    }
    bits &= pm;
    // own-row window: bit 0 = cell -1, bits 1..RHO = the row, bit RHO+1 = cell RHO
    uint64_t own = (uint64_t)bits << 1;
    if (r == 0) own |= (uint64_t)(halo & 1u) | ((uint64_t)((halo >> 1) & 1u) << (RHO + 1));
    if (r == 1) own |= (uint64_t)((halo >> 2) & 1u) << (RHO + 1);
    uint64_t up = __shfl_up_sync(0xffffffffu, own, 1, RHO);
    uint64_t dn = __shfl_down_sync(0xffffffffu, own, 1, RHO);
    if (r == 0) up = ((uint64_t)((halo >> 3) & 1u) << 1) | ((uint64_t)((halo >> 4) & 1u) << (RHO + 1));
    if (r == RHO - 1)
      dn = (uint64_t)((halo >> 5) & 1u) | ((uint64_t)((halo >> 6) & 1u) << 1) | ((uint64_t)((halo >> 7) & 1u) << 2);
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
cudaError_t go_diff(const Launch& L, const CUtensorMap& map, const CUtensorMap& ring, float* out, float a, int* err,
                    cudaStream_t s) {
  auto* k = diffusion_tma_kernel<MODE, LOG_RHO>;
  cudaError_t e = allow_smem((const void*)k, L.smem);
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, L.smem, s>>>(map, ring, out, a, L.geo, err);
  return cudaGetLastError();
}

template <int MODE, int LOG_RHO>
cudaError_t go_ca(const Launch& L, const CUtensorMap& map, const CUtensorMap& ring, uint8_t* out, int* err,
                  cudaStream_t s) {
  auto* k = ca_tma_kernel<MODE, LOG_RHO>;
  cudaError_t e = allow_smem((const void*)k, L.smem);
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, L.smem, s>>>(map, ring, out, L.geo, err);
  return cudaGetLastError();
}

}  // namespace

// Ring cells staged per super-tile: 8 (uint8 automaton, Moore) or 4 (float32 diffusion).
int tma_smem_bytes(const Geo& g, int tile_bytes, int dtype) {
  return TmaLayout(g, tile_bytes, dtype == 0 ? 8 : 4).total;
}

cudaError_t launch_diffusion_tma(int mode, int log_rho, const Launch& L, const CUtensorMap& map,
                                 const CUtensorMap& ring, float* out, float a, int* err, cudaStream_t s) {
  switch (mode * 8 + log_rho) {
    case 0 * 8 + 2: return go_diff<kLambda, 2>(L, map, ring, out, a, err, s);
    case 0 * 8 + 3: return go_diff<kLambda, 3>(L, map, ring, out, a, err, s);
    case 0 * 8 + 4: return go_diff<kLambda, 4>(L, map, ring, out, a, err, s);
    case 0 * 8 + 5: return go_diff<kLambda, 5>(L, map, ring, out, a, err, s);
    case 1 * 8 + 2: return go_diff<kBB, 2>(L, map, ring, out, a, err, s);
    case 1 * 8 + 3: return go_diff<kBB, 3>(L, map, ring, out, a, err, s);
    case 1 * 8 + 4: return go_diff<kBB, 4>(L, map, ring, out, a, err, s);
    case 1 * 8 + 5: return go_diff<kBB, 5>(L, map, ring, out, a, err, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ca_tma(int mode, int log_rho, const Launch& L, const CUtensorMap& map, const CUtensorMap& ring,
                          uint8_t* out, int* err, cudaStream_t s) {
  switch (mode * 8 + log_rho) {
    case 0 * 8 + 4: return go_ca<kLambda, 4>(L, map, ring, out, err, s);
    case 0 * 8 + 5: return go_ca<kLambda, 5>(L, map, ring, out, err, s);
    case 1 * 8 + 4: return go_ca<kBB, 4>(L, map, ring, out, err, s);
    case 1 * 8 + 5: return go_ca<kBB, 5>(L, map, ring, out, err, s);
    default: return cudaErrorInvalidValue;
  }
}

// Bounded-wait self-test: an mbarrier armed for one arrival that never
// comes (no copy is issued), waited for by every thread with the step
// kernels' bounded wait; on timeout the first thread records the code in
// *err and all return.  Nothing is in flight when the wait gives up.
__global__ void __launch_bounds__(32) wait_selftest_kernel(int* __restrict__ err, uint32_t spins) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  mbar_wait_bounded(&bar, 0, threadIdx.x == 0 ? err : nullptr, kErrTmaTimeout, spins);
}

cudaError_t launch_wait_selftest(int* err, uint32_t spins, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(err, spins);
  return cudaGetLastError();
}

}  // namespace fractal
