// Temporally fused automaton: one CTA advances its member super-tile by up to
// `margin` B3/S23 steps per launch on a bit image in shared memory.
//
// Word tiles.  The state is packed one bit per cell, 32 cells of a row per
// word.  Inside a super-tile of side T (T >= 32, super-tile coordinates) the
// word of row y covering columns [32c, 32c + 32) holds members iff
// c & (y >> 5) == 0, whatever the plan's rho: the CTA works on 32 x 32-cell
// word tiles, the member ones being the level-log2(T/32) gasket of word
// tiles, enumerated with lambda (Sec. 5.1 further unrolling) or, in BB mode,
// by discarding the non-member slots of the 2^j x 2^j bounding box.  A word
// tile covers whole rho x rho tiles for rho <= 32; its 32-byte row segments
// are the sectors a rho = 32 tile reads and writes.  Cells of the segment in
// non-member rho-tiles are non-members and are written back as 0.
//
// Margin boxes.  Influence travels along member cells only (non-members are
// dead for ever), at one cell per step in the 8-neighbourhood.  For s <= M <=
// T/2 every member reached from the super-tile in s steps lies in
//   left   [-M, 0) x [0, M)        top    [0, M) x [-M, 0)
//   right  [T, T+M) x [-M, M]      bottom [-M, M] x [T, T+M)
// (the right and bottom boxes reach one row / column further than the
// diffusion's 4-neighbour ones: the corner cell (T-1, 0) reaches (T, M) by M
// diagonal moves).  For M <= 31 these are the words of column -1 (left,
// bottom), 0 (top, bottom) and T/32 (right).  Box words are evolved with the
// tiles; cells whose neighbours were not staged go wrong from the box edge
// inwards, one cell per step, and never reach the super-tile within s steps.
//
// Tasks.  A task is one word column of at most 32 consecutive rows (a word
// tile, or a piece of a box); lane i of the warp that owns it keeps row i.
// Each step a lane reads the 3 x 3 words around its word (rows above and
// below, columns left and right), forms the eight neighbour planes by funnel
// shifts, applies the bit-sliced rule, masks births outside the gasket and
// writes the word to the other image.  Every staged word is the word of exactly one task
// lane; every other word of the image is 0 and stays 0.
//
// Records.  Between the launches of one call the state stays in compact
// records, one per member word tile: its 32 words (row order), 128 bytes
// instead of 32 rows of 32 bytes.  Record s * 3^wlev + j holds word tile j
// (lambda or BB rank order) of member super-tile s (its index in the level-R
// packed grid, or its BB rank); the first launch of a call reads the embedded
// array and the last one writes it.
#include "blocks.cuh"
#include "launch.h"

namespace fractal {
namespace {

constexpr int kCaTasksPerWarp = 6;

// Image geometry: rows [-M-1, T+M] (a guard row beyond each box), word columns
// [-2, T/32+1] (a guard column beyond each box column), padded to an odd
// pitch so that the 32 rows of a task fall into 32 different banks.
__host__ __device__ inline int ca_pitch(int T) { return (T >> 5) + 5; }
__host__ __device__ inline int ca_rows(int T, int M) { return T + 2 * M + 2; }
__host__ __device__ inline int ca_image_words(int T, int M) { return (ca_pitch(T) * ca_rows(T, M) + 3) & ~3; }

// Tasks of a super-tile: word tiles first, then the six box pieces.
__host__ __device__ inline int ca_tasks(int wtiles) { return wtiles + 6; }

// Task -> (word column c, first row y0, rows) in super-tile coordinates.
__device__ __forceinline__ void ca_task(int j, int wtiles, const uint32_t* tab, int T, int M, int& c, int& y0,
                                        int& rows) {
  if (j < wtiles) {
    const uint32_t e = tab[j];
    c = (int)(e & 0xffffu);
    y0 = (int)(e >> 16) * 32;
    rows = 32;
    return;
  }
  const int right = 2 * M + 1;  // rows of the right box
  switch (j - wtiles) {
    case 0: c = -1; y0 = 0; rows = M; return;                                   // left
    case 1: c = 0; y0 = -M; rows = M; return;                                   // top
    case 2: c = T >> 5; y0 = -M; rows = right < 32 ? right : 32; return;        // right, first 32 rows
    case 3: c = T >> 5; y0 = -M + 32; rows = right > 32 ? right - 32 : 0; return;  // right, the rest
    case 4: c = -1; y0 = T; rows = M; return;                                   // bottom, left word
    default: c = 0; y0 = T; rows = M; return;                                   // bottom, right word
  }
}

// 32 bytes of 0/1 cells -> 32 bits (bit i = cell i).
__device__ __forceinline__ uint32_t pack32(uint4 a, uint4 b) {
  return nz4(a.x) | nz4(a.y) << 4 | nz4(a.z) << 8 | nz4(a.w) << 12 | nz4(b.x) << 16 | nz4(b.y) << 20 |
         nz4(b.z) << 24 | nz4(b.w) << 28;
}

// The eight neighbour planes of a 32-cell word from the 3 x 3 words around
// it: for each of the rows above, at and below, the word shifted so that bit
// i holds cell i-1 (funnel shift with the left word's top cell) and cell i+1
// (with the right word's bottom cell); the row itself contributes only its
// two shifts.  Summed with full adders into the count's bits 0..2 (a count
// of 8 wraps to 0, neither 2 nor 3); B3/S23: alive next iff count is 3, or 2
// and alive now.
__device__ __forceinline__ uint32_t life_rule_words(uint32_t ul, uint32_t uc, uint32_t ur, uint32_t ml, uint32_t mc,
                                                    uint32_t mr, uint32_t dl, uint32_t dc, uint32_t dr) {
  const uint32_t a = __funnelshift_l(ul, uc, 1), b = uc, c = __funnelshift_r(uc, ur, 1);
  const uint32_t d = __funnelshift_l(ml, mc, 1), e = __funnelshift_r(mc, mr, 1);
  const uint32_t f = __funnelshift_l(dl, dc, 1), g = dc, h = __funnelshift_r(dc, dr, 1);
  const uint32_t s1 = a ^ b ^ c, c1 = (a & b) | (c & (a ^ b));
  const uint32_t s2 = d ^ e ^ f, c2 = (d & e) | (f & (d ^ e));
  const uint32_t s3 = g ^ h, c3 = g & h;
  const uint32_t bit0 = s1 ^ s2 ^ s3, c4 = (s1 & s2) | (s3 & (s1 ^ s2));
  const uint32_t t1 = c1 ^ c2 ^ c3, c5 = (c1 & c2) | (c3 & (c1 ^ c2));
  const uint32_t bit1 = t1 ^ c4, c6 = t1 & c4;
  const uint32_t bit2 = c5 ^ c6;
  return bit1 & ~bit2 & (bit0 | mc);
}

// TT: the super-tile side, a compile-time constant so that the image pitch
// and the nine neighbour offsets of a word are immediates.
template <int MODE, int TT>
__global__ void __launch_bounds__(512, 2) ca_fused_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                       int nsteps, int M, Geo g,
                                                       unsigned long long* __restrict__ partials,
                                                       const uint32_t* __restrict__ pin, uint32_t* __restrict__ pout) {
  constexpr int TPW = kCaTasksPerWarp;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ unsigned long long red[32];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (partials && threadIdx.x == 0) partials[cta_id()] = 0ull;
    return;
  }
  const int n = g.n;
  constexpr int T = TT;
  constexpr int wlev = ilog2c(TT) - 5;                 // word-tile levels of the super-tile
  constexpr int wside = 1 << wlev;                     // word tiles per super-tile side
  int wtiles = 1, wlw = 1;                             // 3^wlev, 3^ceil(wlev/2)
  for (int i = 0; i < wlev; ++i) wtiles *= 3;
  for (int i = 0; i < (wlev + 1) / 2; ++i) wlw *= 3;
  constexpr int P = (TT >> 5) + 5;                     // ca_pitch(TT)
  const int img = ca_image_words(T, M);
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm);
  uint32_t* A = tab + tab_words(wtiles);
  uint32_t* B = A + img;
  const int ox = sx * T, oy = sy * T;
  int lwR = 1;  // 3^ceil(R/2)
  for (int i = 0; i < (g.R + 1) / 2; ++i) lwR *= 3;
  // first record of this super-tile, and the record of word tile (tx, ty)
  auto st_index = [&](int x, int y) -> int64_t {
    return MODE == kLambda ? lambda_inverse(x, y, g.R, lwR) : bb_rank(x, y, g.R);
  };
  const int64_t srec = (pin || pout) ? st_index(sx, sy) * wtiles : 0;
  auto tile_record = [&](int tx, int ty) -> int64_t {
    const int lx = tx & (wside - 1), ly = ty & (wside - 1);
    const int local = MODE == kLambda ? lambda_inverse(lx, ly, wlev, wlw) : bb_rank(lx, ly, wlev);
    return st_index(tx >> wlev, ty >> wlev) * wtiles + local;
  };

  // member word tiles of the super-tile
  if (MODE == kLambda) {
    for (int j = threadIdx.x; j < wtiles; j += blockDim.x) {
      int ux, uy;
      lambda_scalar((uint32_t)(j % wlw), (uint32_t)(j / wlw), wlev, ux, uy);
      tab[j] = (uint32_t)ux | ((uint32_t)uy << 16);
    }
  } else {
    for (int j = threadIdx.x; j < wside * wside; j += blockDim.x) {
      const int ux = j & (wside - 1), uy = j >> wlev;
      if ((ux & uy) == 0) {
        int rank = 0;
        for (int q = 0; q < j; ++q) rank += ((q & (wside - 1)) & (q >> wlev)) == 0;
        tab[rank] = (uint32_t)ux | ((uint32_t)uy << 16);
      }
    }
  }
  for (int i = threadIdx.x; i < 2 * img / 4; i += blockDim.x)
    reinterpret_cast<uint4*>(A)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  // this lane's row of each of its warp's tasks: image offset and member bits
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ntasks = ca_tasks(wtiles);
  int off[TPW];
  uint32_t mk[TPW];
  // staged in two halves, each with all of its loads in flight
#pragma unroll
  for (int h = 0; h < TPW; h += TPW / 2) {
    uint4 ld[TPW / 2][2];
    uint32_t wd[TPW / 2];
#pragma unroll
    for (int k = h; k < h + TPW / 2; ++k) {
      off[k] = -1;
      mk[k] = 0u;
      const int j = warp + k * nw;
      if (j >= ntasks) continue;
      int c, y0, rows;
      ca_task(j, wtiles, tab, T, M, c, y0, rows);
      if (lane >= rows) continue;
      const int y = y0 + lane;
      const int gx0 = ox + 32 * c, gy = oy + y;
      off[k] = (y + M + 1) * P + c + 2;
      mk[k] = (unsigned)gx0 < (unsigned)n ? chunk_members<32>(gx0, gy, n) : 0u;
      if (mk[k] && pin) {  // a member word: its word tile is a member
        const int64_t rec = j < wtiles ? srec + j : tile_record(gx0 >> 5, gy >> 5);
        wd[k - h] = __ldg(pin + rec * 32 + (gy & 31));
      } else if (mk[k]) {
        const uint4* p = reinterpret_cast<const uint4*>(in + (size_t)gy * n + gx0);
        ld[k - h][0] = __ldg(p);
        ld[k - h][1] = __ldg(p + 1);
      }
    }
#pragma unroll
    for (int k = h; k < h + TPW / 2; ++k)
      if (off[k] >= 0 && mk[k]) A[off[k]] = (pin ? wd[k - h] : pack32(ld[k - h][0], ld[k - h][1])) & mk[k];
  }
  __syncthreads();

  // unrolled: the image pointers of both parities are fixed
#pragma unroll 4
  for (int t = 0; t < nsteps; ++t) {
#pragma unroll
    for (int k = 0; k < TPW; ++k) {
      if (off[k] < 0) continue;
      const uint32_t* p = A + off[k];
      B[off[k]] = life_rule_words(p[-P - 1], p[-P], p[-P + 1], p[-1], p[0], p[1], p[P - 1], p[P], p[P + 1]) & mk[k];
    }
    __syncthreads();
    uint32_t* tmp = A;
    A = B;
    B = tmp;
  }

  // write back the word tiles (whole 32-byte row segments); count the alive
  unsigned alive = 0;
#pragma unroll
  for (int k = 0; k < TPW; ++k) {
    const int j = warp + k * nw;
    if (off[k] < 0 || j >= wtiles) continue;
    const int c = off[k] % P - 2, y = off[k] / P - M - 1;
    const uint32_t w = A[off[k]];
    alive += __popc(w);
    if (pout) {  // record of word tile j, row y mod 32
      pout[(srec + j) * 32 + (y & 31)] = w;
      continue;
    }
    uint4 v0, v1;
    v0.x = spread4(w);
    v0.y = spread4(w >> 4);
    v0.z = spread4(w >> 8);
    v0.w = spread4(w >> 12);
    v1.x = spread4(w >> 16);
    v1.y = spread4(w >> 20);
    v1.z = spread4(w >> 24);
    v1.w = spread4(w >> 28);
    uint4* q = reinterpret_cast<uint4*>(out + (size_t)(oy + y) * n + ox + 32 * c);
    q[0] = v0;
    q[1] = v1;
  }
  if (partials) {  // alive members of the result, per CTA (uniform branch)
    const unsigned long long s = block_sum<unsigned long long>(alive, red);
    if (threadIdx.x == 0) partials[cta_id()] = s;
  }
}

template <int MODE>
cudaError_t go(const Launch& L, const uint8_t* in, uint8_t* out, int nsteps, int margin,
               unsigned long long* partials, const uint32_t* pin, uint32_t* pout, cudaStream_t s) {
  auto run = [&](auto* k) -> cudaError_t {
    cudaError_t e = allow_smem((const void*)k, L.smem);
    if (e != cudaSuccess) return e;
    k<<<L.grid, L.threads, L.smem, s>>>(in, out, nsteps, margin, L.geo, partials, pin, pout);
    return cudaGetLastError();
  };
  switch (L.geo.T) {
    case 32: return run(ca_fused_kernel<MODE, 32>);
    case 64: return run(ca_fused_kernel<MODE, 64>);
    case 128: return run(ca_fused_kernel<MODE, 128>);
    case 256: return run(ca_fused_kernel<MODE, 256>);
    case 512: return run(ca_fused_kernel<MODE, 512>);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int ca_fused_smem_bytes(const Geo& g, int margin) {
  const int wlev = ilog2c(g.T) - 5;
  int wtiles = 1;
  for (int i = 0; i < wlev; ++i) wtiles *= 3;
  return tab_words(wtiles) * 4 + 2 * ca_image_words(g.T, margin) * 4;
}

// Warps of a fused automaton launch: the fewest that give every warp the
// least number of tasks; 0 if the super-tile does not fit the kernel.
int ca_fused_threads(const Geo& g, int margin) {
  if (g.T < 32 || g.T > 512 || margin < 1 || margin > 31 || 2 * margin > g.T) return 0;
  int wtiles = 1;
  for (int i = 0; i < ilog2c(g.T) - 5; ++i) wtiles *= 3;
  const int tasks = ca_tasks(wtiles);
  const int per = (tasks + 15) / 16;  // with 16 warps
  if (per > kCaTasksPerWarp) return 0;
  const int warps = (tasks + per - 1) / per;
  return 32 * warps;
}

cudaError_t launch_ca_fused(int mode, const Launch& L, const uint8_t* in, uint8_t* out, int nsteps, int margin,
                            cudaStream_t s, unsigned long long* partials, const uint32_t* pin, uint32_t* pout) {
  if (nsteps < 1 || nsteps > margin || ca_fused_threads(L.geo, margin) != L.threads || (!in && !pin) ||
      (!out && !pout))
    return cudaErrorInvalidValue;
  return mode == kLambda ? go<kLambda>(L, in, out, nsteps, margin, partials, pin, pout, s)
                         : go<kBB>(L, in, out, nsteps, margin, partials, pin, pout, s);
}

int64_t ca_records(int k) {
  int64_t r = 1;
  for (int i = 5; i < k; ++i) r *= 3;
  return k >= 5 ? r : 0;
}

}  // namespace fractal
