// Fractal Life-like automaton step (Sec. 6.2, test CA), rule B3/S23 on the
// Moore neighbourhood, counting only gasket members.
//
// One CTA per member super-tile.  The super-tile and the few ring cells it
// needs are staged in shared memory as a bit image (1 bit per cell, alive AND
// member), so the eight neighbour counts of 32 cells are a handful of
// bit-sliced full adders on 32-bit words.
#include "launch.h"

namespace fractal {
namespace {

// 34-bit window of image row `row`: bit 0 = cell lx0-1, bit i+1 = cell lx0+i.
// Cell lx lives in word (lx + 32) >> 5, bit lx & 31 (word 0 is the left pad).
__device__ __forceinline__ uint64_t bit_window(const uint32_t* row, int lx0) {
  const int b = ((lx0 + 32) >> 5) - 1;
  const int pos = 31 + (lx0 & 31);  // bit of cell lx0-1 in row[b] | row[b+1] << 32 | row[b+2] << 64
  const uint64_t lo = (uint64_t)row[b] | ((uint64_t)row[b + 1] << 32);
  return (lo >> pos) | ((uint64_t)row[b + 2] << (64 - pos));
}

// B3/S23 on bit rows: bit i of the result is the next state of cell lx0+i.
__device__ __forceinline__ uint32_t life_rule(uint64_t up, uint64_t mid, uint64_t dn) {
  const uint32_t a = (uint32_t)up, b = (uint32_t)(up >> 1), c = (uint32_t)(up >> 2);
  const uint32_t d = (uint32_t)mid, e = (uint32_t)(mid >> 2);
  const uint32_t f = (uint32_t)dn, g = (uint32_t)(dn >> 1), h = (uint32_t)(dn >> 2);
  const uint32_t self = (uint32_t)(mid >> 1);
  // weight-1 column: three full adders and a half adder
  const uint32_t s1 = a ^ b ^ c, c1 = (a & b) | (c & (a ^ b));
  const uint32_t s2 = d ^ e ^ f, c2 = (d & e) | (f & (d ^ e));
  const uint32_t s3 = g ^ h, c3 = g & h;
  const uint32_t bit0 = s1 ^ s2 ^ s3, c4 = (s1 & s2) | (s3 & (s1 ^ s2));
  // weight-2 column: c1 + c2 + c3 + c4
  const uint32_t t1 = c1 ^ c2 ^ c3, c5 = (c1 & c2) | (c3 & (c1 ^ c2));
  const uint32_t bit1 = t1 ^ c4, c6 = t1 & c4;
  // weight-4 column (a count of 8 wraps to 0, which is neither 2 nor 3)
  const uint32_t bit2 = c5 ^ c6;
  // count == 3, or count == 2 and alive
  return bit1 & ~bit2 & (bit0 | self);
}

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) ca_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                 Geo g) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int WC = RHO;                     // update chunk: one tile row (<= 32 cells)
  constexpr int WL = RHO < 16 ? RHO : 16;     // load chunk: at most 16 bytes
  constexpr int LOG_LQ = 2 * LOG_RHO - ilog2c(WL);  // load chunks per tile
  extern __shared__ __align__(16) uint32_t smem[];

  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const int n = g.n;
  const int T = g.T;
  const int wpr = (T >> 5) + 3;  // words per image row
  uint32_t* tab = smem;
  uint32_t* img = smem + tab_words(g.slots);
  const int img_words = (T + 2) * wpr;

  build_slot_table<MODE>(tab, g);
  for (int i = threadIdx.x; i < img_words; i += blockDim.x) img[i] = 0u;
  __syncthreads();

  const int ox = sx * T, oy = sy * T;

  // Stage alive & member bits of every member tile row.  Consecutive threads
  // take consecutive 16-byte pieces of a row, so a warp instruction reads
  // whole 32-byte sectors; each thread issues all its loads first.
  const int total_l = g.slots << LOG_LQ;
  for (int base = threadIdx.x; base < total_l; base += blockDim.x * kIPT) {
    uint32_t bits[kIPT];
    int word[kIPT];
#pragma unroll
    for (int u = 0; u < kIPT; ++u) {
      const int it = base + u * (int)blockDim.x;
      word[u] = -1;
      if (it < total_l) {
        const uint32_t e = tab[it >> LOG_LQ];
        if (e != kNoTile) {
          const int c = it & ((1 << LOG_LQ) - 1);
          const int lx0 = (int)(e & 0xffffu) * RHO + (c & (RHO / WL - 1)) * WL;
          const int ly = (int)(e >> 16) * RHO + c / (RHO / WL);
          const int gx0 = ox + lx0, gy = oy + ly;
          bits[u] = load_alive_bits<WL>(in + (size_t)gy * n + gx0) & chunk_members<WL>(gx0, gy, n);
          // half-word index for 16-cell chunks, else word index and bit shift
          word[u] = WL == 16 ? 2 * ((ly + 1) * wpr + ((lx0 + 32) >> 5)) + ((lx0 >> 4) & 1)
                             : ((ly + 1) * wpr + ((lx0 + 32) >> 5)) * 32 + (lx0 & 31);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kIPT; ++u) {
      if (word[u] < 0) continue;
      if (WL == 16 && T >= 32) {
        // exclusive half-word (ring bits live in other words when T >= 32)
        reinterpret_cast<uint16_t*>(img)[word[u]] = (uint16_t)bits[u];
      } else if (WL == 16) {
        if (bits[u]) atomicOr(img + (word[u] >> 1), bits[u] << (16 * (word[u] & 1)));
      } else if (bits[u]) {
        atomicOr(img + (word[u] >> 5), bits[u] << (word[u] & 31));
      }
    }
  }
  // Stage: ring cells that are members next to a member of the super-tile.
  for (int it = threadIdx.x; it < 4 * T + 4; it += blockDim.x) {
    int lx, ly;
    ring_cell(it, T, lx, ly);
    const int gx = ox + lx, gy = oy + ly;
    if (!is_member(gx, gy, n) || !ring_needed(lx, ly, gx, gy, T, n)) continue;
    if (in[(size_t)gy * n + gx] != 0)
      atomicOr(img + (ly + 1) * wpr + ((lx + 32) >> 5), 1u << ((lx + 32) & 31));
  }
  __syncthreads();

  // Update every member tile row (one row per thread).
  const int total = g.slots << LOG_RHO;
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const uint32_t e = tab[it >> LOG_RHO];
    // With rho = 32 a warp's 32 consecutive rows are one tile, so this exit and
    // the shuffles below are warp-uniform.
    if (e == kNoTile) continue;
    const int lx0 = (int)(e & 0xffffu) * RHO;
    const int ly = (int)(e >> 16) * RHO + (it & (RHO - 1));
    const int gx0 = ox + lx0, gy = oy + ly;
    const uint32_t* row = img + ly * wpr;  // image row ly holds cell row ly - 1
    const uint64_t up = bit_window(row, lx0);
    const uint64_t mid = bit_window(row + wpr, lx0);
    const uint64_t dn = bit_window(row + 2 * wpr, lx0);
    const uint32_t next = life_rule(up, mid, dn) & chunk_members<WC>(gx0, gy, n);
    if constexpr (RHO == 32) {
      // Lanes 2r and 2r+1 store the two 16-byte halves of tile row r (then
      // r + 16), so each store instruction writes whole sectors.
      const int lane = threadIdx.x & 31;
      const int h = lane & 1;
      uint8_t* base = out + (size_t)(gy - (it & 31)) * n + gx0 + 16 * h;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int r = (lane >> 1) + 16 * j;
        const uint32_t b = __shfl_sync(0xffffffffu, next, r);
        store_state_bytes<16>(base + (size_t)r * n, b >> (16 * h), 1u);
      }
    } else {
      store_state_bytes<WC>(out + (size_t)gy * n + gx0, next, 1u);
    }
  }
}

template <int MODE, int LOG_RHO>
cudaError_t go(const Launch& L, const uint8_t* in, uint8_t* out, cudaStream_t s) {
  auto* k = ca_kernel<MODE, LOG_RHO>;
  cudaError_t e = allow_smem((const void*)k, L.smem);
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, L.smem, s>>>(in, out, L.geo);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t by_rho(int log_rho, const Launch& L, const uint8_t* in, uint8_t* out, cudaStream_t s) {
  switch (log_rho) {
    case 0: return go<MODE, 0>(L, in, out, s);
    case 1: return go<MODE, 1>(L, in, out, s);
    case 2: return go<MODE, 2>(L, in, out, s);
    case 3: return go<MODE, 3>(L, in, out, s);
    case 4: return go<MODE, 4>(L, in, out, s);
    case 5: return go<MODE, 5>(L, in, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_ca(int mode, int log_rho, const Launch& L, const uint8_t* in, uint8_t* out,
                      cudaStream_t s) {
  return mode == kLambda ? by_rho<kLambda>(log_rho, L, in, out, s) : by_rho<kBB>(log_rho, L, in, out, s);
}

}  // namespace fractal
