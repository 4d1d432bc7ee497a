// The block-space map lambda(omega) for any fractal of the NBB family
// (Sec. 3.1, Theorem 1, Lemma 2), and the single write of Sec. 6.2 on such a
// fractal with one CTA per tile (the paper's block-per-tile setting), by the
// lambda launch or the bounding-box (BB) launch.
//
// An NBB fractal is given by its step: k cells (dx, dy) of an s x s grid, in
// the order that numbers the replicas (the hash H of Theorem 1).  A cell of
// the level-r fractal is a member iff each of its r base-s digit pairs is a
// step cell; lambda takes block omega = (wx, wy) of the packed
// k^ceil(r/2) x k^floor(r/2) grid to sum_mu H[beta_mu] s^(mu - 1), where
// beta_mu is the next base-k digit of wx (odd mu) or wy (even mu).
#include <cstdint>

#include <cuda_runtime.h>

#include "fractal.h"

namespace {

// The step in the kernels' parameter space: the cells in numbering order,
// four bits each (x | y << 2, s <= 4: at most 16 cells), the s x s
// membership bits (bit dy * s + dx), and kmagic = ceil(2^32 / k) (0 for
// k = 1), with which floor(w / k) = umulhi(w, kmagic) for every w < 2^32 / k
// (the error w * (kmagic - 2^32 / k) / 2^32 stays below 1 / k), so for every
// block coordinate here (below 2^28: the grids are at most 2^20 wide).
struct NbbStep {
  int s, k;
  uint32_t mask;
  uint32_t kmagic;
  uint64_t cells;
};

// lambda(omega) at level r (Theorem 1): the replica offsets of each level
// from the base-k digits of wx and wy, alternately, scaled by s^(mu - 1).
template <int S>
__device__ __forceinline__ void nbb_lambda(uint32_t wx, uint32_t wy, int r, const NbbStep& st, uint32_t& bx,
                                           uint32_t& by) {
  const uint32_t k = (uint32_t)st.k;
  uint32_t px = 1, x = 0, y = 0;
  for (int mu = 1; mu <= r; ++mu) {
    uint32_t d;
    if (mu & 1) {
      const uint32_t q = __umulhi(wx, st.kmagic);
      d = wx - q * k;
      wx = q;
    } else {
      const uint32_t q = __umulhi(wy, st.kmagic);
      d = wy - q * k;
      wy = q;
    }
    const uint32_t c = (uint32_t)(st.cells >> (4 * d)) & 15u;
    x += (c & 3u) * px;
    y += (c >> 2) * px;
    px *= S;
  }
  bx = x;
  by = y;
}

// (x, y) is a member of the level-levels fractal iff every base-S digit pair
// is a step cell.
template <int S>
__device__ __forceinline__ bool nbb_member(uint32_t x, uint32_t y, int levels, uint32_t mask) {
  bool ok = true;
  for (int i = 0; i < levels; ++i) {
    ok &= ((mask >> ((y % S) * S + (x % S))) & 1u) != 0;
    x /= S;
    y /= S;
  }
  return ok;
}

template <int S>
__global__ void __launch_bounds__(256) nbb_map_kernel(NbbStep st, int r, uint32_t W, int64_t total,
                                                      int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bx, by;
    nbb_lambda<S>((uint32_t)(i % W), (uint32_t)(i / W), r, st, bx, by);
    reinterpret_cast<int2*>(out)[i] = make_int2((int)bx, (int)by);
  }
}

// One CTA of t x t threads per tile (t = S^j), one thread per cell: value at
// the tile's members, 0 at its other cells.  MODE 0: the CTA's tile by
// lambda over the packed grid; MODE 1: the CTA's tile is (blockIdx.x,
// blockIdx.y) of the whole n_b x n_b grid, and CTAs on non-member tiles
// return at once (the BB launch).
template <int S, int MODE>
__global__ void nbb_write_kernel(NbbStep st, int rb, int j, int64_t n, float value, float* __restrict__ buf) {
  uint32_t bx, by;
  if (MODE == 0) {
    nbb_lambda<S>(blockIdx.x, blockIdx.y, rb, st, bx, by);
  } else {
    bx = blockIdx.x;
    by = blockIdx.y;
    if (!nbb_member<S>(bx, by, rb, st.mask)) return;
  }
  const int64_t x = (int64_t)bx * blockDim.x + threadIdx.x, y = (int64_t)by * blockDim.y + threadIdx.y;
  buf[y * n + x] = nbb_member<S>(threadIdx.x, threadIdx.y, j, st.mask) ? value : 0.f;
}

// One CTA per super-tile of k^m member tiles (this library's CTA shape, the
// further unrolling of Sec. 5.1): MODE 0: the super-tile by lambda over the
// packed grid of level rb - m and its tiles by lambda again at level m;
// MODE 1: the super-tile (blockIdx.x, blockIdx.y) of the whole grid, left at
// once when it is not a member, and its s^m x s^m tiles, the non-member ones
// skipped.  The CTA's threads stride over tile cells in tile order, so a
// warp's stores run along the rows of one or two tiles.
template <int S, int MODE>
__global__ void __launch_bounds__(256) nbb_write_tiles_kernel(NbbStep st, int rb, int j, int m, int t, int64_t n,
                                                               float value, float* __restrict__ buf) {
  extern __shared__ uint32_t toff[];  // tile offsets inside the super-tile: x | y << 16
  uint32_t sx, sy;
  int ntiles;
  if (MODE == 0) {
    nbb_lambda<S>(blockIdx.x, blockIdx.y, rb - m, st, sx, sy);
    ntiles = 1;
    for (int i = 0; i < m; ++i) ntiles *= st.k;
    uint32_t W = 1;
    for (int i = 0; i < (m + 1) / 2; ++i) W *= (uint32_t)st.k;
    for (int q = threadIdx.x; q < ntiles; q += blockDim.x) {
      uint32_t ox, oy;
      nbb_lambda<S>((uint32_t)q % W, (uint32_t)q / W, m, st, ox, oy);
      toff[q] = ox | oy << 16;
    }
  } else {
    sx = blockIdx.x;
    sy = blockIdx.y;
    if (!nbb_member<S>(sx, sy, rb - m, st.mask)) return;
    int side = 1;
    for (int i = 0; i < m; ++i) side *= S;
    ntiles = side * side;
    for (int q = threadIdx.x; q < ntiles; q += blockDim.x) {
      const uint32_t ox = (uint32_t)(q % side), oy = (uint32_t)(q / side);
      toff[q] = nbb_member<S>(ox, oy, m, st.mask) ? (ox | oy << 16) : 0xffffffffu;
    }
  }
  __syncthreads();
  int sm = 1;
  for (int i = 0; i < m; ++i) sm *= S;
  const int64_t X0 = (int64_t)sx * sm * t, Y0 = (int64_t)sy * sm * t;
  const int cells = t * t;
  for (int i = threadIdx.x; i < ntiles * cells; i += blockDim.x) {
    const int q = i / cells, c = i - q * cells;
    const uint32_t e = toff[q];
    if (MODE == 1 && e == 0xffffffffu) continue;
    const int cx = c % t, cy = c / t;
    const int64_t x = X0 + (int64_t)(e & 0xffffu) * t + cx, y = Y0 + (int64_t)(e >> 16) * t + cy;
    buf[y * n + x] = nbb_member<S>((uint32_t)cx, (uint32_t)cy, j, st.mask) ? value : 0.f;
  }
}

// One B3/S23 step of the CA test (Sec. 6.2) on a tile of t x t cells per
// CTA of t x t threads (the paper's setting), tile by lambda (MODE 0) or by
// identity over the whole grid with non-member tiles returning (MODE 1):
// the tile and its one-cell halo are staged in shared memory as
// "alive and member" (cells outside the array count as dead), then each
// thread counts its eight neighbours.  Member cells get the rule, the tile's
// other cells 0.
template <int S, int MODE>
__global__ void nbb_ca_kernel(NbbStep st, int rb, int j, int64_t n, const uint8_t* __restrict__ in,
                              uint8_t* __restrict__ out) {
  extern __shared__ uint8_t halo[];
  uint32_t bx, by;
  if (MODE == 0) {
    nbb_lambda<S>(blockIdx.x, blockIdx.y, rb, st, bx, by);
  } else {
    bx = blockIdx.x;
    by = blockIdx.y;
    if (!nbb_member<S>(bx, by, rb, st.mask)) return;
  }
  const int t = blockDim.x, h = t + 2, levels = rb + j;
  const int tid = threadIdx.y * t + threadIdx.x;
  const int64_t x0 = (int64_t)bx * t - 1, y0 = (int64_t)by * t - 1;
  for (int i = tid; i < h * h; i += t * t) {
    const int64_t gx = x0 + i % h, gy = y0 + i / h;
    uint8_t v = 0;
    if (gx >= 0 && gy >= 0 && gx < n && gy < n && nbb_member<S>((uint32_t)gx, (uint32_t)gy, levels, st.mask))
      v = in[gy * n + gx] != 0;
    halo[i] = v;
  }
  __syncthreads();
  const int cx = threadIdx.x + 1, cy = threadIdx.y + 1;
  int c = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
      if (dx || dy) c += halo[(cy + dy) * h + cx + dx];
  const bool me = halo[cy * h + cx] != 0;
  const bool alive = nbb_member<S>(threadIdx.x, threadIdx.y, j, st.mask) && (c == 3 || (me && c == 2));
  out[(y0 + cy) * n + x0 + cx] = alive ? 1 : 0;
}

// Block-wide FP64 sum in a fixed order (warp trees over the linear thread
// index, then the first warp over the warps); the result in thread 0.
__device__ __forceinline__ double nbb_block_sum(double v) {
  __shared__ double red[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthreads = blockDim.x * blockDim.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (tid < 32) {
    t = tid < (nthreads + 31) / 32 ? red[tid] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// The reduce test (Sec. 6.2 RD) on a tile per CTA: thread i < t * t takes
// cell (i mod t, i div t) if it is a member, and the CTA's FP64 sum goes to
// its partial (0 for a BB CTA on a non-member tile).  The CTA is one
// dimension of t * t threads rounded up to whole warps (the warp trees use
// full masks), the threads beyond t * t idle.
template <int S, int MODE>
__global__ void nbb_reduce_kernel(NbbStep st, int rb, int j, int t, int64_t n, const float* __restrict__ in,
                                  double* __restrict__ partials) {
  uint32_t bx, by;
  const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  const int tid = threadIdx.x;
  bool tile = true;
  if (MODE == 0) {
    nbb_lambda<S>(blockIdx.x, blockIdx.y, rb, st, bx, by);
  } else {
    bx = blockIdx.x;
    by = blockIdx.y;
    tile = nbb_member<S>(bx, by, rb, st.mask);
  }
  double v = 0.0;
  if (tile && tid < t * t) {
    const int cx = tid % t, cy = tid / t;
    if (nbb_member<S>((uint32_t)cx, (uint32_t)cy, j, st.mask))
      v = (double)in[((int64_t)by * t + cy) * n + (int64_t)bx * t + cx];
  }
  const double sum = nbb_block_sum(v);
  if (tid == 0) partials[cta] = sum;
}

// Sum of `count` partials in a fixed order, one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) nbb_final_sum_kernel(const double* __restrict__ partials, int64_t count,
                                                             double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  const double s = nbb_block_sum(acc);
  if (threadIdx.x == 0) *out = s;
}

// One explicit diffusion step (FP32) on a tile of t x t cells per CTA of
// t x t threads, tile by lambda (MODE 0) or by identity with non-member
// tiles returning (MODE 1): the tile and its one-cell halo are staged in
// shared memory with a membership flag, non-members (and cells outside the
// array) as 0 whatever they hold; each member then takes
// fmaf(a, fmaf(-degree, u, sum), u), the sum and degree over its member
// 4-neighbours in the order up, left, right, down; the tile's other cells
// get 0.
template <int S, int MODE>
__global__ void nbb_diffusion_kernel(NbbStep st, int rb, int j, int64_t n, float a, const float* __restrict__ in,
                                     float* __restrict__ out) {
  extern __shared__ float hv[];  // (t + 2)^2 values, then (t + 2)^2 membership flags as floats (1 / 0)
  uint32_t bx, by;
  if (MODE == 0) {
    nbb_lambda<S>(blockIdx.x, blockIdx.y, rb, st, bx, by);
  } else {
    bx = blockIdx.x;
    by = blockIdx.y;
    if (!nbb_member<S>(bx, by, rb, st.mask)) return;
  }
  const int t = blockDim.x, h = t + 2, levels = rb + j;
  float* hm = hv + h * h;
  const int tid = threadIdx.y * t + threadIdx.x;
  const int64_t x0 = (int64_t)bx * t - 1, y0 = (int64_t)by * t - 1;
  for (int i = tid; i < h * h; i += t * t) {
    const int64_t gx = x0 + i % h, gy = y0 + i / h;
    const bool m = gx >= 0 && gy >= 0 && gx < n && gy < n && nbb_member<S>((uint32_t)gx, (uint32_t)gy, levels, st.mask);
    hv[i] = m ? in[gy * n + gx] : 0.f;
    hm[i] = m ? 1.f : 0.f;
  }
  __syncthreads();
  const int c = (threadIdx.y + 1) * h + threadIdx.x + 1;
  float r = 0.f;
  if (hm[c] != 0.f) {
    const float u = hv[c];
    const int nbs[4] = {c - h, c - 1, c + 1, c + h};
    float sum = 0.f, deg = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sum += hv[nbs[q]];  // 0 at non-members
      deg += hm[nbs[q]];
    }
    r = fmaf(a, fmaf(-deg, u, sum), u);
  }
  out[(y0 + threadIdx.y + 1) * n + x0 + threadIdx.x + 1] = r;
}

int64_t ipow64(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

// Validates the step and fills `st`; FRACTAL_EINVAL if s is not 2..4, k not
// 1..s*s, a cell outside the s x s grid or listed twice.
int make_step(int s, int k, const int32_t* cells, NbbStep& st) {
  if (s < 2 || s > 4 || k < 1 || k > s * s || !cells) return FRACTAL_EINVAL;
  st = NbbStep{};
  st.s = s;
  st.k = k;
  st.kmagic = k > 1 ? (uint32_t)(((uint64_t)1 << 32) / (uint64_t)k + ((((uint64_t)1 << 32) % (uint64_t)k) ? 1 : 0)) : 0u;
  for (int i = 0; i < k; ++i) {
    const int x = cells[2 * i], y = cells[2 * i + 1];
    if (x < 0 || y < 0 || x >= s || y >= s) return FRACTAL_EINVAL;
    const uint32_t bit = 1u << (y * s + x);
    if (st.mask & bit) return FRACTAL_EINVAL;
    st.mask |= bit;
    st.cells |= (uint64_t)(x | y << 2) << (4 * i);
  }
  return FRACTAL_OK;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? FRACTAL_OK : FRACTAL_ECUDA; }

}  // namespace

extern "C" {

int fractal_nbb_map_blocks(int s, int k, const int32_t* cells_xy, int r, void* dev_xy_, void* stream) {
  int32_t* dev_xy = static_cast<int32_t*>(dev_xy_);
  NbbStep st;
  if (make_step(s, k, cells_xy, st) != FRACTAL_OK || r < 0 || !dev_xy ||
      (reinterpret_cast<uintptr_t>(dev_xy) & 7u) != 0)
    return FRACTAL_EINVAL;
  if (r > 0 && (ipow64(k, r) > (int64_t)0x7fffffff || ipow64(s, r) > (int64_t)0x7fffffff)) return FRACTAL_EINVAL;
  const int64_t total = ipow64(k, r);
  const uint32_t W = (uint32_t)ipow64(k, (r + 1) / 2);
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  cudaStream_t cs = (cudaStream_t)stream;
  switch (s) {
    case 2: nbb_map_kernel<2><<<(unsigned)blocks, 256, 0, cs>>>(st, r, W, total, dev_xy); break;
    case 3: nbb_map_kernel<3><<<(unsigned)blocks, 256, 0, cs>>>(st, r, W, total, dev_xy); break;
    default: nbb_map_kernel<4><<<(unsigned)blocks, 256, 0, cs>>>(st, r, W, total, dev_xy); break;
  }
  return status_of(cudaGetLastError());
}

int fractal_nbb_write(int s, int k, const int32_t* cells_xy, int r_b, int j, int cta_levels, int mode, float value,
                      float* dev_buf, void* stream) {
  NbbStep st;
  if (make_step(s, k, cells_xy, st) != FRACTAL_OK || r_b < 0 || j < 0 || !dev_buf ||
      (reinterpret_cast<uintptr_t>(dev_buf) & 3u) != 0 || (mode != FRACTAL_LAMBDA && mode != FRACTAL_BB) ||
      cta_levels < 0 || cta_levels > r_b)
    return FRACTAL_EINVAL;
  const int64_t t = ipow64(s, j);
  if (t > 32) return FRACTAL_EINVAL;  // a CTA holds the tile's t * t cells
  const int64_t nb = ipow64(s, r_b), n = nb * t;
  if (n > (int64_t)1 << 20) return FRACTAL_EINVAL;
  cudaStream_t cs = (cudaStream_t)stream;
  if (cta_levels > 0) {  // one CTA of 256 threads per super-tile of k^m member tiles
    const int m = cta_levels;
    const int64_t tiles = mode == FRACTAL_LAMBDA ? ipow64(k, m) : ipow64(s, 2 * m);
    if (tiles > 4096 || (uint32_t)(ipow64(s, m)) > 0xffffu) return FRACTAL_EINVAL;
    const int64_t W = ipow64(k, (r_b - m + 1) / 2), H = ipow64(k, (r_b - m) / 2), G = ipow64(s, r_b - m);
    dim3 grid;
    if (mode == FRACTAL_LAMBDA) {
      if (W > 0x7fffffff || H > 65535) return FRACTAL_EINVAL;
      grid = dim3((unsigned)W, (unsigned)H);
    } else {
      if (G > 65535) return FRACTAL_EINVAL;
      grid = dim3((unsigned)G, (unsigned)G);
    }
    const size_t smem = (size_t)tiles * 4;
    const bool lam = mode == FRACTAL_LAMBDA;
    const int ti = (int)t;
    switch (s) {
      case 2:
        if (lam) nbb_write_tiles_kernel<2, 0><<<grid, 256, smem, cs>>>(st, r_b, j, m, ti, n, value, dev_buf);
        else nbb_write_tiles_kernel<2, 1><<<grid, 256, smem, cs>>>(st, r_b, j, m, ti, n, value, dev_buf);
        break;
      case 3:
        if (lam) nbb_write_tiles_kernel<3, 0><<<grid, 256, smem, cs>>>(st, r_b, j, m, ti, n, value, dev_buf);
        else nbb_write_tiles_kernel<3, 1><<<grid, 256, smem, cs>>>(st, r_b, j, m, ti, n, value, dev_buf);
        break;
      default:
        if (lam) nbb_write_tiles_kernel<4, 0><<<grid, 256, smem, cs>>>(st, r_b, j, m, ti, n, value, dev_buf);
        else nbb_write_tiles_kernel<4, 1><<<grid, 256, smem, cs>>>(st, r_b, j, m, ti, n, value, dev_buf);
        break;
    }
    return status_of(cudaGetLastError());
  }
  const int64_t W = ipow64(k, (r_b + 1) / 2), H = ipow64(k, r_b / 2);
  dim3 grid;
  if (mode == FRACTAL_LAMBDA) {
    if (W > 0x7fffffff || H > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)W, (unsigned)H);
  } else {
    if (nb > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)nb, (unsigned)nb);
  }
  const dim3 block((unsigned)t, (unsigned)t);
  const bool lam = mode == FRACTAL_LAMBDA;
  switch (s) {
    case 2:
      if (lam) nbb_write_kernel<2, 0><<<grid, block, 0, cs>>>(st, r_b, j, n, value, dev_buf);
      else nbb_write_kernel<2, 1><<<grid, block, 0, cs>>>(st, r_b, j, n, value, dev_buf);
      break;
    case 3:
      if (lam) nbb_write_kernel<3, 0><<<grid, block, 0, cs>>>(st, r_b, j, n, value, dev_buf);
      else nbb_write_kernel<3, 1><<<grid, block, 0, cs>>>(st, r_b, j, n, value, dev_buf);
      break;
    default:
      if (lam) nbb_write_kernel<4, 0><<<grid, block, 0, cs>>>(st, r_b, j, n, value, dev_buf);
      else nbb_write_kernel<4, 1><<<grid, block, 0, cs>>>(st, r_b, j, n, value, dev_buf);
      break;
  }
  return status_of(cudaGetLastError());
}

int fractal_nbb_step_ca(int s, int k, const int32_t* cells_xy, int r_b, int j, int mode, uint8_t* dev_a,
                        uint8_t* dev_b, int steps, void* stream) {
  NbbStep st;
  if (make_step(s, k, cells_xy, st) != FRACTAL_OK || r_b < 0 || j < 0 || !dev_a || !dev_b || dev_a == dev_b ||
      steps < 0 || (mode != FRACTAL_LAMBDA && mode != FRACTAL_BB))
    return FRACTAL_EINVAL;
  const int64_t t = ipow64(s, j);
  if (t > 32) return FRACTAL_EINVAL;
  const int64_t nb = ipow64(s, r_b), n = nb * t;
  if (n > (int64_t)1 << 20) return FRACTAL_EINVAL;
  const int64_t W = ipow64(k, (r_b + 1) / 2), H = ipow64(k, r_b / 2);
  dim3 grid;
  if (mode == FRACTAL_LAMBDA) {
    if (W > 0x7fffffff || H > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)W, (unsigned)H);
  } else {
    if (nb > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)nb, (unsigned)nb);
  }
  const dim3 block((unsigned)t, (unsigned)t);
  const size_t smem = (size_t)(t + 2) * (t + 2);
  cudaStream_t cs = (cudaStream_t)stream;
  const bool lam = mode == FRACTAL_LAMBDA;
  for (int i = 0; i < steps; ++i) {
    const uint8_t* in = (i & 1) ? dev_b : dev_a;
    uint8_t* out = (i & 1) ? dev_a : dev_b;
    switch (s) {
      case 2:
        if (lam) nbb_ca_kernel<2, 0><<<grid, block, smem, cs>>>(st, r_b, j, n, in, out);
        else nbb_ca_kernel<2, 1><<<grid, block, smem, cs>>>(st, r_b, j, n, in, out);
        break;
      case 3:
        if (lam) nbb_ca_kernel<3, 0><<<grid, block, smem, cs>>>(st, r_b, j, n, in, out);
        else nbb_ca_kernel<3, 1><<<grid, block, smem, cs>>>(st, r_b, j, n, in, out);
        break;
      default:
        if (lam) nbb_ca_kernel<4, 0><<<grid, block, smem, cs>>>(st, r_b, j, n, in, out);
        else nbb_ca_kernel<4, 1><<<grid, block, smem, cs>>>(st, r_b, j, n, in, out);
        break;
    }
    const int e = status_of(cudaGetLastError());
    if (e != FRACTAL_OK) return e;
  }
  return FRACTAL_OK;
}

int fractal_nbb_reduce(int s, int k, const int32_t* cells_xy, int r_b, int j, int mode, const float* dev_buf,
                       double* dev_partials, int64_t partials_len, double* dev_out, void* stream) {
  NbbStep st;
  if (make_step(s, k, cells_xy, st) != FRACTAL_OK || r_b < 0 || j < 0 || !dev_buf || !dev_partials || !dev_out ||
      (mode != FRACTAL_LAMBDA && mode != FRACTAL_BB))
    return FRACTAL_EINVAL;
  const int64_t t = ipow64(s, j);
  if (t > 32) return FRACTAL_EINVAL;
  const int64_t nb = ipow64(s, r_b), n = nb * t;
  if (n > (int64_t)1 << 20) return FRACTAL_EINVAL;
  const int64_t W = ipow64(k, (r_b + 1) / 2), H = ipow64(k, r_b / 2);
  dim3 grid;
  int64_t ctas;
  if (mode == FRACTAL_LAMBDA) {
    if (W > 0x7fffffff || H > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)W, (unsigned)H);
    ctas = W * H;
  } else {
    if (nb > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)nb, (unsigned)nb);
    ctas = nb * nb;
  }
  if (partials_len < ctas) return FRACTAL_EINVAL;
  // t * t threads rounded up to whole warps
  const dim3 block((unsigned)((t * t + 31) / 32 * 32));
  cudaStream_t cs = (cudaStream_t)stream;
  const bool lam = mode == FRACTAL_LAMBDA;
  const int ti = (int)t;
  switch (s) {
    case 2:
      if (lam) nbb_reduce_kernel<2, 0><<<grid, block, 0, cs>>>(st, r_b, j, ti, n, dev_buf, dev_partials);
      else nbb_reduce_kernel<2, 1><<<grid, block, 0, cs>>>(st, r_b, j, ti, n, dev_buf, dev_partials);
      break;
    case 3:
      if (lam) nbb_reduce_kernel<3, 0><<<grid, block, 0, cs>>>(st, r_b, j, ti, n, dev_buf, dev_partials);
      else nbb_reduce_kernel<3, 1><<<grid, block, 0, cs>>>(st, r_b, j, ti, n, dev_buf, dev_partials);
      break;
    default:
      if (lam) nbb_reduce_kernel<4, 0><<<grid, block, 0, cs>>>(st, r_b, j, ti, n, dev_buf, dev_partials);
      else nbb_reduce_kernel<4, 1><<<grid, block, 0, cs>>>(st, r_b, j, ti, n, dev_buf, dev_partials);
      break;
  }
  int e = status_of(cudaGetLastError());
  if (e != FRACTAL_OK) return e;
  nbb_final_sum_kernel<<<1, 1024, 0, cs>>>(dev_partials, ctas, dev_out);
  return status_of(cudaGetLastError());
}

int fractal_nbb_step_diffusion(int s, int k, const int32_t* cells_xy, int r_b, int j, int mode, float* dev_a,
                               float* dev_b, float a, int steps, void* stream) {
  NbbStep st;
  if (make_step(s, k, cells_xy, st) != FRACTAL_OK || r_b < 0 || j < 0 || !dev_a || !dev_b || dev_a == dev_b ||
      steps < 0 || !(a == a) || (mode != FRACTAL_LAMBDA && mode != FRACTAL_BB) ||
      (reinterpret_cast<uintptr_t>(dev_a) & 3u) != 0 || (reinterpret_cast<uintptr_t>(dev_b) & 3u) != 0)
    return FRACTAL_EINVAL;
  const int64_t t = ipow64(s, j);
  if (t > 32) return FRACTAL_EINVAL;
  const int64_t nb = ipow64(s, r_b), n = nb * t;
  if (n > (int64_t)1 << 20) return FRACTAL_EINVAL;
  const int64_t W = ipow64(k, (r_b + 1) / 2), H = ipow64(k, r_b / 2);
  dim3 grid;
  if (mode == FRACTAL_LAMBDA) {
    if (W > 0x7fffffff || H > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)W, (unsigned)H);
  } else {
    if (nb > 65535) return FRACTAL_EINVAL;
    grid = dim3((unsigned)nb, (unsigned)nb);
  }
  const dim3 block((unsigned)t, (unsigned)t);
  const size_t smem = (size_t)2 * (t + 2) * (t + 2) * sizeof(float);
  cudaStream_t cs = (cudaStream_t)stream;
  const bool lam = mode == FRACTAL_LAMBDA;
  for (int i = 0; i < steps; ++i) {
    const float* in = (i & 1) ? dev_b : dev_a;
    float* out = (i & 1) ? dev_a : dev_b;
    switch (s) {
      case 2:
        if (lam) nbb_diffusion_kernel<2, 0><<<grid, block, smem, cs>>>(st, r_b, j, n, a, in, out);
        else nbb_diffusion_kernel<2, 1><<<grid, block, smem, cs>>>(st, r_b, j, n, a, in, out);
        break;
      case 3:
        if (lam) nbb_diffusion_kernel<3, 0><<<grid, block, smem, cs>>>(st, r_b, j, n, a, in, out);
        else nbb_diffusion_kernel<3, 1><<<grid, block, smem, cs>>>(st, r_b, j, n, a, in, out);
        break;
      default:
        if (lam) nbb_diffusion_kernel<4, 0><<<grid, block, smem, cs>>>(st, r_b, j, n, a, in, out);
        else nbb_diffusion_kernel<4, 1><<<grid, block, smem, cs>>>(st, r_b, j, n, a, in, out);
        break;
    }
    const int e = status_of(cudaGetLastError());
    if (e != FRACTAL_OK) return e;
  }
  return FRACTAL_OK;
}

}  // extern "C"
