// Temporally fused step kernels: one CTA advances its super-tile by up to
// MARGIN steps per launch, so each member tile is read and written once per
// launch instead of once per step.
//
// Why the halo stays tiny.  A member super-tile of side T (cells (x, y) in
// [0,T)^2 with x & y == 0, T a power of two) meets the rest of the gasket
// only near three contacts: left of (0,0), above (0,0), right of (T-1,0) and
// below (0,T-1).  For s <= T/2 every member cell outside the super-tile
// within distance s of one of its members lies in one of four margin boxes
// (super-tile coordinates, margin width M >= s):
//   left   [-M, 0) x [0, M)        top    [0, M) x [-M, 0)
//   right  [T, T+M) x [-M, M)      bottom [-M, M) x [T, T+M)
// (outside the super-tile, a member in row -i or column -i lies within i
// cells of the contact, and members of the right/bottom neighbours deeper
// than M rows from the contact are more than s cells from every member
// here).  The CTA stages its member tiles and these boxes in a shared-memory
// image with a margin of M cells, evolves every member cell of them for s
// steps (cells of the boxes whose neighbours were not staged go wrong from
// the box edge inwards, one cell per step, and never reach the super-tile),
// and writes back only the member tiles.
#include "launch.h"

namespace fractal {
namespace {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Chunks (4 consecutive cells of a row) the CTA updates: Q per member tile,
// then the margin boxes.  Returns super-tile coordinates of the first cell.
template <int RHO, int M>
__device__ __forceinline__ void fused_chunk(int it, int nt_chunks, const uint32_t* tab, int T, int& lx, int& ly) {
  constexpr int CPR = RHO / 4;  // chunks per tile row
  constexpr int Q = RHO * CPR;  // chunks per tile
  if (it < nt_chunks) {
    const int c = it / Q, q = it - c * Q;
    const uint32_t e = tab[c];
    lx = (int)(e & 0xffffu) * RHO + (q % CPR) * 4;
    ly = (int)(e >> 16) * RHO + q / CPR;
    return;
  }
  int b = it - nt_chunks;
  constexpr int W = M / 4;  // chunks per box row of width M
  // left: M rows x W
  if (b < M * W) { lx = -M + (b % W) * 4; ly = b / W; return; }
  b -= M * W;
  // top: M rows x W
  if (b < M * W) { lx = (b % W) * 4; ly = -M + b / W; return; }
  b -= M * W;
  // right: 2M rows x W
  if (b < 2 * M * W) { lx = T + (b % W) * 4; ly = -M + b / W; return; }
  b -= 2 * M * W;
  // bottom: M rows x 2W
  lx = -M + (b % (2 * W)) * 4;
  ly = T + b / (2 * W);
}

template <int M>
__host__ __device__ constexpr int fused_box_chunks() { return (M / 4) * (M + M + 2 * M + 2 * M); }

template <int MODE, int LOG_RHO, int M>
__global__ void __launch_bounds__(256) diffusion_fused_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                              float a, int nsteps, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;  // >= 4
  extern __shared__ __align__(16) unsigned char sm[];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const int n = g.n, T = g.T;
  const int P = T + 2 * M;            // image pitch (floats)
  const int img = (P + 2) * P;        // floats per image: P rows plus a guard row above and below
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm);
  float* A = reinterpret_cast<float*>(sm + tab_words(g.tiles) * 4);
  float* B = A + img;
  int8_t* D = reinterpret_cast<int8_t*>(B + img);  // per cell: member 4-degree, or -1 for a non-member
  // cell (lx, ly) of the image sits at (ly + M + 1) * P + lx + M; the guard
  // rows keep the neighbour reads of the outermost chunks inside the image
  const int ox = sx * T, oy = sy * T;

  // member tiles of the super-tile (further unrolling, or BB discard)
  for (int j = threadIdx.x; j < g.slots; j += blockDim.x) {
    int ux, uy;
    if (MODE == kLambda) {
      lambda_scalar((uint32_t)(j % g.lw), (uint32_t)(j / g.lw), g.m, ux, uy);
      tab[j] = (uint32_t)ux | ((uint32_t)uy << 16);
    } else {
      ux = j & ((1 << g.m) - 1);
      uy = j >> g.m;
      if ((ux & uy) == 0) {
        int rank = 0;
        for (int q = 0; q < j; ++q) rank += ((q & ((1 << g.m) - 1)) & (q >> g.m)) == 0;
        tab[rank] = (uint32_t)ux | ((uint32_t)uy << 16);
      }
    }
  }
  for (int i = threadIdx.x; i < 2 * img / 4; i += blockDim.x)
    reinterpret_cast<float4*>(A)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();

  const int nt_chunks = g.tiles * RHO * (RHO / 4);
  const int chunks = nt_chunks + fused_box_chunks<M>();
  // stage: async copies of every in-array chunk; degree table
  for (int it = threadIdx.x; it < chunks; it += blockDim.x) {
    int lx, ly;
    fused_chunk<RHO, M>(it, nt_chunks, tab, T, lx, ly);
    const int gx0 = ox + lx, gy = oy + ly;
    const int off = (ly + M + 1) * P + lx + M;
    if ((unsigned)gy < (unsigned)n && (unsigned)gx0 < (unsigned)n)
      cp_async16(A + off, in + (size_t)gy * n + gx0);
    uint32_t dw = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gx = gx0 + i;
      int d = -1;
      if (is_member(gx, gy, n))
        d = (int)is_member(gx, gy - 1, n) + (int)is_member(gx - 1, gy, n) + (int)is_member(gx + 1, gy, n) +
            (int)is_member(gx, gy + 1, n);
      dw |= (uint32_t)(uint8_t)(int8_t)d << (8 * i);
    }
    *reinterpret_cast<uint32_t*>(D + off - P) = dw;
  }
  cp_async_wait_all();
  __syncthreads();
  // non-member cells of staged chunks -> 0, so that neighbour sums need no masks
  for (int it = threadIdx.x; it < chunks; it += blockDim.x) {
    int lx, ly;
    fused_chunk<RHO, M>(it, nt_chunks, tab, T, lx, ly);
    const int off = (ly + M + 1) * P + lx + M;
    const uint32_t dw = *reinterpret_cast<const uint32_t*>(D + off - P);
    float4 v = *reinterpret_cast<const float4*>(A + off);
    v.x = (dw & 0x80u) ? 0.f : v.x;
    v.y = (dw & 0x8000u) ? 0.f : v.y;
    v.z = (dw & 0x800000u) ? 0.f : v.z;
    v.w = (dw & 0x80000000u) ? 0.f : v.w;
    *reinterpret_cast<float4*>(A + off) = v;
  }
  __syncthreads();

  // nsteps updates A -> B -> A ...:  u' = u + a * (sum of member neighbours - deg * u)
  for (int t = 0; t < nsteps; ++t) {
    for (int it = threadIdx.x; it < chunks; it += blockDim.x) {
      int lx, ly;
      fused_chunk<RHO, M>(it, nt_chunks, tab, T, lx, ly);
      const int off = (ly + M + 1) * P + lx + M;
      const float4 c = *reinterpret_cast<const float4*>(A + off);
      const float4 u = *reinterpret_cast<const float4*>(A + off - P);
      const float4 d = *reinterpret_cast<const float4*>(A + off + P);
      const float l = A[off - 1], r = A[off + 4];
      const uint32_t dw = *reinterpret_cast<const uint32_t*>(D + off - P);
      const float cv[4] = {c.x, c.y, c.z, c.w};
      const float nb[4] = {u.x + d.x + l + c.y, u.y + d.y + c.x + c.z, u.z + d.z + c.y + c.w, u.w + d.w + c.z + r};
      float res[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int deg = (int)(int8_t)(dw >> (8 * i));
        res[i] = deg >= 0 ? fmaf(a, fmaf(-(float)deg, cv[i], nb[i]), cv[i]) : 0.f;
      }
      *reinterpret_cast<float4*>(B + off) = make_float4(res[0], res[1], res[2], res[3]);
    }
    __syncthreads();
    float* tmp = A;
    A = B;
    B = tmp;
  }

  // write back the member tiles
  for (int it = threadIdx.x; it < nt_chunks; it += blockDim.x) {
    int lx, ly;
    fused_chunk<RHO, M>(it, nt_chunks, tab, T, lx, ly);
    const int off = (ly + M + 1) * P + lx + M;
    *reinterpret_cast<float4*>(out + (size_t)(oy + ly) * n + ox + lx) = *reinterpret_cast<const float4*>(A + off);
  }
}

template <int MODE, int LOG_RHO, int M>
cudaError_t go(const Launch& L, const float* in, float* out, float a, int nsteps, cudaStream_t s) {
  auto* k = diffusion_fused_kernel<MODE, LOG_RHO, M>;
  cudaError_t e = allow_smem((const void*)k, L.smem);
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, L.smem, s>>>(in, out, a, nsteps, L.geo);
  return cudaGetLastError();
}

template <int MODE, int M>
cudaError_t by_rho(int log_rho, const Launch& L, const float* in, float* out, float a, int nsteps, cudaStream_t s) {
  switch (log_rho) {
    case 2: return go<MODE, 2, M>(L, in, out, a, nsteps, s);
    case 3: return go<MODE, 3, M>(L, in, out, a, nsteps, s);
    case 4: return go<MODE, 4, M>(L, in, out, a, nsteps, s);
    case 5: return go<MODE, 5, M>(L, in, out, a, nsteps, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int fused_margin(int steps_per_launch) { return steps_per_launch <= 4 ? 4 : 8; }

int fused_smem_bytes(const Geo& g, int margin) {
  const int P = g.T + 2 * margin;
  return tab_words(g.tiles) * 4 + 2 * (P + 2) * P * 4 + P * P;
}

int fused_threads(const Geo& g, int rho, int margin) {
  const int chunks = g.tiles * rho * (rho / 4) + (margin / 4) * 6 * margin;
  int t = ((chunks + 1) / 2 + 31) / 32 * 32;
  return t < 32 ? 32 : (t > 256 ? 256 : t);
}

cudaError_t launch_diffusion_fused(int mode, int log_rho, int margin, const Launch& L, const float* in, float* out,
                                   float a, int nsteps, cudaStream_t s) {
  const int M = margin;
  if (nsteps < 1 || nsteps > M) return cudaErrorInvalidValue;
  if (mode == kLambda)
    return M == 4 ? by_rho<kLambda, 4>(log_rho, L, in, out, a, nsteps, s)
                  : by_rho<kLambda, 8>(log_rho, L, in, out, a, nsteps, s);
  return M == 4 ? by_rho<kBB, 4>(log_rho, L, in, out, a, nsteps, s) : by_rho<kBB, 8>(log_rho, L, in, out, a, nsteps, s);
}

}  // namespace fractal
