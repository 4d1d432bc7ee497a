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

// Image pitch (floats): T + 2M, padded so that consecutive rows start in
// different 32-byte bank groups (pitch mod 32 floats is 8 or 24); with 4
// consecutive rows per 8-lane phase of 128-bit accesses, no bank conflicts.
__host__ __device__ inline int fused_pitch(int T, int M) {
  int P = T + 2 * M;
  if ((P & 31) == 0 || (P & 31) == 16) P += 8;
  return P;
}

constexpr int kFusedChunksPerThread = 4;

template <int MODE, int LOG_RHO, int M>
__global__ void __launch_bounds__(512) diffusion_fused_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                              float a, int nsteps, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;  // >= 4
  constexpr int CT = kFusedChunksPerThread;
  extern __shared__ __align__(16) unsigned char sm[];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const int n = g.n, T = g.T;
  const int P = fused_pitch(T, M);
  const int img = (T + 2 * M + 2) * P;  // floats per image: rows plus a guard row above and below
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm);
  float* A = reinterpret_cast<float*>(sm + tab_words(g.tiles) * 4);
  float* B = A + img;
  // cell (lx, ly) of the image sits at (ly + M + 1) * P + lx + M; the guard
  // rows and the padding keep every neighbour read inside the image
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

  // This thread's chunks (4 cells of a row): their image offsets, and per
  // cell the coefficient c (a for a member, 0 otherwise) and the member
  // 4-degree d, so that a step is u' = u + c * (neighbour sum - d * u) for
  // every cell alike (a non-member holds 0 and stays 0).
  const int nt_chunks = g.tiles * RHO * (RHO / 4);
  const int chunks = nt_chunks + fused_box_chunks<M>();
  int off[CT];
  uint32_t mk[CT];  // member bits of the chunk's 4 cells
  float cf[CT][4], dg[CT][4];
#pragma unroll
  for (int k = 0; k < CT; ++k) {
    const int it = threadIdx.x + k * (int)blockDim.x;
    off[k] = -1;
    mk[k] = 0u;
    if (it >= chunks) continue;
    int lx, ly;
    fused_chunk<RHO, M>(it, nt_chunks, tab, T, lx, ly);
    const int gx0 = ox + lx, gy = oy + ly;
    off[k] = (ly + M + 1) * P + lx + M;
    if ((unsigned)gy < (unsigned)n && (unsigned)gx0 < (unsigned)n)
      cp_async16(A + off[k], in + (size_t)gy * n + gx0);
    // membership of the chunk's row and its neighbours, as bit masks (box
    // chunks may lie left of or beyond the array: no members there)
    const bool inx = (unsigned)gx0 < (unsigned)n;
    const uint32_t mc = inx ? chunk_members<4>(gx0, gy, n) : 0u;
    const uint32_t mu = inx ? chunk_members<4>(gx0, gy - 1, n) : 0u;
    const uint32_t md = inx ? chunk_members<4>(gx0, gy + 1, n) : 0u;
    const uint32_t ml = is_member(gx0 - 1, gy, n) ? 1u : 0u;
    const uint32_t mr = is_member(gx0 + 4, gy, n) ? 1u : 0u;
    const uint32_t row = ml | (mc << 1) | (mr << 5);  // bit j+1 = cell j of the chunk
    mk[k] = mc;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t deg = ((mu >> i) & 1u) + ((md >> i) & 1u) + ((row >> i) & 1u) + ((row >> (i + 2)) & 1u);
      const bool mem = (mc >> i) & 1u;
      cf[k][i] = mem ? a : 0.0f;
      dg[k][i] = mem ? (float)deg : 0.0f;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // non-member cells of staged chunks -> 0, so that neighbour sums need no masks
#pragma unroll
  for (int k = 0; k < CT; ++k) {
    if (off[k] < 0) continue;
    float4 v = *reinterpret_cast<const float4*>(A + off[k]);
    v.x = (mk[k] & 1u) ? v.x : 0.f;
    v.y = (mk[k] & 2u) ? v.y : 0.f;
    v.z = (mk[k] & 4u) ? v.z : 0.f;
    v.w = (mk[k] & 8u) ? v.w : 0.f;
    *reinterpret_cast<float4*>(A + off[k]) = v;
  }
  __syncthreads();

  // nsteps updates A -> B -> A ...
  for (int t = 0; t < nsteps; ++t) {
#pragma unroll
    for (int k = 0; k < CT; ++k) {
      if (off[k] < 0) continue;
      const float* p = A + off[k];
      const float4 c = *reinterpret_cast<const float4*>(p);
      const float4 u = *reinterpret_cast<const float4*>(p - P);
      const float4 d = *reinterpret_cast<const float4*>(p + P);
      const float l = p[-1], r = p[4];
      float4 o;
      o.x = fmaf(cf[k][0], fmaf(-dg[k][0], c.x, (u.x + d.x) + (l + c.y)), c.x);
      o.y = fmaf(cf[k][1], fmaf(-dg[k][1], c.y, (u.y + d.y) + (c.x + c.z)), c.y);
      o.z = fmaf(cf[k][2], fmaf(-dg[k][2], c.z, (u.z + d.z) + (c.y + c.w)), c.z);
      o.w = fmaf(cf[k][3], fmaf(-dg[k][3], c.w, (u.w + d.w) + (c.z + r)), c.w);
      *reinterpret_cast<float4*>(B + off[k]) = o;
    }
    __syncthreads();
    float* tmp = A;
    A = B;
    B = tmp;
  }

  // write back the member tiles (the first nt_chunks chunks)
#pragma unroll
  for (int k = 0; k < CT; ++k) {
    const int it = threadIdx.x + k * (int)blockDim.x;
    if (off[k] < 0 || it >= nt_chunks) continue;
    const int lx = off[k] % P - M, ly = off[k] / P - M - 1;
    *reinterpret_cast<float4*>(out + (size_t)(oy + ly) * n + ox + lx) = *reinterpret_cast<const float4*>(A + off[k]);
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
  const int P = fused_pitch(g.T, margin);
  return tab_words(g.tiles) * 4 + 2 * (g.T + 2 * margin + 2) * P * 4;
}

// Threads of a fused launch: every chunk owned by one thread, at most
// kFusedChunksPerThread each; 0 if that needs more than 512 threads.
int fused_threads(const Geo& g, int rho, int margin) {
  const int chunks = g.tiles * rho * (rho / 4) + (margin / 4) * 6 * margin;
  int t = ((chunks + kFusedChunksPerThread - 1) / kFusedChunksPerThread + 31) / 32 * 32;
  if (t < 32) t = 32;
  return t > 512 ? 0 : t;
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
