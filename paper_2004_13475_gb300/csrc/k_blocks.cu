// Single write (SW) and global reduce (RD) of Sec. 6.2 for float32 fields,
// one 8 x 8 block of the gasket per thread.
//
// Launch: a CTA takes a member super-tile of 2^L x 2^L blocks.  lambda mode:
// the CTA's super-tile by lambda(omega) (Theorem 1) and its 3^L member blocks
// by lambda again (Sec. 5.1), L = 5 (243 blocks, 256 threads).  BB mode: the
// bounding-box grid of super-tiles, non-member ones exiting at once, and
// inside, the 4^L block slots by the identity, non-member ones idle (the
// plain method at both levels), L = 4 (256 slots).  Each thread moves whole
// 32-byte rows: 12 16-byte chunks hold its block's members; SW also writes the
// zeros of the non-member cells of member tiles (rho >= 8), so its writes
// cover whole sectors.
#include "blocks.cuh"
#include "launch.h"

namespace fractal {
namespace {

constexpr int kBlkThreads = 256;

// This thread's member block of super-tile (sx, sy); false if it has none.
template <int MODE>
__device__ __forceinline__ bool blk_of_thread(int sx, int sy, int L, int& GX, int& GY) {
  const int t = threadIdx.x;
  int bx, by;
  if (MODE == kLambda) {
    int nb = 1, lw = 1;
    for (int i = 0; i < L; ++i) nb *= 3;
    for (int i = 0; i < (L + 1) / 2; ++i) lw *= 3;
    if (t >= nb) return false;
    lambda_scalar((uint32_t)(t % lw), (uint32_t)(t / lw), L, bx, by);
  } else {
    const int side = 1 << L;
    if (t >= side * side) return false;
    bx = t & (side - 1);
    by = t >> L;
    if (bx & by) return false;
  }
  GX = (sx << L) + bx;
  GY = (sy << L) + by;
  return true;
}

template <int MODE>
__global__ void __launch_bounds__(kBlkThreads) sw_blocks_kernel(float* __restrict__ out, float value, Geo g, int L,
                                                                int log_rho) {
  int sx, sy, GX, GY;
  if (!cta_supertile<MODE>(g, sx, sy) || !blk_of_thread<MODE>(sx, sy, L, GX, GY)) return;
  const int n = g.n;
  float* o = out + (size_t)GY * kB * n + (size_t)GX * kB;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    *reinterpret_cast<float4*>(o + (size_t)j * n) =
        make_float4(value, amem(1, j) ? value : 0.f, amem(2, j) ? value : 0.f, amem(3, j) ? value : 0.f);
    if (j < 4)
      *reinterpret_cast<float4*>(o + (size_t)j * n + 4) =
          make_float4(value, amem(5, j) ? value : 0.f, amem(6, j) ? value : 0.f, amem(7, j) ? value : 0.f);
    else if (log_rho >= 3)
      *reinterpret_cast<float4*>(o + (size_t)j * n + 4) = z;  // lower right quarter: non-members of the tile
  }
  if (log_rho >= 4) {
    // non-member blocks right of this one in its rho-tile row, up to the next member block
    const int bpt = 1 << (log_rho - 3);
    const int tx = GX & (bpt - 1), ty = GY & (bpt - 1);
    for (int q = tx + 1; q < bpt && (q & ty) != 0; ++q) {
      float* p = o + (size_t)(q - tx) * kB;
      for (int j = 0; j < kB; ++j) {
        *reinterpret_cast<float4*>(p + (size_t)j * n) = z;
        *reinterpret_cast<float4*>(p + (size_t)j * n + 4) = z;
      }
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(kBlkThreads) reduce_blocks_kernel(const float* __restrict__ in,
                                                                    double* __restrict__ partials, Geo g, int L) {
  __shared__ double red[32];
  int GX = 0, GY = 0;
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {  // BB: a super-tile off the gasket
    if (threadIdx.x == 0) partials[cta_id()] = 0.0;
    return;
  }
  double acc = 0.0;
  if (blk_of_thread<MODE>(sx, sy, L, GX, GY)) {
    float v[kB * kB];
    load_block(v, in + (size_t)GY * kB * g.n + (size_t)GX * kB, g.n);
    // FP32 within a row (at most 8 members), FP64 over the rows
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      float r = v[j * kB];
#pragma unroll
      for (int i = 1; i < kB; ++i)
        if (amem(i, j)) r += v[j * kB + i];
      acc += (double)r;
    }
  }
  const double s = block_sum<double>(acc, red);
  if (threadIdx.x == 0) partials[cta_id()] = s;
}

}  // namespace

// Super-tile levels of these kernels: 5 (lambda) or 4 (BB) block levels, at
// most the array's k - 3.
bool blocks_geometry(int k, int mode, Launch& L, int& levels) {
  if (k < 3) return false;
  const int want = mode == kLambda ? 5 : 4;
  levels = k - 3 < want ? k - 3 : want;
  if (!supertile_grid(k, 3, mode, levels, L)) return false;
  L.threads = kBlkThreads;
  L.smem = 0;
  return true;
}

cudaError_t launch_sw_blocks(int mode, int log_rho, const Launch& L, int levels, float* out, float value,
                             cudaStream_t s) {
  if (mode == kLambda)
    sw_blocks_kernel<kLambda><<<L.grid, L.threads, 0, s>>>(out, value, L.geo, levels, log_rho);
  else
    sw_blocks_kernel<kBB><<<L.grid, L.threads, 0, s>>>(out, value, L.geo, levels, log_rho);
  return cudaGetLastError();
}

cudaError_t launch_reduce_blocks(int mode, const Launch& L, int levels, const float* in, double* partials,
                                 double* dev_out, cudaStream_t s) {
  if (mode == kLambda)
    reduce_blocks_kernel<kLambda><<<L.grid, L.threads, 0, s>>>(in, partials, L.geo, levels);
  else
    reduce_blocks_kernel<kBB><<<L.grid, L.threads, 0, s>>>(in, partials, L.geo, levels);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_final_sum(1, partials, (int64_t)L.grid.x * L.grid.y, dev_out, s);
}

}  // namespace fractal
