// Global reduce (RD) of Sec. 6.2 for float32 fields, one 8 x 8 block of the
// gasket per thread.
//
// Launch: a CTA takes a member super-tile of 2^L x 2^L blocks.  lambda mode:
// the CTA's super-tile by lambda(omega) (Theorem 1) and its 3^L member blocks
// by lambda again (Sec. 5.1), L = 5 (243 blocks, 256 threads).  BB mode: the
// bounding-box grid of super-tiles, non-member ones exiting at once, and
// inside, the 4^L block slots by the identity, non-member ones idle (the
// plain method at both levels), L = 4 (256 slots).  Each thread reads the 12
// 16-byte chunks that hold its block's members (whole 32-byte rows where a
// row has members in both halves): 192 bytes in flight per thread.
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
