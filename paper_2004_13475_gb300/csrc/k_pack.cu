// Compact storage of the gasket through the block-space map: the member tiles
// of an n x n array packed one after another in lambda order (tile j is the
// tile lambda(omega_j), omega_j = (j mod W, j div W) of the packed grid,
// Theorem 1), and back.  A packed field holds 3^{r_b} rho^2 elements instead
// of n^2, the member tiles' sectors only; moving a field between host and
// device in this form moves no cell outside the member tiles.
//
// One thread per tile row: it maps its tile by lambda (per-thread form) and
// copies the row's rho elements with 16-byte (or narrower) accesses.
#include "launch.h"

namespace fractal {
namespace {

template <int VB>  // bytes per access
struct Vec;
template <> struct Vec<16> { using T = uint4; };
template <> struct Vec<8> { using T = uint2; };
template <> struct Vec<4> { using T = uint32_t; };
template <> struct Vec<2> { using T = uint16_t; };
template <> struct Vec<1> { using T = uint8_t; };

template <int VB, bool PACK>
__global__ void __launch_bounds__(256) pack_kernel(const unsigned char* __restrict__ src,
                                                   unsigned char* __restrict__ dst, int n, int rb, int w,
                                                   int rho, int elem, int64_t rows) {
  using T = typename Vec<VB>::T;
  const int row_bytes = rho * elem;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = r / rho;           // tile, in lambda order
    const int ty = (int)(r - j * rho);   // row of the tile
    int bx, by;
    lambda_scalar((uint32_t)(j % w), (uint32_t)(j / w), rb, bx, by);
    const size_t emb = ((size_t)by * rho + ty) * (size_t)n * elem + (size_t)bx * rho * elem;
    const size_t pk = (size_t)r * row_bytes;
    const T* s = reinterpret_cast<const T*>(src + (PACK ? emb : pk));
    T* d = reinterpret_cast<T*>(dst + (PACK ? pk : emb));
    for (int i = 0; i < row_bytes / VB; ++i) d[i] = s[i];
  }
}

template <bool PACK>
cudaError_t run(const void* src, void* dst, int n, int rb, int rho, int elem, cudaStream_t s) {
  const int w = [rb] {
    int v = 1;
    for (int i = 0; i < (rb + 1) / 2; ++i) v *= 3;
    return v;
  }();
  int64_t tiles = 1;
  for (int i = 0; i < rb; ++i) tiles *= 3;
  const int64_t rows = tiles * rho;
  int64_t blocks = (rows + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  const auto* a = static_cast<const unsigned char*>(src);
  auto* b = static_cast<unsigned char*>(dst);
  const int rb_bytes = rho * elem;
  if (rb_bytes % 16 == 0)
    pack_kernel<16, PACK><<<(unsigned)blocks, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  else if (rb_bytes % 8 == 0)
    pack_kernel<8, PACK><<<(unsigned)blocks, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  else if (rb_bytes % 4 == 0)
    pack_kernel<4, PACK><<<(unsigned)blocks, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  else if (rb_bytes % 2 == 0)
    pack_kernel<2, PACK><<<(unsigned)blocks, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  else
    pack_kernel<1, PACK><<<(unsigned)blocks, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack(const void* embedded, void* packed, int n, int rb, int rho, int elem, cudaStream_t s) {
  return run<true>(embedded, packed, n, rb, rho, elem, s);
}

cudaError_t launch_unpack(const void* packed, void* embedded, int n, int rb, int rho, int elem, cudaStream_t s) {
  return run<false>(packed, embedded, n, rb, rho, elem, s);
}

}  // namespace fractal
