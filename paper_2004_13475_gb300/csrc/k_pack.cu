// Compact storage of the gasket through the block-space map: the member tiles
// of an n x n array packed one after another in lambda order (tile j is the
// tile lambda(omega_j), omega_j = (j mod W, j div W) of the packed grid,
// Theorem 1), and back.  A packed field holds 3^{r_b} rho^2 elements instead
// of n^2, the member tiles' sectors only; moving a field between host and
// device in this form moves no cell outside the member tiles.
//
// Rows of 16 bytes or more: one thread per tile row; it maps its tile by
// lambda (per-thread form) and copies the row with 16-byte (or narrower)
// accesses.  Narrower rows (rho * elem < 16) with the packed side in pinned
// host memory: one thread per 16 bytes of the packed side, i.e. 16 / (rho *
// elem) consecutive rows, so that the host link sees whole 16-byte accesses.
// Narrower rows with the packed side on the device: one CTA per 27 x 27
// rectangle of the packed grid.  The low three base-3 digits of omega_x and
// omega_y give the low six bits of lambda (Theorem 1: digit i of omega_x bit
// 2i, of omega_y bit 2i + 1), so such a rectangle is one level-6 sub-gasket:
// its tiles lie in one 64 x 64-tile square whose corner is lambda of the high
// digits, shifted by six bits.  Each warp maps that corner once (the ballot
// form of the map) and the 729 tiles through a table built at compile time;
// every access the CTA makes stays in that square.
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

// Byte offset of tile row r (packed order) in the embedded array.
__device__ __forceinline__ size_t embedded_offset(int64_t r, int n, int rb, int w, int rho, int elem) {
  const int64_t j = r / rho;  // tile, in lambda order
  const int ty = (int)(r - j * rho);
  int bx, by;
  lambda_scalar((uint32_t)(j % w), (uint32_t)(j / w), rb, bx, by);
  return ((size_t)by * rho + ty) * (size_t)n * elem + (size_t)bx * rho * elem;
}

template <int RB, bool PACK>  // RB = row bytes < 16
__global__ void __launch_bounds__(256) pack_narrow_kernel(const unsigned char* __restrict__ src,
                                                          unsigned char* __restrict__ dst, int n, int rb, int w,
                                                          int rho, int elem, int64_t rows) {
  using T = typename Vec<RB>::T;
  constexpr int G = 16 / RB;
  const int64_t groups = (rows + G - 1) / G;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < groups;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = q * G;
    if (r0 + G <= rows) {
      alignas(16) T e[G];
      if (PACK) {
#pragma unroll
        for (int g = 0; g < G; ++g) e[g] = *reinterpret_cast<const T*>(src + embedded_offset(r0 + g, n, rb, w, rho, elem));
        *reinterpret_cast<uint4*>(dst + r0 * RB) = *reinterpret_cast<const uint4*>(e);
      } else {
        *reinterpret_cast<uint4*>(e) = *reinterpret_cast<const uint4*>(src + r0 * RB);
#pragma unroll
        for (int g = 0; g < G; ++g) *reinterpret_cast<T*>(dst + embedded_offset(r0 + g, n, rb, w, rho, elem)) = e[g];
      }
    } else {  // the last, partial group
      for (int64_t r = r0; r < rows; ++r) {
        const size_t emb = embedded_offset(r, n, rb, w, rho, elem);
        if (PACK)
          *reinterpret_cast<T*>(dst + r * RB) = *reinterpret_cast<const T*>(src + emb);
        else
          *reinterpret_cast<T*>(dst + emb) = *reinterpret_cast<const T*>(src + r * RB);
      }
    }
  }
}

// Local offsets of the 729 tiles of a level-6 sub-gasket, x | y << 8, for
// (u mod 27, u div 27): lambda of the low three digits of omega_x and omega_y
// (the per-thread form of the map, evaluated at compile time).
struct Lambda6 {
  uint16_t v[729];
  constexpr Lambda6() : v() {
    for (int u = 0; u < 729; ++u) {
      int wx = u % 27, wy = u / 27, x = 0, y = 0;
      for (int mu = 1; mu <= 6; ++mu) {
        int beta = 0;
        if (mu & 1) {
          beta = wx % 3;
          wx /= 3;
        } else {
          beta = wy % 3;
          wy /= 3;
        }
        x |= (beta >> 1) << (mu - 1);
        y |= (1 - (beta - (beta >> 1))) << (mu - 1);
      }
      v[u] = (uint16_t)(x | (y << 8));
    }
  }
};
__constant__ Lambda6 kLambda6 = Lambda6();

// One CTA per 27 x 27 rectangle (blockIdx.x, blockIdx.y) of the packed grid
// (width w, level rb >= 6): item i = (tile u, row ty) of the rectangle, u in
// row-major order, so that consecutive threads walk consecutive packed rows.
template <int ELEM, int RHO, bool PACK>
__global__ void __launch_bounds__(256) pack_rect_kernel(const unsigned char* __restrict__ src,
                                                        unsigned char* __restrict__ dst, int n, int rb, int w) {
  constexpr int RB = ELEM * RHO;
  using T = typename Vec<RB>::T;
  constexpr int kSide = 27, kItems = kSide * kSide * RHO;
  int ox, oy;  // the sub-gasket's corner: lambda of the high digits, six bits up
  warp_lambda(blockIdx.x, blockIdx.y, rb - 6, ox, oy);
  ox <<= 6;
  oy <<= 6;
  for (int i = threadIdx.x; i < kItems; i += blockDim.x) {
    const int u = i / RHO, ty = i - u * RHO;
    const int ux = u % kSide, uy = u / kSide;
    const int64_t j = ((int64_t)blockIdx.y * kSide + uy) * w + (int64_t)blockIdx.x * kSide + ux;  // packed tile
    const uint32_t e = kLambda6.v[u];
    const int bx = ox + (int)(e & 0xffu), by = oy + (int)(e >> 8);
    const size_t emb = ((size_t)by * RHO + ty) * (size_t)n * ELEM + (size_t)bx * RB;
    const size_t pk = ((size_t)j * RHO + ty) * RB;
    if (PACK)
      *reinterpret_cast<T*>(dst + pk) = *reinterpret_cast<const T*>(src + emb);
    else
      *reinterpret_cast<T*>(dst + emb) = *reinterpret_cast<const T*>(src + pk);
  }
}

template <bool PACK>
cudaError_t run(const void* src, void* dst, int n, int rb, int rho, int elem, bool packed_on_device,
                cudaStream_t s) {
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
  const int rb_bytes = rho * elem;  // a power of two: rho is, elem is 1 or 4
  if (rb_bytes >= 16) {
    pack_kernel<16, PACK><<<(unsigned)blocks, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
    return cudaGetLastError();
  }
  if (packed_on_device && rb >= 6) {
    const dim3 grid((unsigned)(w / 27), (unsigned)(tiles / w / 27));
    if (elem == 4) {  // rho 1 or 2
      if (rho == 1) pack_rect_kernel<4, 1, PACK><<<grid, 256, 0, s>>>(a, b, n, rb, w);
      else pack_rect_kernel<4, 2, PACK><<<grid, 256, 0, s>>>(a, b, n, rb, w);
    } else {          // rho 1, 2, 4 or 8
      if (rho == 1) pack_rect_kernel<1, 1, PACK><<<grid, 256, 0, s>>>(a, b, n, rb, w);
      else if (rho == 2) pack_rect_kernel<1, 2, PACK><<<grid, 256, 0, s>>>(a, b, n, rb, w);
      else if (rho == 4) pack_rect_kernel<1, 4, PACK><<<grid, 256, 0, s>>>(a, b, n, rb, w);
      else pack_rect_kernel<1, 8, PACK><<<grid, 256, 0, s>>>(a, b, n, rb, w);
    }
    return cudaGetLastError();
  }
  int64_t groups = (rows * rb_bytes + 15) / 16;
  int64_t gblocks = (groups + 255) / 256;
  if (gblocks > 152 * 64) gblocks = 152 * 64;
  const unsigned g = (unsigned)gblocks;
  if (rb_bytes == 8)
    pack_narrow_kernel<8, PACK><<<g, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  else if (rb_bytes == 4)
    pack_narrow_kernel<4, PACK><<<g, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  else if (rb_bytes == 2)
    pack_narrow_kernel<2, PACK><<<g, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  else
    pack_narrow_kernel<1, PACK><<<g, 256, 0, s>>>(a, b, n, rb, w, rho, elem, rows);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack(const void* embedded, void* packed, int n, int rb, int rho, int elem, bool packed_on_device,
                        cudaStream_t s) {
  return run<true>(embedded, packed, n, rb, rho, elem, packed_on_device, s);
}

cudaError_t launch_unpack(const void* packed, void* embedded, int n, int rb, int rho, int elem,
                          bool packed_on_device, cudaStream_t s) {
  return run<false>(packed, embedded, n, rb, rho, elem, packed_on_device, s);
}

}  // namespace fractal
