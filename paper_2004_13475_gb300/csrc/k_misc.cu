// Map export, single write (SW) and reduction (RD) kernels (Sec. 6.2), and
// the allocation-free variant of the reduction.
#include <mutex>

#include "../../include/fractal.h"
#include "launch.h"

namespace fractal {

cudaError_t allow_smem(const void* func, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

namespace {

// ---------------------------------------------------------------- map -------
// One warp per omega: the same warp_lambda the step kernels run.
__global__ void map_blocks_kernel(int32_t* __restrict__ out, int w, int h, int levels) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t total = (int64_t)w * h;
  for (int64_t id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); id < total; id += warps) {
    int bx, by;
    warp_lambda((uint32_t)(id % w), (uint32_t)(id / w), levels, bx, by);
    if ((threadIdx.x & 31) == 0) {
      out[2 * id] = bx;
      out[2 * id + 1] = by;
    }
  }
}

// One thread per omega: the per-thread form of the map.
__global__ void map_blocks_scalar_kernel(int32_t* __restrict__ out, int w, int h, int levels) {
  const int64_t total = (int64_t)w * h;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (int64_t)gridDim.x * blockDim.x) {
    int bx, by;
    lambda_scalar((uint32_t)(id % w), (uint32_t)(id / w), levels, bx, by);
    reinterpret_cast<int2*>(out)[id] = make_int2(bx, by);
  }
}

// Tensor-core form of the digit-to-offset sum (Sec. 6.3, many blocks per
// MMA): for 16 omegas per warp, A (16 x 16, bf16 0/1) holds in column c < 8
// the x bit tau_x of level mu = c + 1 + 8h and in column c >= 8 the flipped y
// bit of level mu = c - 7 + 8h; B (16 x 8) holds 2^c in column 0 for c < 8
// and 2^(c-8) in column 1 for c >= 8.  D = A B has lambda_x and lambda_y of
// those 8 levels in its columns 0 and 1 (bf16 holds 0, 1 and 2^c exactly;
// FP32 sums < 2^24 are exact).  Half h = 1 (levels 9..16) is a second MMA,
// weighted by 2^8.  Fragment layouts of mma.m16n8k16 (PTX ISA): lane =
// 4 * group + tig; A registers {r0,r1} of rows group / group+8 at columns
// 2 tig + {0,1}, {r2,r3} at columns 2 tig + 8 + {0,1}; B registers at rows
// 2 tig + {0,1} and 2 tig + 8 + {0,1} of column group; D {d0,d1} row group,
// {d2,d3} row group + 8, columns 2 tig + {0,1}.
__device__ __forceinline__ uint32_t bf16_bits(bool one_lo, bool one_hi) {
  return (one_lo ? 0x3F80u : 0u) | (one_hi ? 0x3F800000u : 0u);
}

// bit of level mu (1-based) of omega (wx, wy): x bit [beta == 2] or flipped
// y bit [beta == 0], beta = digit ceil(mu/2)-1 of wx (odd mu) or wy (even mu)
__device__ __forceinline__ bool level_bit(uint32_t wx, uint32_t wy, int mu, int levels, bool ybit) {
  if (mu > levels) return false;
  uint32_t v = (mu & 1) ? wx : wy;
  for (int j = 0; j < (mu + 1) / 2 - 1; ++j) v /= 3u;
  const uint32_t beta = v % 3u;
  return ybit ? beta == 0u : beta == 2u;
}

__global__ void map_blocks_mma_kernel(int32_t* __restrict__ out, int w, int h, int levels) {
  const int64_t total = (int64_t)w * h;
  const int lane = threadIdx.x & 31, group = lane >> 2, tig = lane & 3;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // B fragment (the same for both halves): rows k = 2 tig + {0,1} and
  // 2 tig + 8 + {0,1}, column n = group
  auto bval = [&](int k) -> uint32_t {
    if (group == 0 && k < 8) return 0x3F80u + ((uint32_t)k << 7);         // 2^k
    if (group == 1 && k >= 8) return 0x3F80u + ((uint32_t)(k - 8) << 7);  // 2^(k-8)
    return 0u;
  };
  const uint32_t b0 = bval(2 * tig) | (bval(2 * tig + 1) << 16);
  const uint32_t b1 = bval(2 * tig + 8) | (bval(2 * tig + 9) << 16);
  for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 16; base < total;
       base += warps * 16) {
    const int64_t id0 = base + group, id1 = base + group + 8;
    const uint32_t x0 = (uint32_t)(id0 % w), y0 = (uint32_t)(id0 / w);
    const uint32_t x1 = (uint32_t)(id1 % w), y1 = (uint32_t)(id1 / w);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int half = 0; half < 2 && 8 * half < levels; ++half) {
      // A entry for (omega, column c) of this half
      auto abit = [&](uint32_t wx, uint32_t wy, int c) -> bool {
        return c < 8 ? level_bit(wx, wy, c + 1 + 8 * half, levels, false)
                     : level_bit(wx, wy, c - 7 + 8 * half, levels, true);
      };
      const int c0 = 2 * tig, c1 = 2 * tig + 8;
      const uint32_t a0 = bf16_bits(abit(x0, y0, c0), abit(x0, y0, c0 + 1));
      const uint32_t a1 = bf16_bits(abit(x1, y1, c0), abit(x1, y1, c0 + 1));
      const uint32_t a2 = bf16_bits(abit(x0, y0, c1), abit(x0, y0, c1 + 1));
      const uint32_t a3 = bf16_bits(abit(x1, y1, c1), abit(x1, y1, c1 + 1));
      float d0, d1, d2, d3;
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%10,%11,%12,%13};"
          : "=f"(d0), "=f"(d1), "=f"(d2), "=f"(d3)
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.f), "f"(0.f), "f"(0.f), "f"(0.f));
      const float scale = half ? 256.f : 1.f;
      acc[0] += scale * d0;
      acc[1] += scale * d1;
      acc[2] += scale * d2;
      acc[3] += scale * d3;
    }
    if (tig == 0) {
      if (id0 < total) reinterpret_cast<int2*>(out)[id0] = make_int2((int)acc[0], (int)acc[1]);
      if (id1 < total) reinterpret_cast<int2*>(out)[id1] = make_int2((int)acc[2], (int)acc[3]);
    }
  }
}

// ----------------------------------------------------------------- SW -------
// Sec. 6.2 SW: `value` at every member of every member tile, 0 at the tile's
// other cells; no loads.
//
// uint8: the super-tile row by row, so that a warp's stores run along one
// array row across the member tiles it crosses (chunks of non-member tiles
// skipped).  Rows of a uint8 tile narrower than a 32-byte sector (rho <= 16)
// then reach L2 together with their neighbours' parts of the same sector:
// 82 / 75 us against 135 / 115 us tile by tile at k = 16, rho = 8 / 16.
template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) sw_u8_kernel(uint8_t* __restrict__ out, uint32_t value, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int WL = RHO < 16 ? RHO : 16;  // bytes per store
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const int lcpr = LOG_RHO + g.m - ilog2c(WL);  // log2 of the stores per super-tile row
  const int total = g.T << lcpr;
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const int y = it >> lcpr, cx = it & ((1 << lcpr) - 1);
    if (((cx * WL) >> LOG_RHO) & (y >> LOG_RHO)) continue;  // a non-member tile of the super-tile
    const int gx0 = sx * g.T + cx * WL, gy = sy * g.T + y;
    store_state_bytes<WL>(out + (size_t)gy * g.n + gx0, chunk_members<WL>(gx0, gy, g.n), value);
  }
}

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) sw_f32_kernel(float* __restrict__ out, float value, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int WC = RHO < 4 ? RHO : 4;
  constexpr int LOG_C = LOG_RHO - ilog2c(WC);
  constexpr int LOG_Q = LOG_RHO + LOG_C;
  extern __shared__ __align__(16) uint32_t smem[];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  build_slot_table<MODE>(smem, g);
  __syncthreads();
  const int total = g.slots << LOG_Q;
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const uint32_t e = smem[it >> LOG_Q];
    if (e == kNoTile) continue;
    const int c = it & ((1 << LOG_Q) - 1);
    const int gx0 = sx * g.T + (int)(e & 0xffffu) * RHO + (c & ((1 << LOG_C) - 1)) * WC;
    const int gy = sy * g.T + (int)(e >> 16) * RHO + (c >> LOG_C);
    const uint32_t mm = chunk_members<WC>(gx0, gy, g.n);
    FVec<WC> r;
#pragma unroll
    for (int i = 0; i < WC; ++i) r.v[i] = ((mm >> i) & 1u) ? value : 0.0f;
    store_f<WC>(out + (size_t)gy * g.n + gx0, r);
  }
}

// ----------------------------------------------------------------- RD -------
// Sec. 6.2 RD: sum over all members.  Each CTA writes one partial (0 for a
// discarded BB block); a single-CTA pass adds the partials in a fixed order.

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) reduce_u8_kernel(const uint8_t* __restrict__ in,
                                                        unsigned long long* __restrict__ partials, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int WL = RHO < 16 ? RHO : 16;
  constexpr int LOG_LQ = 2 * LOG_RHO - ilog2c(WL);
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long red[32];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (threadIdx.x == 0) partials[cta_id()] = 0ull;
    return;
  }
  build_slot_table<MODE>(smem, g);
  __syncthreads();
  const int total = g.slots << LOG_LQ;
  unsigned count = 0;
  for (int base = threadIdx.x; base < total; base += blockDim.x * kIPT) {
    uint32_t bits[kIPT];
#pragma unroll
    for (int u = 0; u < kIPT; ++u) {
      const int it = base + u * (int)blockDim.x;
      bits[u] = 0u;
      if (it < total) {
        const uint32_t e = smem[it >> LOG_LQ];
        if (e != kNoTile) {
          const int c = it & ((1 << LOG_LQ) - 1);
          const int gx0 = sx * g.T + (int)(e & 0xffffu) * RHO + (c & (RHO / WL - 1)) * WL;
          const int gy = sy * g.T + (int)(e >> 16) * RHO + c / (RHO / WL);
          bits[u] = load_alive_bits<WL>(in + (size_t)gy * g.n + gx0) & chunk_members<WL>(gx0, gy, g.n);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kIPT; ++u) count += __popc(bits[u]);
  }
  const unsigned long long s = block_sum<unsigned long long>(count, red);
  if (threadIdx.x == 0) partials[cta_id()] = s;
}

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) reduce_f32_kernel(const float* __restrict__ in,
                                                         double* __restrict__ partials, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int WC = RHO < 4 ? RHO : 4;
  constexpr int LOG_C = LOG_RHO - ilog2c(WC);
  constexpr int LOG_Q = LOG_RHO + LOG_C;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ double red[32];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (threadIdx.x == 0) partials[cta_id()] = 0.0;
    return;
  }
  build_slot_table<MODE>(smem, g);
  __syncthreads();
  const int total = g.slots << LOG_Q;
  double acc = 0.0;
  for (int base = threadIdx.x; base < total; base += blockDim.x * kIPT) {
    FVec<WC> v[kIPT];
    uint32_t mm[kIPT];
#pragma unroll
    for (int u = 0; u < kIPT; ++u) {
      const int it = base + u * (int)blockDim.x;
      mm[u] = 0u;
      if (it < total) {
        const uint32_t e = smem[it >> LOG_Q];
        if (e != kNoTile) {
          const int c = it & ((1 << LOG_Q) - 1);
          const int gx0 = sx * g.T + (int)(e & 0xffffu) * RHO + (c & ((1 << LOG_C) - 1)) * WC;
          const int gy = sy * g.T + (int)(e >> 16) * RHO + (c >> LOG_C);
          mm[u] = chunk_members<WC>(gx0, gy, g.n);
          if (mm[u]) v[u] = load_f<WC>(in + (size_t)gy * g.n + gx0, true);
        }
      }
    }
    // FP32 partial over at most kIPT chunks (16 cells), then FP64
    float part = 0.0f;
#pragma unroll
    for (int u = 0; u < kIPT; ++u) {
#pragma unroll
      for (int i = 0; i < WC; ++i) part += ((mm[u] >> i) & 1u) ? v[u].v[i] : 0.0f;
    }
    acc += (double)part;
  }
  const double s = block_sum<double>(acc, red);
  if (threadIdx.x == 0) partials[cta_id()] = s;
}

// Fixed-order final pass: thread t adds partials t, t+1024, ...; then a fixed tree.
template <typename V>
__global__ void __launch_bounds__(1024) final_sum_kernel(const V* __restrict__ partials, int64_t count,
                                                         double* __restrict__ out) {
  __shared__ V red[32];
  V acc = V(0);
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  const V s = block_sum<V>(acc, red);
  if (threadIdx.x == 0) *out = (double)s;
}

template <int MODE, int LOG_RHO>
cudaError_t go_sw(int dtype, const Launch& L, void* out, double value, cudaStream_t s) {
  if (dtype == 0) {
    sw_u8_kernel<MODE, LOG_RHO><<<L.grid, L.threads, L.smem, s>>>(static_cast<uint8_t*>(out),
                                                                 (uint32_t)(uint8_t)value, L.geo);
  } else {
    sw_f32_kernel<MODE, LOG_RHO><<<L.grid, L.threads, L.smem, s>>>(static_cast<float*>(out), (float)value,
                                                                  L.geo);
  }
  return cudaGetLastError();
}

template <int MODE, int LOG_RHO>
cudaError_t go_reduce(int dtype, const Launch& L, const void* in, void* partials, double* dev_out,
                      cudaStream_t s) {
  const int64_t count = (int64_t)L.grid.x * L.grid.y;
  if (dtype == 0) {
    auto* p = static_cast<unsigned long long*>(partials);
    reduce_u8_kernel<MODE, LOG_RHO><<<L.grid, L.threads, L.smem, s>>>(static_cast<const uint8_t*>(in), p, L.geo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    final_sum_kernel<unsigned long long><<<1, 1024, 0, s>>>(p, count, dev_out);
  } else {
    auto* p = static_cast<double*>(partials);
    reduce_f32_kernel<MODE, LOG_RHO><<<L.grid, L.threads, L.smem, s>>>(static_cast<const float*>(in), p, L.geo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    final_sum_kernel<double><<<1, 1024, 0, s>>>(p, count, dev_out);
  }
  return cudaGetLastError();
}

}  // namespace

// Sum of `count` per-CTA partials (uint64 counts for dtype 0, doubles for 1)
// into *dev_out, one CTA, fixed order.
cudaError_t launch_final_sum(int dtype, const void* partials, int64_t count, double* dev_out, cudaStream_t s) {
  if (dtype == 0)
    final_sum_kernel<unsigned long long>
        <<<1, 1024, 0, s>>>(static_cast<const unsigned long long*>(partials), count, dev_out);
  else
    final_sum_kernel<double><<<1, 1024, 0, s>>>(static_cast<const double*>(partials), count, dev_out);
  return cudaGetLastError();
}

namespace {

template <int MODE>
cudaError_t sw_by_rho(int log_rho, int dtype, const Launch& L, void* out, double value, cudaStream_t s) {
  switch (log_rho) {
    case 0: return go_sw<MODE, 0>(dtype, L, out, value, s);
    case 1: return go_sw<MODE, 1>(dtype, L, out, value, s);
    case 2: return go_sw<MODE, 2>(dtype, L, out, value, s);
    case 3: return go_sw<MODE, 3>(dtype, L, out, value, s);
    case 4: return go_sw<MODE, 4>(dtype, L, out, value, s);
    case 5: return go_sw<MODE, 5>(dtype, L, out, value, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE>
cudaError_t rd_by_rho(int log_rho, int dtype, const Launch& L, const void* in, void* partials, double* dev_out,
                      cudaStream_t s) {
  switch (log_rho) {
    case 0: return go_reduce<MODE, 0>(dtype, L, in, partials, dev_out, s);
    case 1: return go_reduce<MODE, 1>(dtype, L, in, partials, dev_out, s);
    case 2: return go_reduce<MODE, 2>(dtype, L, in, partials, dev_out, s);
    case 3: return go_reduce<MODE, 3>(dtype, L, in, partials, dev_out, s);
    case 4: return go_reduce<MODE, 4>(dtype, L, in, partials, dev_out, s);
    case 5: return go_reduce<MODE, 5>(dtype, L, in, partials, dev_out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_map_blocks(int32_t* out, int w, int h, int levels, cudaStream_t s, int method) {
  const int64_t total = (int64_t)w * h;
  // per pass: one omega per warp (ballot), per thread (scalar), 16 per warp (MMA)
  const int64_t per_cta = method == 1 ? 256 : method == 2 ? 8 * 16 : 8;
  int64_t blocks = (total + per_cta - 1) / per_cta;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  if (method == 1)
    map_blocks_scalar_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, w, h, levels);
  else if (method == 2)
    map_blocks_mma_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, w, h, levels);
  else
    map_blocks_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, w, h, levels);
  return cudaGetLastError();
}

cudaError_t launch_sw(int mode, int log_rho, int dtype, const Launch& L, void* out, double value,
                      cudaStream_t s) {
  return mode == kLambda ? sw_by_rho<kLambda>(log_rho, dtype, L, out, value, s)
                         : sw_by_rho<kBB>(log_rho, dtype, L, out, value, s);
}

cudaError_t launch_reduce(int mode, int log_rho, int dtype, const Launch& L, const void* in, void* partials,
                          double* dev_out, cudaStream_t s) {
  return mode == kLambda ? rd_by_rho<kLambda>(log_rho, dtype, L, in, partials, dev_out, s)
                         : rd_by_rho<kBB>(log_rho, dtype, L, in, partials, dev_out, s);
}

// ---------------------------------------------------------------------------
// Allocation-free reduce: the per-CTA partial sums live in this fixed device
// array instead of plan-owned memory.  Every GPU that loads the library holds
// it (512 KiB) until the process exits; all calls share it.
// ---------------------------------------------------------------------------

static __device__ __align__(256) double g_noalloc_partials[FRACTAL_NOALLOC_MAX_PARTIALS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the array on the current device `dev`.  The host-side
// name of the array is not a device address, so it is resolved once per
// device, with that device current, and cached for the life of the process.
cudaError_t noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace fractal

extern "C" int fractal_reduce_noalloc(int k, int rho, const void* dev_buf, int dtype, double* dev_out,
                                      void* stream) {
  using namespace fractal;
  if (k < 0 || k > FRACTAL_MAX_LEVEL || rho < 1 || rho > 32 || (rho & (rho - 1)) != 0 || rho > (1 << k))
    return FRACTAL_EINVAL;
  if (!dev_buf || !dev_out || (reinterpret_cast<uintptr_t>(dev_buf) & 15u) != 0) return FRACTAL_EINVAL;
  if (dtype != FRACTAL_U8 && dtype != FRACTAL_F32) return FRACTAL_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FRACTAL_ECUDA;
  }
  if (!device_addressable(dev_buf, dev) || !device_addressable(dev_out, dev)) return FRACTAL_EINVAL;
  const int log_rho = ilog2c(rho);
  void* partials = nullptr;
  // float32 at rho >= 4: the 8 x 8-block reduce of a default lambda plan
  // (6561 partials at k = 16), so the sum is that plan's bit for bit
  Launch B;
  int blevels = 0;
  if (dtype == FRACTAL_F32 && log_rho >= 2 && blocks_geometry(k, kLambda, B, blevels) &&
      (int64_t)B.grid.x * B.grid.y <= FRACTAL_NOALLOC_MAX_PARTIALS) {
    if (noalloc_scratch(dev, &partials) != cudaSuccess) return FRACTAL_ECUDA;
    cudaError_t e = launch_reduce_blocks(kLambda, B, blevels, static_cast<const float*>(dev_buf),
                                         static_cast<double*>(partials), dev_out, (cudaStream_t)stream);
    return e == cudaSuccess ? FRACTAL_OK : FRACTAL_ECUDA;
  }
  // otherwise the rho-tile reduce of a default lambda plan; more tile levels
  // per CTA only where its partials would not fit the array
  Launch step, aux, tma;
  bool tma_ok = false;
  int levels = default_cta_levels(k, log_rho, kLambda, dtype);
  bool fits = false;
  for (; levels <= 5 && levels <= k - log_rho; ++levels) {
    if (!plan_geometry(k, log_rho, kLambda, dtype, levels, step, aux, tma, tma_ok)) continue;
    if ((int64_t)aux.grid.x * aux.grid.y <= FRACTAL_NOALLOC_MAX_PARTIALS) {
      fits = true;
      break;
    }
  }
  if (!fits) return FRACTAL_ETOOBIG;
  if (noalloc_scratch(dev, &partials) != cudaSuccess) return FRACTAL_ECUDA;
  cudaError_t e = launch_reduce(kLambda, log_rho, dtype, aux, dev_buf, partials, dev_out, (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : FRACTAL_ECUDA;
}
