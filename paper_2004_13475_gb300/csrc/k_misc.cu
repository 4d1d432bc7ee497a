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

// ----------------------------------------------------------------- SW -------
// Sec. 6.2 SW: `value` at every member of every member tile, 0 at the tile's
// other cells; no loads.
template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) sw_u8_kernel(uint8_t* __restrict__ out, uint32_t value, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int WL = RHO < 16 ? RHO : 16;           // bytes per store
  constexpr int LOG_LQ = 2 * LOG_RHO - ilog2c(WL);  // stores per tile
  extern __shared__ __align__(16) uint32_t smem[];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  build_slot_table<MODE>(smem, g);
  __syncthreads();
  const int total = g.slots << LOG_LQ;
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const uint32_t e = smem[it >> LOG_LQ];
    if (e == kNoTile) continue;
    const int c = it & ((1 << LOG_LQ) - 1);
    const int gx0 = sx * g.T + (int)(e & 0xffffu) * RHO + (c & (RHO / WL - 1)) * WL;
    const int gy = sy * g.T + (int)(e >> 16) * RHO + c / (RHO / WL);
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

cudaError_t launch_map_blocks(int32_t* out, int w, int h, int levels, cudaStream_t s) {
  const int64_t total = (int64_t)w * h;
  int64_t blocks = (total + 7) / 8;  // 8 warps per block, one omega per warp per pass
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
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

// Device address of the array on the current device.  The host-side name of
// the array is not a device address, so it is resolved once per device, with
// that device current, and cached.
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
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
  const int log_rho = ilog2c(rho);
  // lambda launch; more tile levels per CTA until the partials fit the array
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
  void* partials = nullptr;
  if (noalloc_scratch(&partials) != cudaSuccess) return FRACTAL_ECUDA;
  cudaError_t e = launch_reduce(kLambda, log_rho, dtype, aux, dev_buf, partials, dev_out, (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : FRACTAL_ECUDA;
}
