// Explicit FDM heat-diffusion step on the gasket, FP32 (the FDM time-step
// pattern named in Sec. 1), zero flux towards absent cells:
//   u'_c = u_c + a * sum_{nb in N4(c), nb member} (u_nb - u_c).
//
// One CTA per member super-tile; the member tiles and the ring cells they
// touch are staged in shared memory as floats, then every member tile row is
// updated from shared memory and stored with vector stores.  Cells of the
// shared image that belong to no member tile are never written and never
// used: every neighbour read is selected by the arithmetic membership test.
#include "launch.h"

namespace fractal {
namespace {

template <int MODE, int LOG_RHO>
__global__ void __launch_bounds__(512) diffusion_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                        float a, Geo g) {
  constexpr int RHO = 1 << LOG_RHO;
  constexpr int WC = RHO < 4 ? RHO : 4;       // cells per chunk (one float4 at most)
  constexpr int LOG_C = LOG_RHO - ilog2c(WC);  // chunks per tile row
  constexpr int LOG_Q = LOG_RHO + LOG_C;       // chunks per tile
  extern __shared__ __align__(16) uint32_t smem[];

  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const int n = g.n;
  const int T = g.T;
  const int P = ((T + 3) & ~3) + 8;  // image pitch (floats); interior column 0 at offset 4
  uint32_t* tab = smem;
  float* img = reinterpret_cast<float*>(smem + tab_words(g.slots));
  const int ox = sx * T, oy = sy * T;

  build_slot_table<MODE>(tab, g);
  for (int it = threadIdx.x; it < 4 * T + 4; it += blockDim.x) {
    int lx, ly;
    ring_cell(it, T, lx, ly);
    const int gx = ox + lx, gy = oy + ly;
    float v = 0.0f;
    if (is_member(gx, gy, n) && ring_needed(lx, ly, gx, gy, T, n)) v = __ldg(in + (size_t)gy * n + gx);
    img[(ly + 1) * P + 4 + lx] = v;
  }
  __syncthreads();

  // Stage the member tiles.  Each thread issues all of its (up to kIPT)
  // loads before it writes any of them to shared memory, so the CTA keeps
  // every load of its super-tile in flight at once.
  const int total = g.slots << LOG_Q;
  for (int base = threadIdx.x; base < total; base += blockDim.x * kIPT) {
    FVec<WC> v[kIPT];
    int off[kIPT];
#pragma unroll
    for (int u = 0; u < kIPT; ++u) {
      const int it = base + u * (int)blockDim.x;
      off[u] = -1;
      if (it < total) {
        const uint32_t e = tab[it >> LOG_Q];
        if (e != kNoTile) {
          const int c = it & ((1 << LOG_Q) - 1);
          const int lx0 = (int)(e & 0xffffu) * RHO + (c & ((1 << LOG_C) - 1)) * WC;
          const int ly = (int)(e >> 16) * RHO + (c >> LOG_C);
          v[u] = load_f<WC>(in + (size_t)(oy + ly) * n + ox + lx0, true);
          off[u] = (ly + 1) * P + 4 + lx0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kIPT; ++u)
      if (off[u] >= 0) store_f<WC>(img + off[u], v[u]);
  }
  __syncthreads();

  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const uint32_t e = tab[it >> LOG_Q];
    if (e == kNoTile) continue;
    const int c = it & ((1 << LOG_Q) - 1);
    const int lx0 = (int)(e & 0xffffu) * RHO + (c & ((1 << LOG_C) - 1)) * WC;
    const int ly = (int)(e >> 16) * RHO + (c >> LOG_C);
    const int gx0 = ox + lx0, gy = oy + ly;
    const float* pm = img + (ly + 1) * P + 4 + lx0;
    const FVec<WC> up = load_f<WC>(pm - P, false);
    const FVec<WC> md = load_f<WC>(pm, false);
    const FVec<WC> dn = load_f<WC>(pm + P, false);
    const float left = pm[-1];
    const float right = pm[WC];
    const uint32_t mu = chunk_members<WC>(gx0, gy - 1, n);
    const uint32_t mm = chunk_members<WC>(gx0, gy, n);
    const uint32_t md_ = chunk_members<WC>(gx0, gy + 1, n);
    const bool ml = is_member(gx0 - 1, gy, n);
    const bool mr = is_member(gx0 + WC, gy, n);
    FVec<WC> r;
#pragma unroll
    for (int i = 0; i < WC; ++i) {
      const float u = md.v[i];
      // N4 in the order up, left, right, down; absent neighbours carry no flux.
      float s = ((mu >> i) & 1u) ? up.v[i] - u : 0.0f;
      const bool hl = i == 0 ? ml : (((mm >> (i - 1)) & 1u) != 0u);
      const float vl = i == 0 ? left : md.v[i > 0 ? i - 1 : 0];
      s += hl ? vl - u : 0.0f;
      const bool hr = i == WC - 1 ? mr : (((mm >> (i + 1)) & 1u) != 0u);
      const float vr = i == WC - 1 ? right : md.v[i < WC - 1 ? i + 1 : 0];
      s += hr ? vr - u : 0.0f;
      s += ((md_ >> i) & 1u) ? dn.v[i] - u : 0.0f;
      r.v[i] = ((mm >> i) & 1u) ? fmaf(a, s, u) : 0.0f;
    }
    store_f<WC>(out + (size_t)gy * n + gx0, r);
  }
}

template <int MODE, int LOG_RHO>
cudaError_t go(const Launch& L, const float* in, float* out, float a, cudaStream_t s) {
  auto* k = diffusion_kernel<MODE, LOG_RHO>;
  cudaError_t e = allow_smem((const void*)k, L.smem);
  if (e != cudaSuccess) return e;
  k<<<L.grid, L.threads, L.smem, s>>>(in, out, a, L.geo);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t by_rho(int log_rho, const Launch& L, const float* in, float* out, float a, cudaStream_t s) {
  switch (log_rho) {
    case 0: return go<MODE, 0>(L, in, out, a, s);
    case 1: return go<MODE, 1>(L, in, out, a, s);
    case 2: return go<MODE, 2>(L, in, out, a, s);
    case 3: return go<MODE, 3>(L, in, out, a, s);
    case 4: return go<MODE, 4>(L, in, out, a, s);
    case 5: return go<MODE, 5>(L, in, out, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_diffusion(int mode, int log_rho, const Launch& L, const float* in, float* out,
                             float a, cudaStream_t s) {
  return mode == kLambda ? by_rho<kLambda>(log_rho, L, in, out, a, s)
                         : by_rho<kBB>(log_rho, L, in, out, a, s);
}

}  // namespace fractal
