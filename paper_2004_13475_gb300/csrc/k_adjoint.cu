// Diffusion with a per-cell conductivity and its adjoint (reverse) step, for
// gradients of a loss with respect to the initial state and the conductivity.
//
// The step: u'_c = u_c + a * sum_{nb in N4(c), nb member} g_{c,nb} (u_nb - u_c),
// with g_{c,nb} = (kappa_c + kappa_nb) / 2, i.e. u_{t+1} = A u_t with A
// symmetric.  The reverse step of a loss J with p_{t+1} = dJ/du_{t+1}:
//   p_t = A^T p_{t+1} = A p_{t+1}
//   dJ/dkappa_c += (a / 2) sum_{nb} (u_t,nb - u_t,c) (p_{t+1},c - p_{t+1},nb)
// (g_{c,nb} enters row c and row nb of A u_t).
//
// State precision.  The states u and p are float, double or double-float
// (template T); kappa is float; dJ/dkappa is accumulated in double (float and
// double states) or double-float (double-float state).  An FP32 trajectory
// rounds u every step, and those roundings reach the gradients through
// differences of neighbouring values: over 200 steps they alone move the
// gradients by a few 1e-4 of their scale from the exact ones.  A double or a
// double-float state keeps the adjoint within 1e-4 of an FP64 reference; the
// double-float one runs on the FP32 pipes (FP64 issues at a small fraction of
// the FP32 rate on this GPU) and converts nothing per step.
//
// Launch: the lambda map at the level of 8 x 8 blocks.  A CTA takes a member
// super-tile of 2^L x 2^L blocks (Theorem 1 for the CTA, lambda again for the
// 3^L member blocks inside, Sec. 5.1), one thread per block.  A member block
// (BX & BY == 0) holds the 27 members (i, j), i & j == 0, of a level-3
// gasket and meets the rest of the gasket through four links only: (0,0) to
// (0,7) of the block above and to (7,0) of the block left, (7,0) to (0,0) of
// the block right, (0,7) to (0,0) of the block below.  Each thread reads its
// block's member chunks and those four neighbour cells, and writes whole
// 32-byte rows of its block (0 at the non-members).
#include "blocks.cuh"
#include "launch.h"

namespace fractal {
namespace {

__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

template <int MODE, typename T>
__global__ void __launch_bounds__(128) diffusion_kappa_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                              const float* __restrict__ kappa, T a, Geo g, int L) {
  BlockPos b;
  if (!block_pos<MODE>(g, L, b) || !b.active) return;
  const int n = g.n;
  T u[kB * kB], w[kB * kB];
  float k[kB * kB];
  load_block(u, in + b.base, n);
  load_block(k, kappa + b.base, n);
  const Ports<T> pu = load_ports(in + b.base, n, b.hu, b.hl, b.hr, b.hd);
  const Ports<float> pk = load_ports(kappa + b.base, n, b.hu, b.hl, b.hr, b.hd);
  const T ha = T(0.5) * a;
#pragma unroll
  for (int j = 0; j < kB; ++j) {
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const int c = j * kB + i;
      if (!amem(i, j)) {
        w[c] = T(0);
        continue;
      }
      T s = T(0);
      for_neighbours(i, j, u, k, u, pu, pk, pu, b.hu, b.hl, b.hr, b.hd,
                     [&](T un, float kn, T) { s = fmat(T(k[c]) + T(kn), un - u[c], s); });
      w[c] = fmat(ha, s, u[c]);
    }
  }
  store_block(out + b.base, n, w);
}

// Accumulator of dJ/dkappa for state type T.
template <typename T>
struct GradOf {
  using type = double;
};
template <>
struct GradOf<dfloat> {
  using type = dfloat;
};

template <int MODE, typename T, typename G = typename GradOf<T>::type>
__global__ void __launch_bounds__(128) diffusion_adjoint_kernel(const T* __restrict__ ut, const T* __restrict__ pin,
                                                                T* __restrict__ pout, const float* __restrict__ kappa,
                                                                G* __restrict__ gkappa, T a, Geo g, int L) {
  BlockPos b;
  if (!block_pos<MODE>(g, L, b) || !b.active) return;
  const int n = g.n;
  T u[kB * kB], p[kB * kB], w[kB * kB];
  float k[kB * kB];
  load_block(u, ut + b.base, n);
  load_block(k, kappa + b.base, n);
  load_block(p, pin + b.base, n);
  const Ports<T> pu = load_ports(ut + b.base, n, b.hu, b.hl, b.hr, b.hd);
  const Ports<float> pk = load_ports(kappa + b.base, n, b.hu, b.hl, b.hr, b.hd);
  const Ports<T> pp = load_ports(pin + b.base, n, b.hu, b.hl, b.hr, b.hd);
  const T ha = T(0.5) * a;
  const G hd = G(0.5) * G(a);
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    G* grow = gkappa + b.base + (size_t)j * n;
    G gr[kB];
    ld4(grow, gr);
    ld4(grow + 4, gr + 4);
#pragma unroll
    for (int i = 0; i < kB; ++i) {
      const int c = j * kB + i;
      if (!amem(i, j)) {
        w[c] = T(0);
        gr[i] = G(0);
        continue;
      }
      T sp = T(0);
      G sg = G(0);
      for_neighbours(i, j, u, k, p, pu, pk, pp, b.hu, b.hl, b.hr, b.hd, [&](T un, float kn, T pn) {
        sp = fmat(T(k[c]) + T(kn), pn - p[c], sp);          // ((A p)_c - p_c) * 2 / a
        sg = fmat(G(un - u[c]), G(p[c] - pn), sg);          // dJ/dkappa_c of this step * 2 / a
      });
      w[c] = fmat(ha, sp, p[c]);
      gr[i] = fmat(hd, sg, gr[i]);
    }
    st4(grow, gr);
    st4(grow + 4, gr + 4);
  }
  store_block(pout + b.base, n, w);
}

}  // namespace

// Geometry: super-tiles of 2^L x 2^L blocks (L = 4: 81 member blocks, 96
// threads; smaller arrays take one super-tile).
bool kappa_geometry(int k, int mode, Launch& L, int& levels) {
  if (k < 3) return false;
  const int rb = k - 3;          // block levels of the array
  levels = rb < 4 ? rb : 4;
  if (!supertile_grid(k, 3, mode, levels, L)) return false;
  int nb = 1;
  for (int i = 0; i < levels; ++i) nb *= 3;
  L.threads = (nb + 31) / 32 * 32;
  L.smem = 0;
  return true;
}

template <typename T>
cudaError_t launch_diffusion_kappa(int mode, const Launch& L, int levels, const T* in, T* out, const float* kappa,
                                   T a, cudaStream_t s) {
  if (mode == kLambda)
    diffusion_kappa_kernel<kLambda, T><<<L.grid, L.threads, 0, s>>>(in, out, kappa, a, L.geo, levels);
  else
    diffusion_kappa_kernel<kBB, T><<<L.grid, L.threads, 0, s>>>(in, out, kappa, a, L.geo, levels);
  return cudaGetLastError();
}

template <typename T, typename G>
cudaError_t launch_diffusion_adjoint(int mode, const Launch& L, int levels, const T* ut, const T* pin, T* pout,
                                     const float* kappa, G* gkappa, T a, cudaStream_t s) {
  if (mode == kLambda)
    diffusion_adjoint_kernel<kLambda, T><<<L.grid, L.threads, 0, s>>>(ut, pin, pout, kappa, gkappa, a, L.geo, levels);
  else
    diffusion_adjoint_kernel<kBB, T><<<L.grid, L.threads, 0, s>>>(ut, pin, pout, kappa, gkappa, a, L.geo, levels);
  return cudaGetLastError();
}

template cudaError_t launch_diffusion_kappa<float>(int, const Launch&, int, const float*, float*, const float*, float,
                                                   cudaStream_t);
template cudaError_t launch_diffusion_kappa<double>(int, const Launch&, int, const double*, double*, const float*,
                                                    double, cudaStream_t);
template cudaError_t launch_diffusion_kappa<dfloat>(int, const Launch&, int, const dfloat*, dfloat*, const float*,
                                                    dfloat, cudaStream_t);
template cudaError_t launch_diffusion_adjoint<float, double>(int, const Launch&, int, const float*, const float*,
                                                             float*, const float*, double*, float, cudaStream_t);
template cudaError_t launch_diffusion_adjoint<double, double>(int, const Launch&, int, const double*, const double*,
                                                              double*, const float*, double*, double, cudaStream_t);
template cudaError_t launch_diffusion_adjoint<dfloat, dfloat>(int, const Launch&, int, const dfloat*, const dfloat*,
                                                              dfloat*, const float*, dfloat*, dfloat, cudaStream_t);

}  // namespace fractal
