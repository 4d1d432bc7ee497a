// Host-side launch descriptors and per-family dispatchers (internal).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "gasket.cuh"

namespace fractal {

struct Launch {
  dim3 grid;
  int threads;
  int smem;  // dynamic shared memory bytes
  Geo geo;
};

// Every device allocation of the library goes through here, so that a test
// can make the n-th one fail (fractal_debug_fail_allocs).
cudaError_t lib_malloc(void** p, size_t bytes);
template <typename T>
cudaError_t lib_malloc(T** p, size_t bytes) {
  return lib_malloc(reinterpret_cast<void**>(p), bytes);
}

// One CTA arms an mbarrier that nothing completes and waits on it with the
// step kernels' bounded wait, `spins` polls at most: the timeout path (code
// 1 in *err, then return).
cudaError_t launch_wait_selftest(int* err, uint32_t spins, cudaStream_t s);

// Kernels on `device` can dereference p (device, managed, or mapped pinned
// host memory); a host-side query that touches nothing.
bool device_addressable(const void* p, int device);

// Each returns the launch error (cudaSuccess when queued).
cudaError_t launch_ca(int mode, int log_rho, const Launch& L, const uint8_t* in, uint8_t* out,
                      cudaStream_t s);
cudaError_t launch_diffusion(int mode, int log_rho, const Launch& L, const float* in, float* out,
                             float a, cudaStream_t s);
cudaError_t launch_sw(int mode, int log_rho, int dtype, const Launch& L, void* out, double value,
                      cudaStream_t s);
cudaError_t launch_reduce(int mode, int log_rho, int dtype, const Launch& L, const void* in,
                          void* partials, double* dev_out, cudaStream_t s);
// method: 0 warp ballot (one omega per warp), 1 per thread, 2 tensor-core MMA
cudaError_t launch_map_blocks(int32_t* out, int w, int h, int levels, cudaStream_t s, int method = 0);

// TMA-staged step kernels (rho * element size >= 16 bytes; see k_tma.cu).
// `map` has rho x rho boxes over the input array, `ring` 16-byte boxes of one row.
cudaError_t launch_diffusion_tma(int mode, int log_rho, const Launch& L, const CUtensorMap& map,
                                 const CUtensorMap& ring, float* out, float a, int* err, cudaStream_t s);
cudaError_t launch_ca_tma(int mode, int log_rho, const Launch& L, const CUtensorMap& map, const CUtensorMap& ring,
                          uint8_t* out, int* err, cudaStream_t s);
int tma_smem_bytes(const Geo& g, int tile_bytes, int dtype);

// Temporally fused diffusion: nsteps (<= margin) steps per launch (k_fused.cu).
// partials (nullable): one double per CTA of L, the sum of the result's
// members over the CTA's super-tile (finish with launch_final_sum).
// in / out: embedded arrays; pin / pout (when not null): compact records in
// place of in / out (the state between the launches of one call).
// desc (when not null): the launch's per-thread descriptors from
// launch_fused_describe for the same geometry, margin and reach.
// reach (<= margin): the most steps a launch of the configuration takes
// (nsteps <= reach); margin-box blocks further than that from the
// super-tile are not staged.
cudaError_t launch_diffusion_fused(int mode, int log_rho, int margin, int reach, const Launch& L, const float* in,
                                   float* out, float a, int nsteps, cudaStream_t s, double* partials = nullptr,
                                   const float* pin = nullptr, float* pout = nullptr, const int4* desc = nullptr);
// Descriptors of a fused launch (one per thread of each member super-tile's
// CTA, 16 bytes) and the kernel that writes them.
int64_t fused_descriptors(const Launch& L);
cudaError_t launch_fused_describe(int mode, int log_rho, int margin, int reach, const Launch& L, int4* desc,
                                  cudaStream_t s);
// Compact records of a level-k gasket (3^(k-3), one per member 8 x 8 block)
// and the bytes of one.
int64_t fused_records(int k);
int fused_record_bytes();
int fused_margin(int steps_per_launch);
int fused_smem_bytes(const Geo& g, int margin, int reach);
int fused_threads(const Geo& g, int rho, int margin, int reach);
// Block slots of the one-warp fused launch (super-tiles of side 128, margins
// up to 16 cells).
int fused_warp_slots();
// Double-float conductivity launches for the gradient path (super-tiles of
// side min(128, n), margins min(32, side / 2), k >= 4): `nsteps` <= margin
// steps in -> out (out may be null) recording the state before each step
// (and after the last when out is null) into traj (may be null); and the
// kappa gradient of a segment from two recorded trajectories.  in_f32 (when
// not null) replaces in: a float32 state read as (x, 0) pairs; out_f32 (when
// not null) replaces out: hi + lo written as float32.
bool kappa_fused_geometry(int k, int mode, Launch& L, int& margin);
int64_t kappa_record_float4s(int k);
cudaError_t launch_kappa_fused_df(int mode, int k, const dfloat* in, dfloat* out, float4* traj, const float* kappa,
                                  dfloat ha, int nsteps, cudaStream_t s, const float* in_f32 = nullptr,
                                  float* out_f32 = nullptr);
// The gradient pass adds to gk (accumulate != 0) or starts from 0, and
// writes gk, or out_f32 as float32 when that is not null.
cudaError_t launch_kappa_grad_df(int mode, int k, const float4* utraj, const float4* ptraj, dfloat* gk, dfloat ha,
                                 int nsteps, cudaStream_t s, int accumulate = 1, float* out_f32 = nullptr);

// Block slots of the four-warp fused launch (super-tiles of side 256,
// margins of 64 cells at a reach of at most 56 steps).
int fused_q3_slots();
// Most member blocks of the margin boxes (W blocks wide) of a level-L
// super-tile within `reach` cells of it.
int box_cap_reach(int L, int W, int reach);

// Temporally fused automaton on a bit image: nsteps (<= margin <= 31) steps
// per launch over 32 x 32-cell word tiles (k_fused_ca.cu).
// in / out: embedded arrays; pin / pout (when not null): bit records of the
// member word tiles in place of in / out (the state between the launches of
// one call).
cudaError_t launch_ca_fused(int mode, const Launch& L, const uint8_t* in, uint8_t* out, int nsteps, int margin,
                            cudaStream_t s, unsigned long long* partials = nullptr, const uint32_t* pin = nullptr,
                            uint32_t* pout = nullptr);
// Bit records of a level-k gasket: 3^(k-5) member 32 x 32 word tiles, 128
// bytes each.
int64_t ca_records(int k);

// Sum of per-CTA partials (dtype 0: uint64 counts, 1: doubles) into *dev_out.
cudaError_t launch_final_sum(int dtype, const void* partials, int64_t count, double* dev_out, cudaStream_t s);
int ca_fused_smem_bytes(const Geo& g, int margin);
int ca_fused_threads(const Geo& g, int margin);

// Diffusion with per-cell conductivity and its reverse step (k_adjoint.cu):
// one thread per member 8 x 8 block, super-tiles of 2^levels blocks a side.
// Member tiles in lambda order <-> the embedded array (k_pack.cu); elem =
// bytes per element.
// packed_on_device: the packed side is device memory (else pinned host
// memory mapped into the device).
cudaError_t launch_pack(const void* embedded, void* packed, int n, int rb, int rho, int elem, bool packed_on_device,
                        cudaStream_t s);
cudaError_t launch_unpack(const void* packed, void* embedded, int n, int rb, int rho, int elem,
                          bool packed_on_device, cudaStream_t s);

// Float32 reduce with one 8 x 8 block per thread (k_blocks.cu); k >= 3,
// rho >= 4.
bool blocks_geometry(int k, int mode, Launch& L, int& levels);
cudaError_t launch_reduce_blocks(int mode, const Launch& L, int levels, const float* in, double* partials,
                                 double* dev_out, cudaStream_t s);

// T = float, double or dfloat (the state precision); G = the dJ/dkappa
// accumulator: double for float and double states, dfloat for dfloat.
bool kappa_geometry(int k, int mode, Launch& L, int& levels);
template <typename T>
cudaError_t launch_diffusion_kappa(int mode, const Launch& L, int levels, const T* in, T* out, const float* kappa,
                                   T a, cudaStream_t s);
template <typename T, typename G>
cudaError_t launch_diffusion_adjoint(int mode, const Launch& L, int levels, const T* ut, const T* pin, T* pout,
                                     const float* kappa, G* gkappa, T a, cudaStream_t s);

// One instance of a batch (device table entry).
struct BatchInst {
  float* a;       // the instance's two n x n buffers
  float* b;
  int64_t first;  // its first item (member super-tile) in the batch
  int32_t n;      // 2^k
  int32_t R;      // super-tile levels of its grid: k - log2(T)
  int32_t lwR;    // 3^ceil(R/2)
  int32_t pad;
};

// Persistent fused diffusion over `items` super-tiles of side T of the
// instances (which = 0: a -> b, 1: b -> a); threads = fused_threads for T,
// margin and reach.  Per-instance member sums through `partials` (items doubles).
// pin / pout (when not null): the block records of all instances (item w's
// at w * 3^log2(T/8)) in place of the instances' buffers.
// desc (when not null): the batch's per-thread setups from
// launch_batch_describe for the same table, super-tile side and margin.
cudaError_t launch_diffusion_batch(const BatchInst* inst, int count, int64_t items, int which, float a, int nsteps,
                                   int margin, int reach, int T, int ctas, int threads, cudaStream_t s,
                                   const float* pin = nullptr, float* pout = nullptr, const int4* desc = nullptr);
cudaError_t launch_batch_describe(const BatchInst* inst, int count, int64_t items, int margin, int reach, int T,
                                  int ctas, int threads, int4* desc, cudaStream_t s);
cudaError_t launch_batch_reduce(const BatchInst* inst, int count, int64_t items, int which, int T, int ctas,
                                double* partials, double* out, cudaStream_t s);
int fused_batch_smem_bytes(int threads);
const void* fused_batch_kernel();

// Grid and Geo of super-tiles of `levels` tile levels (threads and shared
// memory left 0); false if levels or the grid are out of range.
bool supertile_grid(int k, int log_rho, int mode, int levels, Launch& L);

// Launch geometry of the kernels for level k, tile side 2^log_rho, mode,
// dtype and `levels` tile levels per CTA (false if it does not fit).
bool plan_geometry(int k, int log_rho, int mode, int dtype, int levels, Launch& step, Launch& aux, Launch& tma,
                   bool& tma_ok);
int default_cta_levels(int k, int log_rho, int mode, int dtype);

// Dynamic shared memory above the 48 KB default needs an opt-in per kernel.
cudaError_t allow_smem(const void* func, int bytes);

}  // namespace fractal
