// Device twin of synth/__init__.py: SplitMix64 counter-based fill of an
// n x n embedding.  Cell (x, y) receives output number y*n + x of the stream
// seeded with `seed`: mix(seed + (y*n + x + 1) * GAMMA), with the 64-bit
// finaliser of Steele, Lea and Flood (OOPSLA 2014) as published by Vigna.
// Like the host module it knows nothing about the gasket: every cell is filled.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// dist 0: uint8 Bernoulli(1/2) = h >> 63.
// dist 1: float32 lo + width * ((h >> 40) * 2^-24).
__global__ void fill_kernel(void* out, int dist, uint64_t total, uint64_t seed,
                            float lo, float width) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    uint64_t h = mix64(seed + (i + 1) * kGamma);
    if (dist == 0) {
      static_cast<uint8_t*>(out)[i] = (uint8_t)(h >> 63);
    } else {
      double u = (double)(h >> 40) * (1.0 / 16777216.0);
      static_cast<float*>(out)[i] = (float)((double)lo + (double)width * u);
    }
  }
}

}  // namespace

extern "C" int synth_fill(void* dev_out, int dist, int64_t n, uint64_t seed, float lo,
                          float width, void* stream) {
  if (dev_out == nullptr || n <= 0 || (dist != 0 && dist != 1)) return -1;
  uint64_t total = (uint64_t)n * (uint64_t)n;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -3;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (total + 255) / 256;
  uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 32;
  if (blocks > cap) blocks = cap;
  fill_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(dev_out, dist, total, seed, lo,
                                                                 width);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
