// C ABI of the library (declared in include/fractal.h): plans, validation,
// launch geometry and the step drivers.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <type_traits>
#include <new>

#include <cudaTypedefs.h>

#include "../../include/fractal.h"
#include "launch.h"

namespace fractal {
namespace {

thread_local char g_last_cuda_error[256] = "";

int cuda_fail(cudaError_t e, const char* where) {
  std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", where, cudaGetErrorString(e));
  return FRACTAL_ECUDA;
}

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  while (e-- > 0) r *= b;
  return r;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Allocations left before an injected failure (-1: none pending).
std::atomic<int> g_fail_after{-1};

}  // namespace

cudaError_t lib_malloc(void** p, size_t bytes) {
  int left = g_fail_after.load();
  while (left >= 0) {
    if (g_fail_after.compare_exchange_weak(left, left - 1)) {
      if (left == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

// p can be dereferenced by kernels on `device` at the same address: device
// or managed memory, or pinned host memory mapped into the device's address
// space (unified addressing).  Pageable host memory and unknown pointers are
// not.  Host-side query only: nothing touches the memory.
bool device_addressable(const void* p, int device) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the query's error
    return false;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
      return at.device == device;
    case cudaMemoryTypeManaged:
      return true;
    case cudaMemoryTypeHost:
      return at.devicePointer == p;
    default:
      return false;
  }
}

namespace {

// p is device memory (not host memory mapped into the device).
bool on_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice;
}

constexpr int kMaxLevelsPerCta = 5;
constexpr int kMaxSmem = 200 * 1024;
// Loads per thread a launch is sized for (at most kIPT; fewer keeps more warps
// for the update phase).
constexpr int kLoadsPerThread = 2;

}  // namespace
}  // namespace fractal

using namespace fractal;

struct fractal_plan_s {
  int k = 0, log_rho = 0, rb = 0, mode = 0;
  int32_t n = 1;
  int device = 0;
  int sched = FRACTAL_SCHED_AUTO;
  int m[2] = {0, 0};            // tile levels per CTA, per dtype
  Launch step[2];               // staged CA (u8) / diffusion (f32) kernels
  Launch tma[2];                // TMA-staged CA / diffusion kernels
  bool tma_ok[2] = {false, false};
  Launch aux[2];                // SW / reduce kernels (slot table only in shared memory)
  int spl[2] = {1, 1};          // steps per launch (temporal fusion), per dtype
  bool kappa_fused = true;      // double-float conductivity steps temporally fused (k >= 4)
  bool user_levels[2] = {false, false};  // tile levels fixed by the caller
  Launch fused[2];              // fused kernel launch for the plan's steps per launch
  bool fused_ok[2] = {false, false};
  float* d_pack[2] = {nullptr, nullptr};  // float32 fused: compact records between launches
  size_t pack_cap = 0;          // bytes per record buffer
  uint32_t* d_bits[2] = {nullptr, nullptr};  // uint8 fused: bit records between launches
  size_t bits_cap = 0;          // bytes per bit-record buffer
  int4* d_desc = nullptr;       // float32 fused: per-thread setup of the current fused launch
  size_t desc_cap = 0;          // bytes
  bool desc_ok = false;         // d_desc matches fused[FRACTAL_F32] and its margin
  int* d_err = nullptr;         // device error word of the TMA kernels
  void* d_partials = nullptr;   // reduce scratch: one 8-byte partial per CTA
  size_t partials_cap = 0;      // elements
  double* d_result = nullptr;
  double* h_result = nullptr;   // pinned
};

namespace {

// Geometry for one dtype at `levels` tile levels per CTA; returns false if it
// does not fit (grid limits, shared memory).  `tma` receives the TMA-staged
// step kernel's launch and `tma_ok` whether that kernel applies (rows of at
// least 16 bytes: float32 rho >= 4, uint8 rho >= 16).
bool make_launch(const fractal_plan_s& p, int dtype, int levels, Launch& step, Launch& aux, Launch& tma,
                 bool& tma_ok) {
  return plan_geometry(p.k, p.log_rho, p.mode, dtype, levels, step, aux, tma, tma_ok);
}

// Largest steps per launch of the fused kernels: float32 margins of 8 to 128
// cells (whole 8 x 8 blocks, a power of two of them); uint8 margins of up to
// 31 cells (one word column of the bit image).
int max_spl(int dtype) { return dtype == FRACTAL_U8 ? 31 : 128; }

// Launch of the temporally fused kernel for `spl` steps per launch (super-tile
// side >= twice the margin).  The float32 kernel (rho >= 4) keeps one 8 x 8
// block per thread, the uint8 kernel at most a few 32-row word columns per
// warp, so either may take fewer tile levels per CTA than the plan's `step`.
// False if none fits.
bool make_fused(const fractal_plan_s& p, int dtype, int spl, const Launch& step, Launch& fused) {
  if (spl < 2 || spl > max_spl(dtype)) return false;
  if (dtype == FRACTAL_U8) {
    for (int m = step.geo.m; m >= 0; --m) {
      Launch st, aux, tma;
      bool tok = false;
      if (!plan_geometry(p.k, p.log_rho, p.mode, dtype, m, st, aux, tma, tok)) continue;
      const int threads = ca_fused_threads(st.geo, spl);
      const int smem = ca_fused_smem_bytes(st.geo, spl);
      if (threads > 0 && smem <= kMaxSmem) {
        fused = st;
        fused.threads = threads;
        fused.smem = smem;
        return true;
      }
      if (st.geo.T < 2 * spl) break;
    }
    return false;
  }
  // float32: the largest super-tile the kernel takes (at most 512 threads),
  // whatever the plan's step kernels use
  (void)step;
  const int rho = 1 << p.log_rho;
  const int margin = fused_margin(spl);
  if (rho < 4) return false;
  // margins up to 16 cells: super-tiles of side 128, one warp per CTA
  if (margin <= 16 && rho <= 128 && (128 >> p.log_rho) >= 1) {
    Launch st;
    const int m = 7 - p.log_rho;
    if (m <= kMaxLevelsPerCta && supertile_grid(p.k, p.log_rho, p.mode, m, st) &&
        fused_threads(st.geo, rho, margin, spl) == fused_warp_slots()) {
      fused = st;
      fused.threads = fused_warp_slots();
      fused.smem = 0;
      return true;
    }
  }
  for (int m = kMaxLevelsPerCta; m >= 0; --m) {
    Launch st;
    if (!supertile_grid(p.k, p.log_rho, p.mode, m, st)) continue;
    if (st.geo.T < 2 * margin) break;
    const int threads = fused_threads(st.geo, rho, margin, spl);
    const int smem = fused_smem_bytes(st.geo, margin, spl);
    if (threads > 0 && smem <= kMaxSmem) {
      fused = st;
      fused.threads = threads;
      fused.smem = smem;
      return true;
    }
  }
  return false;
}
}  // namespace

bool fractal::supertile_grid(int k, int log_rho, int mode, int levels, Launch& L) {
  const int rb = k - log_rho;
  if (levels < 0 || levels > rb || levels > kMaxLevelsPerCta) return false;
  const int R = rb - levels;
  Geo g;
  g.n = 1 << k;
  g.m = levels;
  g.R = R;
  g.T = (1 << log_rho) << levels;
  g.slots = (int)(mode == kLambda ? ipow(3, levels) : ipow(4, levels));
  g.lw = (int)ipow(3, (levels + 1) / 2);
  g.tiles = (int)ipow(3, levels);
  if (mode == kLambda) {
    L.grid = dim3((unsigned)ipow(3, (R + 1) / 2), (unsigned)ipow(3, R / 2), 1);
  } else {
    if (R > 15) return false;  // gridDim.y <= 65535
    L.grid = dim3(1u << R, 1u << R, 1);
  }
  L.geo = g;
  L.threads = 0;
  L.smem = 0;
  return true;
}

bool fractal::plan_geometry(int k, int log_rho, int mode, int dtype, int levels, Launch& step, Launch& aux, Launch& tma,
                   bool& tma_ok) {
  struct {
    int k, log_rho, rb, mode;
    int32_t n;
  } p{k, log_rho, k - log_rho, mode, 1 << k};
  if (levels < 0 || levels > p.rb || levels > kMaxLevelsPerCta) return false;
  const int R = p.rb - levels;
  const int rho = 1 << p.log_rho;
  Geo g;
  g.n = p.n;
  g.m = levels;
  g.R = R;
  g.T = rho << levels;
  g.slots = (int)(p.mode == kLambda ? ipow(3, levels) : ipow(4, levels));
  g.lw = (int)ipow(3, (levels + 1) / 2);
  g.tiles = (int)ipow(3, levels);
  dim3 grid;
  if (p.mode == kLambda) {
    grid = dim3((unsigned)ipow(3, (R + 1) / 2), (unsigned)ipow(3, R / 2), 1);
  } else {
    if (R > 15) return false;  // gridDim.y <= 65535
    grid = dim3(1u << R, 1u << R, 1);
  }
  // Vector accesses per tile: uint8 rows in pieces of at most 16 bytes, float
  // rows in float4s.  A staging pass of kIPT loads per thread covers the
  // whole super-tile.
  const int wc = dtype == FRACTAL_U8 ? (rho < 16 ? rho : 16) : (rho < 4 ? rho : 4);
  const int64_t chunks = (int64_t)g.slots * rho * (rho / wc);
  int threads = (int)(((chunks + kLoadsPerThread - 1) / kLoadsPerThread + 31) / 32 * 32);
  if (threads < 32) threads = 32;
  if (threads > 512) threads = 512;
  const int tab_bytes = tab_words(g.slots) * 4;
  int smem;
  if (dtype == FRACTAL_U8) {
    smem = tab_bytes + (g.T + 2) * ((g.T >> 5) + 3) * 4;
  } else {
    smem = tab_bytes + (g.T + 2) * (((g.T + 3) & ~3) + 8) * 4;
  }
  if (smem > kMaxSmem) return false;
  step.grid = grid;
  step.threads = threads;
  step.smem = smem;
  step.geo = g;
  aux = step;
  aux.smem = tab_bytes;
  // TMA-staged kernel: uint8 one thread per tile row, float32 one per 4x4 cells
  tma_ok = dtype == FRACTAL_U8 ? rho >= 16 : rho >= 4;
  tma = step;
  if (tma_ok) {
    // one thread per tile row (uint8) or per 4-column strip of a tile
    // (float32), capped at the kernels' launch bounds (the update loop
    // strides over the rest)
    const int64_t items = dtype == FRACTAL_U8 ? (int64_t)g.tiles * rho : (int64_t)g.tiles * (rho / 4);
    const int cap = dtype == FRACTAL_U8 ? 512 : 256;
    int t = (int)((items + 31) / 32 * 32);
    if (t > cap) t = cap;
    tma.threads = t;
    tma.smem = tma_smem_bytes(g, rho * rho * (dtype == FRACTAL_U8 ? 1 : 4), dtype);
    if (tma.smem > kMaxSmem) tma_ok = false;
  }
  return true;
}

int fractal::default_cta_levels(int k, int log_rho, int mode, int dtype) {
  // Super-tile side: the TMA kernels (uint8 rho >= 16, float32 rho >= 4) keep
  // the whole super-tile in flight, 256 uint8 / 128 float cells per side; the
  // vector-load kernels stage an image of it, 128 uint8 / 64 float cells.
  const int rb = k - log_rho;
  const int rho = 1 << log_rho;
  const bool tma = dtype == FRACTAL_U8 ? rho >= 16 : rho >= 4;
  const int target = dtype == FRACTAL_U8 ? (tma ? 8 : 7) : (tma ? 7 : 6);
  int m = target - log_rho;
  if (m < 0) m = 0;
  if (m > rb) m = rb;
  if (m > kMaxLevelsPerCta) m = kMaxLevelsPerCta;
  if (mode == kBB && rb - m > 15) m = rb - 15;
  return m;
}

namespace {

// Tensor map of an n x n array for bw x bh boxes (driver entry point).
bool encode_box_map(CUtensorMap* map, const void* base, int n, int bw, int bh, int dtype) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int e = dtype == FRACTAL_U8 ? 1 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)n * e};
  cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, dtype == FRACTAL_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                      const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// rho x rho tile boxes and 16-byte ring boxes of one array.
bool encode_maps(CUtensorMap* tile, CUtensorMap* ring, const void* base, int n, int rho, int dtype) {
  return encode_box_map(tile, base, n, rho, rho, dtype) &&
         encode_box_map(ring, base, n, dtype == FRACTAL_U8 ? 16 : 4, 1, dtype);
}

bool use_tma(const fractal_plan_s* p, int dtype) {
  return p->tma_ok[dtype] && p->sched != FRACTAL_SCHED_STAGED;
}

int default_levels(const fractal_plan_s& p, int dtype) { return default_cta_levels(p.k, p.log_rho, p.mode, dtype); }

// The float32 reduce runs one 8 x 8 block per thread (its own super-tiles)
// unless the caller fixed the tile levels of the plan, which then hold for
// it too (rho-tiles per CTA, the paper's setting at levels 0).
bool use_blocks(const fractal_plan_s* p, int dtype, Launch& B, int& levels) {
  return dtype == FRACTAL_F32 && !p->user_levels[FRACTAL_F32] && p->log_rho >= 2 &&
         blocks_geometry(p->k, p->mode, B, levels);
}

// A pair of device buffers of `need` bytes each, allocated once (kept while
// large enough).
template <typename T>
int ensure_pair(T* (&buf)[2], size_t& cap, size_t need) {
  if (need == 0 || need <= cap) return FRACTAL_OK;
  for (int i = 0; i < 2; ++i) {
    if (buf[i]) cudaFree(buf[i]);
    buf[i] = nullptr;
  }
  cap = 0;
  for (int i = 0; i < 2; ++i) {
    if (lib_malloc(&buf[i], need) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < 2; ++j) {
        if (buf[j]) cudaFree(buf[j]);
        buf[j] = nullptr;
      }
      return FRACTAL_ENOMEM;
    }
  }
  cap = need;
  return FRACTAL_OK;
}

// The two record buffers of the fused launches of `dtype`: float32 3^(k-3)
// block records of 112 bytes (179 MB at k = 16), uint8 3^(k-5) word-tile
// records of 128 bytes (22.7 MB at k = 16).
int ensure_records(fractal_plan_s* p, int dtype) {
  if (dtype == FRACTAL_F32)
    return ensure_pair(p->d_pack, p->pack_cap, (size_t)fused_records(p->k) * (size_t)fused_record_bytes());
  return ensure_pair(p->d_bits, p->bits_cap, (size_t)ca_records(p->k) * 128);
}

// Descriptors of the float32 fused launch (fused[FRACTAL_F32], margin of
// spl[FRACTAL_F32]): written by one launch of the describe kernel on `s`
// (then waited for when `sync`); every later fused launch reads its threads'
// setup from them.  16 bytes per thread (37 MB at k = 16, rho = 8).
int build_descriptors(fractal_plan_s* p, cudaStream_t s, bool sync) {
  p->desc_ok = false;
  // no launch of this plan may still read the descriptors being replaced
  if (sync && cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(cudaGetLastError(), "describe");
  const Launch& F = p->fused[FRACTAL_F32];
  const size_t need = (size_t)fused_descriptors(F) * sizeof(int4);
  if (need > p->desc_cap) {
    if (p->d_desc) cudaFree(p->d_desc);
    p->d_desc = nullptr;
    p->desc_cap = 0;
    if (lib_malloc(&p->d_desc, need) != cudaSuccess) {
      cudaGetLastError();
      p->d_desc = nullptr;
      return FRACTAL_ENOMEM;
    }
    p->desc_cap = need;
  }
  cudaError_t e = launch_fused_describe(p->mode, p->log_rho, fused_margin(p->spl[FRACTAL_F32]), p->spl[FRACTAL_F32], F,
                                        p->d_desc, s);
  if (e == cudaSuccess && sync) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "describe");
  p->desc_ok = true;
  return FRACTAL_OK;
}

int ensure_partials(fractal_plan_s* p) {
  size_t need = 1;
  {
    Launch B;
    int levels = 0;
    if (use_blocks(p, FRACTAL_F32, B, levels)) need = (size_t)B.grid.x * B.grid.y;
  }
  for (int d = 0; d < 2; ++d) {
    const size_t c = (size_t)p->aux[d].grid.x * p->aux[d].grid.y;
    if (c > need) need = c;
    const size_t f = p->fused_ok[d] ? (size_t)p->fused[d].grid.x * p->fused[d].grid.y : 0;
    if (f > need) need = f;
  }
  if (need <= p->partials_cap) return FRACTAL_OK;
  void* buf = nullptr;
  cudaError_t e = lib_malloc(&buf, need * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FRACTAL_ENOMEM;
  }
  if (p->d_partials) cudaFree(p->d_partials);
  p->d_partials = buf;
  p->partials_cap = need;
  return FRACTAL_OK;
}

int check_plan(const fractal_plan_s* p) { return p ? FRACTAL_OK : FRACTAL_EINVAL; }

}  // namespace

namespace {

// L launches of at most spl steps with the parity of `steps`, for fused
// calls that ping-pong a and b without records (the result lands where the
// single-step ping-pong would leave it): steps per launch i.
struct FusedSplit {
  int L, base, extra;
  FusedSplit(int steps, int spl) {
    L = (steps + spl - 1) / spl;
    if ((L & 1) != (steps & 1)) ++L;
    base = steps / L;
    extra = steps % L;
  }
  int of(int i) const { return base + (i < extra ? 1 : 0); }
};

// Launches of a fused call of `steps` steps at `spl` per launch when the
// state stays in records between them: ceil(steps / spl), but two when one
// launch would have to end where it started (an even number of steps).
int fused_launches(int steps, int spl) {
  const int L = (steps + spl - 1) / spl;
  return L == 1 && (steps & 1) == 0 ? 2 : L;
}

// `steps` automaton steps; with dev_count, also the alive count of the result
// (fused into the last launch of the fused kernel, else a reduce after).
int step_ca(fractal_plan_t p, uint8_t* a, uint8_t* b, int steps, double* dev_count, void* stream) {
  if (check_plan(p) || !a || !b || a == b || !aligned16(a) || !aligned16(b) || steps < 0)
    return FRACTAL_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  uint8_t* buf[2] = {a, b};
  if (steps > 0 && p->spl[FRACTAL_U8] > 1 && p->fused_ok[FRACTAL_U8]) {
    const int spl = p->spl[FRACTAL_U8];
    if (p->d_bits[0] && p->d_bits[1]) {
      // between launches the state stays in the bit records (the first
      // launch reads a, the last one writes the result buffer)
      const int L = fused_launches(steps, spl), base = steps / L, extra = steps % L;
      for (int i = 0; i < L; ++i) {
        const bool first = i == 0, last = i == L - 1;
        auto* part = last && dev_count ? static_cast<unsigned long long*>(p->d_partials) : nullptr;
        cudaError_t e = launch_ca_fused(p->mode, p->fused[FRACTAL_U8], first ? a : nullptr,
                                        last ? buf[steps & 1] : nullptr, base + (i < extra ? 1 : 0), spl, st, part,
                                        first ? nullptr : p->d_bits[(i - 1) & 1], last ? nullptr : p->d_bits[i & 1]);
        if (e != cudaSuccess) return cuda_fail(e, "step_ca");
      }
    } else {  // no records: ping-pong of a and b, the launches' parity that of steps
      const FusedSplit sp(steps, spl);
      for (int i = 0; i < sp.L; ++i) {
        auto* part = i == sp.L - 1 && dev_count ? static_cast<unsigned long long*>(p->d_partials) : nullptr;
        cudaError_t e = launch_ca_fused(p->mode, p->fused[FRACTAL_U8], buf[i & 1], buf[(i + 1) & 1], sp.of(i), spl,
                                        st, part);
        if (e != cudaSuccess) return cuda_fail(e, "step_ca");
      }
    }
    if (dev_count) {
      const Launch& F = p->fused[FRACTAL_U8];
      cudaError_t e = launch_final_sum(0, p->d_partials, (int64_t)F.grid.x * F.grid.y, dev_count, st);
      if (e != cudaSuccess) return cuda_fail(e, "step_ca count");
    }
    return FRACTAL_OK;
  }
  if (steps > 0 && use_tma(p, FRACTAL_U8)) {
    CUtensorMap maps[2], rings[2];
    const int rho = 1 << p->log_rho;
    if (!encode_maps(&maps[0], &rings[0], a, p->n, rho, FRACTAL_U8) ||
        !encode_maps(&maps[1], &rings[1], b, p->n, rho, FRACTAL_U8))
      return cuda_fail(cudaErrorInvalidValue, "tensor map");
    for (int s = 0; s < steps; ++s) {
      cudaError_t e = launch_ca_tma(p->mode, p->log_rho, p->tma[FRACTAL_U8], maps[s & 1], rings[s & 1],
                                    buf[(s + 1) & 1], p->d_err, st);
      if (e != cudaSuccess) return cuda_fail(e, "step_ca");
    }
  } else {
    for (int s = 0; s < steps; ++s) {
      cudaError_t e = launch_ca(p->mode, p->log_rho, p->step[FRACTAL_U8], buf[s & 1], buf[(s + 1) & 1], st);
      if (e != cudaSuccess) return cuda_fail(e, "step_ca");
    }
  }
  if (!dev_count) return FRACTAL_OK;
  cudaError_t e = launch_reduce(p->mode, p->log_rho, FRACTAL_U8, p->aux[FRACTAL_U8], buf[steps & 1], p->d_partials,
                                dev_count, st);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "step_ca count");
}

// `steps` diffusion steps from a (the result in a for even steps, in b for
// odd); with dev_sums, the global sum of the state after every `every` steps
// (steps / every values; steps must be a multiple of every).
int step_diffusion(fractal_plan_t p, float* a, float* b, float coef, int steps, int every, double* dev_sums,
                   void* stream) {
  if (check_plan(p) || !a || !b || a == b || !aligned16(a) || !aligned16(b) || steps < 0 || every < 1 ||
      steps % every != 0 || !std::isfinite(coef))
    return FRACTAL_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  float* buf[2] = {a, b};
  const int nseg = steps / every;
  if (steps > 0 && p->spl[FRACTAL_F32] > 1 && p->fused_ok[FRACTAL_F32] && p->d_pack[0] && p->d_pack[1]) {
    // fused launches; between them the state stays in the compact records
    // (the first launch reads a, the last writes the result buffer), also
    // across the segments: the launch that ends a segment takes its sum
    const int spl = p->spl[FRACTAL_F32];
    const int per = nseg == 1 ? fused_launches(every, spl) : (every + spl - 1) / spl;
    const int total = nseg * per, base = every / per, extra = every % per;
    const Launch& F = p->fused[FRACTAL_F32];
    const int4* desc = p->desc_ok ? p->d_desc : nullptr;
    for (int i = 0; i < total; ++i) {
      const int seg = i / per, l = i % per;
      const bool first = i == 0, last = i == total - 1;
      double* part = l == per - 1 && dev_sums ? static_cast<double*>(p->d_partials) : nullptr;
      cudaError_t e = launch_diffusion_fused(p->mode, p->log_rho, fused_margin(spl), spl, F, first ? a : nullptr,
                                             last ? buf[steps & 1] : nullptr, coef, base + (l < extra ? 1 : 0), st,
                                             part, first ? nullptr : p->d_pack[(i - 1) & 1],
                                             last ? nullptr : p->d_pack[i & 1], desc);
      if (e == cudaSuccess && part)
        e = launch_final_sum(1, p->d_partials, (int64_t)F.grid.x * F.grid.y, dev_sums + seg, st);
      if (e != cudaSuccess) return cuda_fail(e, "step_diffusion");
    }
    return FRACTAL_OK;
  }
  // one launch per step; after each segment a reduce of its result
  CUtensorMap maps[2], rings[2];
  const bool tma = steps > 0 && use_tma(p, FRACTAL_F32);
  if (tma) {
    const int rho = 1 << p->log_rho;
    if (!encode_maps(&maps[0], &rings[0], a, p->n, rho, FRACTAL_F32) ||
        !encode_maps(&maps[1], &rings[1], b, p->n, rho, FRACTAL_F32))
      return cuda_fail(cudaErrorInvalidValue, "tensor map");
  }
  for (int s = 0; s < steps; ++s) {
    cudaError_t e = tma ? launch_diffusion_tma(p->mode, p->log_rho, p->tma[FRACTAL_F32], maps[s & 1], rings[s & 1],
                                               buf[(s + 1) & 1], coef, p->d_err, st)
                        : launch_diffusion(p->mode, p->log_rho, p->step[FRACTAL_F32], buf[s & 1], buf[(s + 1) & 1],
                                           coef, st);
    if (e == cudaSuccess && dev_sums && (s + 1) % every == 0)
      e = launch_reduce(p->mode, p->log_rho, FRACTAL_F32, p->aux[FRACTAL_F32], buf[(s + 1) & 1], p->d_partials,
                        dev_sums + (s + 1) / every - 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "step_diffusion");
  }
  if (steps == 0 && dev_sums) {  // a zero-step call with a sum: the sum of a
    cudaError_t e = launch_reduce(p->mode, p->log_rho, FRACTAL_F32, p->aux[FRACTAL_F32], a, p->d_partials, dev_sums, st);
    if (e != cudaSuccess) return cuda_fail(e, "step_diffusion sum");
  }
  return FRACTAL_OK;
}

// Record form: the state of a fused configuration as the compact records its
// launches keep between them (float32: 112-byte block records; uint8:
// 128-byte bit records of word tiles), indexed by the configuration's
// super-tiles.  The fused kernels convert with zero steps.
bool records_config(const fractal_plan_s* p, int dtype) {
  return (dtype == FRACTAL_U8 || dtype == FRACTAL_F32) && p->spl[dtype] > 1 && p->fused_ok[dtype];
}

int64_t records_bytes(const fractal_plan_s* p, int dtype) {
  return dtype == FRACTAL_F32 ? fused_records(p->k) * (int64_t)fused_record_bytes() : ca_records(p->k) * 128;
}

// One fused call of the float32 diffusion from records rin to records rout
// (distinct buffers), the state in the plan's records between launches.
int diffusion_records_call(fractal_plan_t p, const float* rin, float* rout, float coef, int steps, int every,
                           double* dev_sums, cudaStream_t st) {
  const int spl = p->spl[FRACTAL_F32];
  const int nseg = steps / every, per = (every + spl - 1) / spl;
  const int total = nseg * per, base = every / per, extra = every % per;
  const Launch& F = p->fused[FRACTAL_F32];
  const int4* desc = p->desc_ok ? p->d_desc : nullptr;
  for (int i = 0; i < total; ++i) {
    const int seg = i / per, l = i % per;
    const bool first = i == 0, last = i == total - 1;
    double* part = l == per - 1 && dev_sums ? static_cast<double*>(p->d_partials) : nullptr;
    cudaError_t e = launch_diffusion_fused(p->mode, p->log_rho, fused_margin(spl), spl, F, nullptr, nullptr, coef,
                                           base + (l < extra ? 1 : 0), st, part,
                                           first ? rin : p->d_pack[(i - 1) & 1], last ? rout : p->d_pack[i & 1],
                                           desc);
    if (e == cudaSuccess && part)
      e = launch_final_sum(1, p->d_partials, (int64_t)F.grid.x * F.grid.y, dev_sums + seg, st);
    if (e != cudaSuccess) return cuda_fail(e, "step_diffusion_records");
  }
  return FRACTAL_OK;
}

int ca_records_call(fractal_plan_t p, const uint32_t* rin, uint32_t* rout, int steps, double* dev_count,
                    cudaStream_t st) {
  const int spl = p->spl[FRACTAL_U8];
  const int L = (steps + spl - 1) / spl, base = steps / L, extra = steps % L;
  for (int i = 0; i < L; ++i) {
    const bool first = i == 0, last = i == L - 1;
    auto* part = last && dev_count ? static_cast<unsigned long long*>(p->d_partials) : nullptr;
    cudaError_t e = launch_ca_fused(p->mode, p->fused[FRACTAL_U8], nullptr, nullptr, base + (i < extra ? 1 : 0), spl, st,
                                    part, first ? rin : p->d_bits[(i - 1) & 1], last ? rout : p->d_bits[i & 1]);
    if (e != cudaSuccess) return cuda_fail(e, "step_ca_records");
  }
  if (dev_count) {
    const Launch& F = p->fused[FRACTAL_U8];
    cudaError_t e = launch_final_sum(0, p->d_partials, (int64_t)F.grid.x * F.grid.y, dev_count, st);
    if (e != cudaSuccess) return cuda_fail(e, "step_ca_records count");
  }
  return FRACTAL_OK;
}

// Steps with per-cell conductivity, state type T (float or double).
template <typename T>
int step_kappa(fractal_plan_t p, T* a, T* b, const float* kappa, T coef, int steps, void* stream) {
  if (check_plan(p) || !a || !b || !kappa || a == b || (const void*)kappa == (const void*)a ||
      (const void*)kappa == (const void*)b || !aligned16(a) || !aligned16(b) || !aligned16(kappa) || steps < 0)
    return FRACTAL_EINVAL;
  Launch L;
  int levels = 0;
  if (!kappa_geometry(p->k, p->mode, L, levels)) return FRACTAL_EINVAL;
  if (steps == 0) return FRACTAL_OK;
  T* buf[2] = {a, b};
  if constexpr (std::is_same<T, dfloat>::value) {
    // double-float: temporally fused launches of up to `margin` steps,
    // ping-pong between a and b with the parity of `steps`
    Launch F;
    int margin = 0;
    if (p->kappa_fused && kappa_fused_geometry(p->k, p->mode, F, margin)) {
      const FusedSplit sp(steps, margin);
      const dfloat ha(0.5f * coef.hi, 0.5f * coef.lo);  // halving is exact
      for (int i = 0; i < sp.L; ++i) {
        cudaError_t e = launch_kappa_fused_df(p->mode, p->k, buf[i & 1], buf[(i + 1) & 1], nullptr, kappa, ha,
                                              sp.of(i), (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "step_diffusion_kappa");
      }
      return FRACTAL_OK;
    }
  }
  for (int s = 0; s < steps; ++s) {
    cudaError_t e =
        launch_diffusion_kappa<T>(p->mode, L, levels, buf[s & 1], buf[(s + 1) & 1], kappa, coef, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "step_diffusion_kappa");
  }
  return FRACTAL_OK;
}

template <typename T, typename G>
int adjoint_step(fractal_plan_t p, const T* u, const T* p_in, T* p_out, const float* kappa, G* gkappa, T coef,
                 void* stream) {
  if (check_plan(p) || !u || !p_in || !p_out || !kappa || !gkappa) return FRACTAL_EINVAL;
  const void* all[5] = {u, p_in, p_out, kappa, gkappa};
  for (int i = 0; i < 5; ++i) {
    if (!aligned16(all[i])) return FRACTAL_EINVAL;
    for (int j = 0; j < i; ++j)
      if (all[i] == all[j]) return FRACTAL_EINVAL;
  }
  Launch L;
  int levels = 0;
  if (!kappa_geometry(p->k, p->mode, L, levels)) return FRACTAL_EINVAL;
  cudaError_t e = launch_diffusion_adjoint<T>(p->mode, L, levels, u, p_in, p_out, kappa, gkappa, coef,
                                              (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "adjoint_diffusion_step");
}

}  // namespace

extern "C" {

const char* fractal_strerror(int status) {
  switch (status) {
    case FRACTAL_OK: return "ok";
    case FRACTAL_EINVAL: return "invalid argument";
    case FRACTAL_ENOMEM: return "out of memory";
    case FRACTAL_ECUDA: return "CUDA error";
    case FRACTAL_ETOOBIG: return "launch needs more partial sums than the fixed scratch array holds";
    default: return "unknown status";
  }
}

const char* fractal_last_cuda_error(void) { return g_last_cuda_error; }

int fractal_map(int k, int rho, int mode, fractal_plan_t* out) {
  if (out == nullptr) return FRACTAL_EINVAL;
  *out = nullptr;
  if (k < 0 || k > FRACTAL_MAX_LEVEL) return FRACTAL_EINVAL;
  if (rho < 1 || rho > 32 || (rho & (rho - 1)) != 0 || rho > (1 << k)) return FRACTAL_EINVAL;
  if (mode != FRACTAL_LAMBDA && mode != FRACTAL_BB) return FRACTAL_EINVAL;
  fractal_plan_s* p = new (std::nothrow) fractal_plan_s();
  if (!p) return FRACTAL_ENOMEM;
  p->k = k;
  p->log_rho = ilog2c(rho);
  p->rb = k - p->log_rho;
  p->mode = mode;
  p->n = 1 << k;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  for (int d = 0; d < 2; ++d) {
    p->m[d] = default_levels(*p, d);
    if (!make_launch(*p, d, p->m[d], p->step[d], p->aux[d], p->tma[d], p->tma_ok[d])) {
      delete p;
      return FRACTAL_EINVAL;
    }
  }
  int st = ensure_partials(p);
  if (st != FRACTAL_OK) {
    delete p;
    return st;
  }
  if (lib_malloc(&p->d_result, sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&p->h_result, sizeof(double)) != cudaSuccess || lib_malloc(&p->d_err, sizeof(int)) != cudaSuccess ||
      cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    fractal_plan_destroy(p);
    return FRACTAL_ENOMEM;
  }
  *out = p;
  return FRACTAL_OK;
}

int fractal_plan_destroy(fractal_plan_t p) {
  if (!p) return FRACTAL_OK;
  if (p->d_partials) cudaFree(p->d_partials);
  for (int i = 0; i < 2; ++i) {
    if (p->d_pack[i]) cudaFree(p->d_pack[i]);
    if (p->d_bits[i]) cudaFree(p->d_bits[i]);
  }
  if (p->d_desc) cudaFree(p->d_desc);
  if (p->d_result) cudaFree(p->d_result);
  if (p->h_result) cudaFreeHost(p->h_result);
  if (p->d_err) cudaFree(p->d_err);
  delete p;
  return FRACTAL_OK;
}

int fractal_plan_get_info(fractal_plan_t p, fractal_plan_info* info) {
  if (!p || !info) return FRACTAL_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->k = p->k;
  info->rho = 1 << p->log_rho;
  info->mode = p->mode;
  info->r_b = p->rb;
  info->n = p->n;
  info->n_b = (int64_t)1 << p->rb;
  info->grid_w = (int32_t)ipow(3, (p->rb + 1) / 2);
  info->grid_h = (int32_t)ipow(3, p->rb / 2);
  info->member_tiles = ipow(3, p->rb);
  info->members = ipow(3, p->k);
  for (int d = 0; d < 2; ++d) {
    // the kernel a step call launches: fused, TMA-staged or vector-staged
    const bool fused = p->spl[d] > 1 && p->fused_ok[d];
    const Launch& L = fused ? p->fused[d] : (use_tma(p, d) ? p->tma[d] : p->step[d]);
    info->cta_levels[d] = L.geo.m;
    info->ctas[d] = (int64_t)L.grid.x * L.grid.y;
    info->threads[d] = L.threads;
    info->smem_bytes[d] = L.smem;
    info->tma[d] = !fused && use_tma(p, d) ? 1 : 0;
    info->steps_per_launch[d] = fused ? p->spl[d] : 1;
  }
  info->sched = p->sched;
  return FRACTAL_OK;
}

static int set_levels(fractal_plan_t p, int dtype, int levels);

int fractal_plan_set_cta_levels(fractal_plan_t p, int dtype, int levels) {
  const int st = set_levels(p, dtype, levels);
  if (st == FRACTAL_OK) p->user_levels[dtype] = true;
  return st;
}

static int set_levels(fractal_plan_t p, int dtype, int levels) {
  if (!p || (dtype != FRACTAL_U8 && dtype != FRACTAL_F32)) return FRACTAL_EINVAL;
  Launch s, a, t;
  bool ok = false;
  if (!make_launch(*p, dtype, levels, s, a, t, ok)) return FRACTAL_EINVAL;
  const Launch old_s = p->step[dtype], old_a = p->aux[dtype], old_t = p->tma[dtype], old_f = p->fused[dtype];
  const int old_m = p->m[dtype];
  const bool old_ok = p->tma_ok[dtype], old_fok = p->fused_ok[dtype];
  p->step[dtype] = s;
  p->aux[dtype] = a;
  p->tma[dtype] = t;
  p->tma_ok[dtype] = ok;
  p->m[dtype] = levels;
  p->fused_ok[dtype] = p->spl[dtype] > 1 && make_fused(*p, dtype, p->spl[dtype], s, p->fused[dtype]);
  int st = ensure_partials(p);
  if (st != FRACTAL_OK) {
    p->step[dtype] = old_s;
    p->aux[dtype] = old_a;
    p->tma[dtype] = old_t;
    p->tma_ok[dtype] = old_ok;
    p->m[dtype] = old_m;
    p->fused[dtype] = old_f;
    p->fused_ok[dtype] = old_fok;
  }
  return st;
}

int fractal_fused_box_blocks(int supertile, int margin, int reach) {
  if (supertile < 16 || supertile > 256 || (supertile & (supertile - 1)) != 0 || margin < 8 || margin > 128 ||
      (margin & (margin - 1)) != 0 || 2 * margin > supertile || reach < 1 || reach > margin)
    return FRACTAL_EINVAL;
  return box_cap_reach(ilog2c(supertile) - 3, margin / 8, reach);
}

int fractal_plan_set_steps_per_launch(fractal_plan_t p, int dtype, int spl) {
  if (!p || (dtype != FRACTAL_U8 && dtype != FRACTAL_F32) || spl < 1 || spl > max_spl(dtype)) return FRACTAL_EINVAL;
  if (dtype == FRACTAL_F32) p->desc_ok = false;
  if (spl == 1) {
    p->spl[dtype] = 1;
    p->fused_ok[dtype] = false;
    return FRACTAL_OK;
  }
  Launch f;
  if (!make_fused(*p, dtype, spl, p->step[dtype], f)) return FRACTAL_EINVAL;
  const int old_spl = p->spl[dtype];
  const bool old_ok = p->fused_ok[dtype];
  const Launch old_f = p->fused[dtype];
  p->spl[dtype] = spl;
  p->fused[dtype] = f;
  p->fused_ok[dtype] = true;
  int st = ensure_partials(p);  // the fused kernels' per-CTA sums
  if (st == FRACTAL_OK) st = ensure_records(p, dtype);
  if (st == FRACTAL_OK && dtype == FRACTAL_F32) st = build_descriptors(p, nullptr, true);
  if (st != FRACTAL_OK) {
    // the previous configuration stays in force (its partials still fit;
    // without records or descriptors its launches ping-pong the caller's
    // buffers and compute their threads' setup themselves)
    p->spl[dtype] = old_spl;
    p->fused_ok[dtype] = old_ok;
    p->fused[dtype] = old_f;
  }
  return st;
}

int fractal_plan_set_schedule(fractal_plan_t p, int sched) {
  if (!p || (sched != FRACTAL_SCHED_AUTO && sched != FRACTAL_SCHED_STAGED && sched != FRACTAL_SCHED_TMA))
    return FRACTAL_EINVAL;
  if (sched == FRACTAL_SCHED_TMA && !(p->tma_ok[0] || p->tma_ok[1])) return FRACTAL_EINVAL;
  p->sched = sched;
  return FRACTAL_OK;
}

int fractal_plan_autotune(fractal_plan_t p, int dtype, const void* dev_in, void* dev_scratch, int reps,
                          float* best_us, void* stream) {
  if (check_plan(p) || (dtype != FRACTAL_U8 && dtype != FRACTAL_F32) || !dev_in || !dev_scratch ||
      dev_in == dev_scratch || !aligned16(dev_in) || !aligned16(dev_scratch) || reps < 1)
    return FRACTAL_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return FRACTAL_ENOMEM;
  }
  const int old_sched = p->sched, old_m = p->m[dtype], old_spl = p->spl[dtype];
  float best = -1.0f;
  int best_sched = old_sched, best_m = old_m, best_spl = old_spl;
  // best single-step candidate: its tile levels also serve the single-write
  // and reduce kernels when the float32 fused kernel (own super-tile) wins
  float best1 = -1.0f;
  int best1_m = old_m;
  int status = FRACTAL_OK;
  // One timed unit dev_in -> dev_scratch: a single step; `spl` fused steps;
  // with records, the launches of a call of 100 steps (2 spl when longer)
  // as the step driver runs them -- the first from dev_in, the last into
  // dev_scratch, records between -- so that the middle launches count too.
  // Returns the steps in `done`.
  const bool records = ensure_records(p, dtype) == FRACTAL_OK;
  auto launch = [&](int spl, int& done) -> int {
    done = spl;
    if (spl > 1 && records) {
      const int S = spl <= 50 ? 100 : 2 * spl;
      const int L = fused_launches(S, spl), base = S / L, extra = S % L;
      const Launch& F = p->fused[dtype];
      const int4* desc = p->desc_ok ? p->d_desc : nullptr;
      cudaError_t e = cudaSuccess;
      for (int i = 0; i < L && e == cudaSuccess; ++i) {
        const bool first = i == 0, last = i == L - 1;
        const int ns = base + (i < extra ? 1 : 0);
        if (dtype == FRACTAL_U8) {
          e = launch_ca_fused(p->mode, F, first ? (const uint8_t*)dev_in : nullptr,
                              last ? (uint8_t*)dev_scratch : nullptr, ns, spl, st, nullptr,
                              first ? nullptr : p->d_bits[(i - 1) & 1], last ? nullptr : p->d_bits[i & 1]);
        } else {
          e = launch_diffusion_fused(p->mode, p->log_rho, fused_margin(spl), spl, F,
                                     first ? (const float*)dev_in : nullptr, last ? (float*)dev_scratch : nullptr,
                                     0.2f, ns, st, nullptr, first ? nullptr : p->d_pack[(i - 1) & 1],
                                     last ? nullptr : p->d_pack[i & 1], desc);
        }
      }
      done = S;
      return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "autotune");
    }
    if (spl > 1) {
      const cudaError_t e =
          dtype == FRACTAL_U8
              ? launch_ca_fused(p->mode, p->fused[dtype], (const uint8_t*)dev_in, (uint8_t*)dev_scratch, spl, spl, st)
              : launch_diffusion_fused(p->mode, p->log_rho, fused_margin(spl), spl, p->fused[dtype],
                                       (const float*)dev_in, (float*)dev_scratch, 0.2f, spl, st);
      return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "autotune");
    }
    return dtype == FRACTAL_U8 ? fractal_step_ca(p, (uint8_t*)dev_in, (uint8_t*)dev_scratch, 1, stream)
                               : fractal_step_diffusion(p, (float*)dev_in, (float*)dev_scratch, 0.2f, 1, stream);
  };
  bool f32_fused_timed = false;  // the float32 fused kernel picks its own super-tile: time it once
  for (int m = 0; m <= kMaxLevelsPerCta && m <= p->rb && status == FRACTAL_OK; ++m) {
    if (set_levels(p, dtype, m) != FRACTAL_OK) continue;
    const bool skip_f32_fused = dtype == FRACTAL_F32 && f32_fused_timed;
    f32_fused_timed = true;
    // candidates: (schedule, steps per launch)
    const int cands_f32[6][2] = {{FRACTAL_SCHED_STAGED, 1}, {FRACTAL_SCHED_TMA, 1}, {FRACTAL_SCHED_AUTO, 16},
                                 {FRACTAL_SCHED_AUTO, 25}, {FRACTAL_SCHED_AUTO, 50}, {FRACTAL_SCHED_AUTO, 100}};
    const int cands_u8[6][2] = {{FRACTAL_SCHED_STAGED, 1}, {FRACTAL_SCHED_TMA, 1}, {FRACTAL_SCHED_AUTO, 8},
                                {FRACTAL_SCHED_AUTO, 16}, {FRACTAL_SCHED_AUTO, 25}, {FRACTAL_SCHED_AUTO, 31}};
    const int(*cands)[2] = dtype == FRACTAL_U8 ? cands_u8 : cands_f32;
    for (int ci = 0; ci < 6 && status == FRACTAL_OK; ++ci) {
      const int sched = cands[ci][0], spl = cands[ci][1];
      if (sched == FRACTAL_SCHED_TMA && !p->tma_ok[dtype]) continue;
      if (spl > 1 && skip_f32_fused) continue;
      if (spl > 1) {
        if (!make_fused(*p, dtype, spl, p->step[dtype], p->fused[dtype])) continue;
        p->spl[dtype] = spl;
        p->fused_ok[dtype] = true;
        if (dtype == FRACTAL_F32) build_descriptors(p, st, false);  // on failure: the kernels' own setup
      } else {
        p->spl[dtype] = 1;
        p->fused_ok[dtype] = false;
      }
      p->sched = sched;
      int done = spl;
      for (int i = 0; i < 2 && status == FRACTAL_OK; ++i) status = launch(spl, done);
      if (status != FRACTAL_OK) break;
      if (cudaEventRecord(e0, st) != cudaSuccess) { status = cuda_fail(cudaGetLastError(), "autotune"); break; }
      for (int i = 0; i < reps && status == FRACTAL_OK; ++i) status = launch(spl, done);
      if (status != FRACTAL_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        status = cuda_fail(cudaGetLastError(), "autotune");
        break;
      }
      const float us = 1000.f * ms / (float)(reps * done);
      if (spl == 1 && (best1 < 0.f || us < best1)) {
        best1 = us;
        best1_m = m;
      }
      if (best < 0.f || us < best) {
        best = us;
        best_sched = sched;
        best_m = m;
        best_spl = spl;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // keep the winner (or restore the previous choice on failure)
  const bool ok = status == FRACTAL_OK && best >= 0.f;
  const bool own_tile = dtype == FRACTAL_F32 && best_spl > 1;
  set_levels(p, dtype, ok ? (own_tile ? best1_m : best_m) : old_m);
  p->sched = ok ? (best_sched == FRACTAL_SCHED_STAGED ? FRACTAL_SCHED_STAGED : FRACTAL_SCHED_AUTO) : old_sched;
  fractal_plan_set_steps_per_launch(p, dtype, ok ? best_spl : old_spl);
  if (ok && best_us) *best_us = best;
  return status;
}

int fractal_debug_fail_allocs(int after) {
  g_fail_after.store(after < 0 ? -1 : after);
  return FRACTAL_OK;
}

int fractal_plan_selftest_wait(fractal_plan_t p, unsigned spins, void* stream) {
  if (check_plan(p) || spins == 0 || spins > (1u << 22)) return FRACTAL_EINVAL;
  cudaError_t e = launch_wait_selftest(p->d_err, spins, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "wait self-test");
}

int fractal_plan_records_bytes(fractal_plan_t p, int dtype, int64_t* bytes) {
  if (check_plan(p) || !bytes || !records_config(p, dtype)) return FRACTAL_EINVAL;
  *bytes = records_bytes(p, dtype);
  return FRACTAL_OK;
}

int fractal_records_from_array(fractal_plan_t p, int dtype, const void* dev_embedded, void* dev_records,
                               void* stream) {
  if (check_plan(p) || !records_config(p, dtype) || !dev_embedded || !dev_records || dev_embedded == dev_records ||
      !aligned16(dev_embedded) || !aligned16(dev_records))
    return FRACTAL_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  const int spl = p->spl[dtype];
  cudaError_t e;
  if (dtype == FRACTAL_F32)  // a fused launch of no steps: stage from the array, write the records
    e = launch_diffusion_fused(p->mode, p->log_rho, fused_margin(spl), spl, p->fused[dtype],
                               static_cast<const float*>(dev_embedded), nullptr, 0.f, 0, st, nullptr, nullptr,
                               static_cast<float*>(dev_records), p->desc_ok ? p->d_desc : nullptr);
  else
    e = launch_ca_fused(p->mode, p->fused[dtype], static_cast<const uint8_t*>(dev_embedded), nullptr, 0, spl, st,
                        nullptr, nullptr, static_cast<uint32_t*>(dev_records));
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "records_from_array");
}

int fractal_records_to_array(fractal_plan_t p, int dtype, const void* dev_records, void* dev_embedded,
                             void* stream) {
  if (check_plan(p) || !records_config(p, dtype) || !dev_embedded || !dev_records || dev_embedded == dev_records ||
      !aligned16(dev_embedded) || !aligned16(dev_records))
    return FRACTAL_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  const int spl = p->spl[dtype];
  cudaError_t e;
  if (dtype == FRACTAL_F32)
    e = launch_diffusion_fused(p->mode, p->log_rho, fused_margin(spl), spl, p->fused[dtype], nullptr,
                               static_cast<float*>(dev_embedded), 0.f, 0, st, nullptr,
                               static_cast<const float*>(dev_records), nullptr, p->desc_ok ? p->d_desc : nullptr);
  else
    e = launch_ca_fused(p->mode, p->fused[dtype], nullptr, static_cast<uint8_t*>(dev_embedded), 0, spl, st, nullptr,
                        static_cast<const uint32_t*>(dev_records), nullptr);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "records_to_array");
}

int fractal_step_diffusion_records(fractal_plan_t p, const float* rec_in, float* rec_out, float coef, int steps,
                                   int every, double* dev_sums, void* stream) {
  if (check_plan(p) || !records_config(p, FRACTAL_F32) || !rec_in || !rec_out || rec_in == rec_out ||
      !aligned16(rec_in) || !aligned16(rec_out) || steps < 1 || every < 1 || steps % every != 0 ||
      !std::isfinite(coef))
    return FRACTAL_EINVAL;
  if (!p->d_pack[0] || !p->d_pack[1]) return FRACTAL_ENOMEM;
  return diffusion_records_call(p, rec_in, rec_out, coef, steps, every, dev_sums, (cudaStream_t)stream);
}

int fractal_step_ca_records(fractal_plan_t p, const void* rec_in, void* rec_out, int steps, double* dev_count,
                            void* stream) {
  if (check_plan(p) || !records_config(p, FRACTAL_U8) || !rec_in || !rec_out || rec_in == rec_out ||
      !aligned16(rec_in) || !aligned16(rec_out) || steps < 1)
    return FRACTAL_EINVAL;
  if (!p->d_bits[0] || !p->d_bits[1]) return FRACTAL_ENOMEM;
  return ca_records_call(p, static_cast<const uint32_t*>(rec_in), static_cast<uint32_t*>(rec_out), steps, dev_count,
                         (cudaStream_t)stream);
}

int fractal_plan_set_kappa_fusion(fractal_plan_t p, int on) {
  if (check_plan(p)) return FRACTAL_EINVAL;
  p->kappa_fused = on != 0;
  return FRACTAL_OK;
}

int fractal_kappa_fused_limits(int k, int mode, int64_t* record_floats, int* max_steps) {
  if (!record_floats || !max_steps || (mode != FRACTAL_LAMBDA && mode != FRACTAL_BB)) return FRACTAL_EINVAL;
  Launch L;
  int margin = 0;
  if (!kappa_fused_geometry(k, mode, L, margin)) return FRACTAL_EINVAL;
  *record_floats = kappa_record_float4s(k) * 4;
  *max_steps = margin;
  return FRACTAL_OK;
}

int fractal_kappa_trajectory_df_io(fractal_plan_t p, const void* dev_in, int in_format, void* dev_out,
                                   int out_format, float* dev_traj, const float* dev_kappa, double coef, int steps,
                                   void* stream) {
  if (check_plan(p) || !dev_in || !dev_kappa || (!dev_out && !dev_traj) || !std::isfinite(coef)) return FRACTAL_EINVAL;
  if ((in_format != FRACTAL_F32 && in_format != FRACTAL_DF) || (out_format != FRACTAL_F32 && out_format != FRACTAL_DF))
    return FRACTAL_EINVAL;
  const void* all[4] = {dev_in, dev_out, dev_traj, dev_kappa};
  for (int i = 0; i < 4; ++i) {
    if (all[i] && !aligned16(all[i])) return FRACTAL_EINVAL;
    for (int j = 0; j < i; ++j)
      if (all[i] && all[i] == all[j]) return FRACTAL_EINVAL;
  }
  Launch L;
  int margin = 0;
  if (!kappa_fused_geometry(p->k, p->mode, L, margin) || steps < 1 || steps > margin) return FRACTAL_EINVAL;
  const bool fin = in_format == FRACTAL_F32, fout = out_format == FRACTAL_F32;
  cudaError_t e = launch_kappa_fused_df(
      p->mode, p->k, fin ? nullptr : static_cast<const dfloat*>(dev_in),
      fout ? nullptr : static_cast<dfloat*>(dev_out), reinterpret_cast<float4*>(dev_traj), dev_kappa,
      dfloat_from_double(0.5 * coef), steps, (cudaStream_t)stream, fin ? static_cast<const float*>(dev_in) : nullptr,
      fout ? static_cast<float*>(dev_out) : nullptr);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "kappa_trajectory_df");
}

int fractal_kappa_trajectory_df(fractal_plan_t p, const float* dev_in, float* dev_out, float* dev_traj,
                                const float* dev_kappa, double coef, int steps, void* stream) {
  return fractal_kappa_trajectory_df_io(p, dev_in, FRACTAL_DF, dev_out, FRACTAL_DF, dev_traj, dev_kappa, coef, steps,
                                        stream);
}

int fractal_kappa_gradient_df_io(fractal_plan_t p, const float* dev_utraj, const float* dev_ptraj, float* dev_gkappa,
                                 int accumulate, float* dev_out_f32, double coef, int steps, void* stream) {
  if (check_plan(p) || !dev_utraj || !dev_ptraj || !std::isfinite(coef) || steps < 1) return FRACTAL_EINVAL;
  if (!dev_gkappa && (accumulate || !dev_out_f32)) return FRACTAL_EINVAL;
  const void* all[4] = {dev_utraj, dev_ptraj, dev_gkappa, dev_out_f32};
  for (int i = 0; i < 4; ++i) {
    if (all[i] && !aligned16(all[i])) return FRACTAL_EINVAL;
    for (int j = 0; j < i; ++j)
      if (all[i] && all[i] == all[j]) return FRACTAL_EINVAL;
  }
  Launch L;
  int margin = 0;
  if (!kappa_fused_geometry(p->k, p->mode, L, margin)) return FRACTAL_EINVAL;
  cudaError_t e = launch_kappa_grad_df(p->mode, p->k, reinterpret_cast<const float4*>(dev_utraj),
                                       reinterpret_cast<const float4*>(dev_ptraj), reinterpret_cast<dfloat*>(dev_gkappa),
                                       dfloat_from_double(0.5 * coef), steps, (cudaStream_t)stream,
                                       accumulate ? 1 : 0, dev_out_f32);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "kappa_gradient_df");
}

int fractal_kappa_gradient_df(fractal_plan_t p, const float* dev_utraj, const float* dev_ptraj, float* dev_gkappa,
                              double coef, int steps, void* stream) {
  if (!dev_gkappa) return FRACTAL_EINVAL;
  return fractal_kappa_gradient_df_io(p, dev_utraj, dev_ptraj, dev_gkappa, 1, nullptr, coef, steps, stream);
}

int fractal_plan_device_status(fractal_plan_t p, int* code) {
  if (!p || !code) return FRACTAL_EINVAL;
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "device status");
  *code = v;
  return FRACTAL_OK;
}

int fractal_map_blocks(fractal_plan_t p, int32_t* dev_xy, void* stream) {
  return fractal_map_blocks_method(p, dev_xy, FRACTAL_MAP_BALLOT, stream);
}

int fractal_map_blocks_method(fractal_plan_t p, int32_t* dev_xy, int method, void* stream) {
  if (check_plan(p) || !dev_xy || (reinterpret_cast<uintptr_t>(dev_xy) & 7u) != 0) return FRACTAL_EINVAL;
  if (method != FRACTAL_MAP_BALLOT && method != FRACTAL_MAP_SCALAR && method != FRACTAL_MAP_MMA)
    return FRACTAL_EINVAL;
  const int w = (int)ipow(3, (p->rb + 1) / 2), h = (int)ipow(3, p->rb / 2);
  cudaError_t e = launch_map_blocks(dev_xy, w, h, p->rb, (cudaStream_t)stream, method);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "map_blocks");
}

int fractal_map_write(fractal_plan_t p, void* dev_buf, int dtype, double value, void* stream) {
  if (check_plan(p) || !dev_buf || !aligned16(dev_buf)) return FRACTAL_EINVAL;
  if (dtype != FRACTAL_U8 && dtype != FRACTAL_F32) return FRACTAL_EINVAL;
  cudaError_t e = launch_sw(p->mode, p->log_rho, dtype, p->aux[dtype], dev_buf, value, (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "map_write");
}

int fractal_step_ca(fractal_plan_t p, uint8_t* a, uint8_t* b, int steps, void* stream) {
  return step_ca(p, a, b, steps, nullptr, stream);
}

int fractal_step_ca_count(fractal_plan_t p, uint8_t* a, uint8_t* b, int steps, double* dev_count, void* stream) {
  if (!dev_count) return FRACTAL_EINVAL;
  return step_ca(p, a, b, steps, dev_count, stream);
}

int fractal_step_diffusion(fractal_plan_t p, float* a, float* b, float coef, int steps, void* stream) {
  return step_diffusion(p, a, b, coef, steps, steps > 0 ? steps : 1, nullptr, stream);
}

int fractal_step_diffusion_sum(fractal_plan_t p, float* a, float* b, float coef, int steps, double* dev_sum,
                               void* stream) {
  if (!dev_sum) return FRACTAL_EINVAL;
  return step_diffusion(p, a, b, coef, steps, steps > 0 ? steps : 1, dev_sum, stream);
}

int fractal_step_diffusion_sums(fractal_plan_t p, float* a, float* b, float coef, int steps, int every,
                                double* dev_sums, void* stream) {
  if (!dev_sums || every < 1 || steps < 0 || steps % every != 0) return FRACTAL_EINVAL;
  if (steps == 0) return step_diffusion(p, a, b, coef, 0, 1, nullptr, stream);  // validation only
  return step_diffusion(p, a, b, coef, steps, every, dev_sums, stream);
}

int fractal_step_diffusion_kappa(fractal_plan_t p, float* a, float* b, const float* kappa, float coef, int steps,
                                 void* stream) {
  if (!std::isfinite(coef)) return FRACTAL_EINVAL;
  return step_kappa(p, a, b, kappa, coef, steps, stream);
}

int fractal_step_diffusion_kappa_f64(fractal_plan_t p, double* a, double* b, const float* kappa, double coef,
                                     int steps, void* stream) {
  if (!std::isfinite(coef)) return FRACTAL_EINVAL;
  return step_kappa(p, a, b, kappa, coef, steps, stream);
}

int fractal_step_diffusion_kappa_df(fractal_plan_t p, float* a, float* b, const float* kappa, double coef,
                                    int steps, void* stream) {
  if (!std::isfinite(coef)) return FRACTAL_EINVAL;
  return step_kappa(p, reinterpret_cast<dfloat*>(a), reinterpret_cast<dfloat*>(b), kappa, dfloat_from_double(coef),
                    steps, stream);
}

int fractal_adjoint_diffusion_step(fractal_plan_t p, const float* u, const float* p_in, float* p_out,
                                   const float* kappa, double* gkappa, float coef, void* stream) {
  if (!std::isfinite(coef)) return FRACTAL_EINVAL;
  return adjoint_step(p, u, p_in, p_out, kappa, gkappa, coef, stream);
}

int fractal_adjoint_diffusion_step_f64(fractal_plan_t p, const double* u, const double* p_in, double* p_out,
                                       const float* kappa, double* gkappa, double coef, void* stream) {
  if (!std::isfinite(coef)) return FRACTAL_EINVAL;
  return adjoint_step(p, u, p_in, p_out, kappa, gkappa, coef, stream);
}

int fractal_adjoint_diffusion_step_df(fractal_plan_t p, const float* u, const float* p_in, float* p_out,
                                      const float* kappa, float* gkappa, double coef, void* stream) {
  if (!std::isfinite(coef)) return FRACTAL_EINVAL;
  return adjoint_step(p, reinterpret_cast<const dfloat*>(u), reinterpret_cast<const dfloat*>(p_in),
                      reinterpret_cast<dfloat*>(p_out), kappa, reinterpret_cast<dfloat*>(gkappa),
                      dfloat_from_double(coef), stream);
}

int fractal_reduce_async(fractal_plan_t p, const void* dev_buf, int dtype, double* dev_out, void* stream) {
  if (check_plan(p) || !dev_buf || !dev_out || !aligned16(dev_buf)) return FRACTAL_EINVAL;
  if (dtype != FRACTAL_U8 && dtype != FRACTAL_F32) return FRACTAL_EINVAL;
  Launch B;
  int levels = 0;
  cudaError_t e;
  if (use_blocks(p, dtype, B, levels))
    e = launch_reduce_blocks(p->mode, B, levels, static_cast<const float*>(dev_buf),
                             static_cast<double*>(p->d_partials), dev_out, (cudaStream_t)stream);
  else
    e = launch_reduce(p->mode, p->log_rho, dtype, p->aux[dtype], dev_buf, p->d_partials, dev_out,
                      (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "reduce");
}

int fractal_reduce(fractal_plan_t p, const void* dev_buf, int dtype, double* host_out, void* stream) {
  if (check_plan(p) || !host_out) return FRACTAL_EINVAL;
  int st = fractal_reduce_async(p, dev_buf, dtype, p->d_result, stream);
  if (st != FRACTAL_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(p->h_result, p->d_result, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "reduce copy");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "reduce sync");
  *host_out = *p->h_result;
  return FRACTAL_OK;
}

int fractal_pack(fractal_plan_t p, const void* dev_embedded, int dtype, void* dev_packed, void* stream) {
  if (check_plan(p) || !dev_embedded || !dev_packed || dev_embedded == dev_packed || !aligned16(dev_embedded) ||
      !aligned16(dev_packed) || (dtype != FRACTAL_U8 && dtype != FRACTAL_F32) ||
      !device_addressable(dev_embedded, p->device) || !device_addressable(dev_packed, p->device))
    return FRACTAL_EINVAL;
  cudaError_t e = launch_pack(dev_embedded, dev_packed, p->n, p->rb, 1 << p->log_rho, dtype == FRACTAL_U8 ? 1 : 4,
                              on_device(dev_packed), (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "pack");
}

int fractal_unpack(fractal_plan_t p, const void* dev_packed, int dtype, void* dev_embedded, void* stream) {
  if (check_plan(p) || !dev_embedded || !dev_packed || dev_embedded == dev_packed || !aligned16(dev_embedded) ||
      !aligned16(dev_packed) || (dtype != FRACTAL_U8 && dtype != FRACTAL_F32) ||
      !device_addressable(dev_embedded, p->device) || !device_addressable(dev_packed, p->device))
    return FRACTAL_EINVAL;
  cudaError_t e = launch_unpack(dev_packed, dev_embedded, p->n, p->rb, 1 << p->log_rho,
                                dtype == FRACTAL_U8 ? 1 : 4, on_device(dev_packed), (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "unpack");
}

int fractal_set_l2_fetch_granularity(int bytes) {
  if (bytes != 32 && bytes != 64 && bytes != 128) return FRACTAL_EINVAL;
  cudaError_t e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes);
  return e == cudaSuccess ? FRACTAL_OK : cuda_fail(e, "set L2 fetch granularity");
}

int fractal_get_l2_fetch_granularity(int* bytes) {
  if (!bytes) return FRACTAL_EINVAL;
  size_t v = 0;
  cudaError_t e = cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity);
  if (e != cudaSuccess) return cuda_fail(e, "get L2 fetch granularity");
  *bytes = (int)v;
  return FRACTAL_OK;
}

}  // extern "C"
