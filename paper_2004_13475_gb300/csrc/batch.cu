// C ABI of batches (declared in include/fractal.h): many independent gaskets
// of uneven levels advanced by one persistent launch per group of steps,
// driven by a per-instance table of super-tile offsets; CUDA graphs of whole
// multi-step runs.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fractal.h"
#include "launch.h"

using namespace fractal;

struct fractal_batch_s {
  int count = 0;
  int device = 0;
  int kmin = 99, kmax = -1;
  std::vector<int> ks;
  int T = 0;                       // super-tile side
  int spl = 8, margin = 8;         // steps per launch, margin of the fused kernel
  int threads = 0, ctas = 0;       // persistent launch
  int64_t items = 0, members = 0;
  std::vector<BatchInst> h;        // host copy of the table
  BatchInst* d_inst = nullptr;
  double* d_partials = nullptr;    // one per item (reduce)
  int64_t partials_cap = 0;
  bool bound = false;
  cudaStream_t capture = nullptr;  // stream graphs are captured on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_steps = 0;
  float* d_rec[2] = {nullptr, nullptr};  // block records between the launches of one call
  int4* d_desc = nullptr;                // per-thread setups of the current configuration
  size_t desc_cap = 0;                   // bytes
  bool desc_ok = false;
};

namespace {

int64_t pow3(int e) {
  int64_t r = 1;
  while (e-- > 0) r *= 3;
  return r;
}

int log2i(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

void drop_graph(fractal_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_steps = 0;
}

// Threads for side T, margin M and reach (0 if invalid for this batch).
// Launches of 320 slots (side 256, margins of 64 cells at reach <= 56) run
// four warps per item; the others one block per thread in at most 288.
int batch_threads(const fractal_batch_s* b, int T, int margin, int reach) {
  if (T < 16 || (T & (T - 1)) != 0 || T > (1 << b->kmin)) return 0;
  Geo g{};
  g.T = T;
  const int t = fused_threads(g, 0, margin, reach);
  return t <= 288 || t == fused_q3_slots() ? t : 0;
}

// Offsets, R and the persistent grid for the current T; table upload if bound.
int rebuild(fractal_batch_s* b) {
  const int lt = log2i(b->T);
  int64_t first = 0;
  for (int i = 0; i < b->count; ++i) {
    BatchInst& e = b->h[i];
    e.n = 1 << b->ks[i];
    e.R = b->ks[i] - lt;
    e.lwR = (int32_t)pow3((e.R + 1) / 2);
    e.first = first;
    first += pow3(e.R);
  }
  b->items = first;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_batch_kernel(), b->threads,
                                                    fused_batch_smem_bytes(b->threads)) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    cudaGetLastError();
    return FRACTAL_ECUDA;
  }
  if (per_sm < 1) per_sm = 1;
  const int64_t grid = (int64_t)per_sm * sms;
  b->ctas = (int)(grid < b->items ? grid : b->items);
  if (b->threads == fused_q3_slots()) b->ctas = (int)b->items;  // one CTA per item
  if (b->bound &&
      cudaMemcpy(b->d_inst, b->h.data(), sizeof(BatchInst) * b->count, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return FRACTAL_ECUDA;
  }
  // the launches' per-thread setups, once per configuration (the kernels
  // compute them themselves when there is no room for them)
  b->desc_ok = false;
  if (b->bound) {
    const size_t need = (size_t)b->items * (size_t)b->threads * sizeof(int4);
    if (need > b->desc_cap) {
      if (b->d_desc) cudaFree(b->d_desc);
      b->d_desc = nullptr;
      b->desc_cap = 0;
      if (lib_malloc(&b->d_desc, need) == cudaSuccess) {
        b->desc_cap = need;
      } else {
        cudaGetLastError();
        b->d_desc = nullptr;
      }
    }
    if (b->d_desc) {
      if (launch_batch_describe(b->d_inst, b->count, b->items, b->margin, b->spl, b->T, b->ctas, b->threads, b->d_desc,
                                nullptr) != cudaSuccess ||
          cudaStreamSynchronize(nullptr) != cudaSuccess) {
        cudaGetLastError();
        return FRACTAL_ECUDA;
      }
      b->desc_ok = true;
    }
    // the four-warp launch reads its threads' setups from the descriptors
    if (!b->desc_ok && b->threads == fused_q3_slots()) return FRACTAL_ENOMEM;
  }
  return FRACTAL_OK;
}

int launch_steps(fractal_batch_s* b, float a, int steps, cudaStream_t s) {
  // As fractal_step_diffusion: with records, ceil(steps / spl) launches (two
  // for one even-step launch), the first from the instances' a buffers, the
  // last into a (even steps) or b (odd), the state in the block records
  // between them; without, ping-pong launches with the parity of `steps`.
  const bool rec = b->d_rec[0] && b->d_rec[1];
  int L = (steps + b->spl - 1) / b->spl;
  if (rec ? (L == 1 && (steps & 1) == 0) : ((L & 1) != (steps & 1))) ++L;
  const int base = steps / L, extra = steps % L;
  for (int i = 0; i < L; ++i) {
    const int ns = base + (i < extra ? 1 : 0);
    const bool first = i == 0, last = i == L - 1;
    const float* pin = rec && !first ? b->d_rec[(i - 1) & 1] : nullptr;
    float* pout = rec && !last ? b->d_rec[i & 1] : nullptr;
    // which = 0: a -> b, 1: b -> a (in / out where they are the buffers)
    const int which = !rec ? (i & 1) : (first ? 0 : ((steps & 1) == 0 ? 1 : 0));
    const cudaError_t e = launch_diffusion_batch(b->d_inst, b->count, b->items, which, a, ns, b->margin, b->spl, b->T,
                                                 b->ctas, b->threads, s, pin, pout,
                                                 b->desc_ok ? b->d_desc : nullptr);
    if (e != cudaSuccess) return FRACTAL_ECUDA;
  }
  return FRACTAL_OK;
}

}  // namespace

extern "C" {

int fractal_batch_create(int count, const int32_t* ks, fractal_batch_t* out) {
  if (!out) return FRACTAL_EINVAL;
  *out = nullptr;
  if (count < 1 || count > 65536 || !ks) return FRACTAL_EINVAL;
  for (int i = 0; i < count; ++i)
    if (ks[i] < 4 || ks[i] > FRACTAL_MAX_LEVEL) return FRACTAL_EINVAL;
  fractal_batch_s* b = new (std::nothrow) fractal_batch_s();
  if (!b) return FRACTAL_ENOMEM;
  b->count = count;
  b->ks.assign(ks, ks + count);
  b->h.assign(count, BatchInst{});
  for (int k : b->ks) {
    if (k < b->kmin) b->kmin = k;
    if (k > b->kmax) b->kmax = k;
    b->members += pow3(k);
  }
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return FRACTAL_ECUDA;
  }
  // default: 8 steps per launch, the largest side <= 256 all instances hold
  b->spl = 8;
  b->margin = fused_margin(8);
  b->T = 1 << (b->kmin < 8 ? b->kmin : 8);
  b->threads = batch_threads(b, b->T, b->margin, b->spl);
  if (b->threads == 0) {
    delete b;
    return FRACTAL_EINVAL;
  }
  if (lib_malloc(&b->d_inst, sizeof(BatchInst) * count) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    fractal_batch_destroy(b);
    return FRACTAL_ENOMEM;
  }
  const int st = rebuild(b);
  if (st != FRACTAL_OK) {
    fractal_batch_destroy(b);
    return st;
  }
  *out = b;
  return FRACTAL_OK;
}

int fractal_batch_destroy(fractal_batch_t b) {
  if (!b) return FRACTAL_OK;
  drop_graph(b);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_partials) cudaFree(b->d_partials);
  for (int i = 0; i < 2; ++i)
    if (b->d_rec[i]) cudaFree(b->d_rec[i]);
  if (b->d_desc) cudaFree(b->d_desc);
  delete b;
  return FRACTAL_OK;
}

int fractal_batch_bind(fractal_batch_t b, float* const* dev_a, float* const* dev_b) {
  if (!b || !dev_a || !dev_b) return FRACTAL_EINVAL;
  for (int i = 0; i < b->count; ++i)
    if (!dev_a[i] || !dev_b[i] || dev_a[i] == dev_b[i] || !aligned16(dev_a[i]) || !aligned16(dev_b[i]))
      return FRACTAL_EINVAL;
  // block records of all instances, 3^(k_i - 3) of 112 bytes each, whatever
  // the super-tile side (allocated once, before any launch or capture; a
  // failure leaves the batch as it was)
  if (!b->d_rec[0]) {
    int64_t recs = 0;
    for (int k : b->ks) recs += pow3(k - 3);
    const size_t bytes = (size_t)recs * (size_t)fused_record_bytes();
    for (int i = 0; i < 2; ++i) {
      if (lib_malloc(&b->d_rec[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        for (int j = 0; j < 2; ++j) {
          if (b->d_rec[j]) cudaFree(b->d_rec[j]);
          b->d_rec[j] = nullptr;
        }
        return FRACTAL_ENOMEM;
      }
    }
  }
  for (int i = 0; i < b->count; ++i) {
    b->h[i].a = dev_a[i];
    b->h[i].b = dev_b[i];
  }
  b->bound = true;
  return rebuild(b);
}

int fractal_batch_configure(fractal_batch_t b, int supertile, int spl) {
  if (!b || spl < 1 || spl > 56 || supertile < 0) return FRACTAL_EINVAL;
  const int T = supertile ? supertile : b->T;
  const int margin = fused_margin(spl);
  const int threads = batch_threads(b, T, margin, spl);
  if (threads == 0) return FRACTAL_EINVAL;
  drop_graph(b);
  b->T = T;
  b->spl = spl;
  b->margin = margin;
  b->threads = threads;
  return rebuild(b);
}

int fractal_batch_step_diffusion(fractal_batch_t b, float a, int steps, void* stream) {
  if (!b || !b->bound || steps < 0 || !std::isfinite(a)) return FRACTAL_EINVAL;
  if (steps == 0) return FRACTAL_OK;
  return launch_steps(b, a, steps, (cudaStream_t)stream);
}

int fractal_batch_reduce(fractal_batch_t b, int which, double* dev_out, void* stream) {
  if (!b || !b->bound || !dev_out || (which != 0 && which != 1)) return FRACTAL_EINVAL;
  if (b->partials_cap < b->items) {
    double* p = nullptr;
    if (lib_malloc(&p, sizeof(double) * b->items) != cudaSuccess) {
      cudaGetLastError();
      return FRACTAL_ENOMEM;
    }
    if (b->d_partials) cudaFree(b->d_partials);
    b->d_partials = p;
    b->partials_cap = b->items;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const int64_t grid = (int64_t)(sms > 0 ? sms : 1) * 8;
  const int ctas = (int)(grid < b->items ? grid : b->items);
  const cudaError_t e = launch_batch_reduce(b->d_inst, b->count, b->items, which, b->T, ctas, b->d_partials, dev_out,
                                            (cudaStream_t)stream);
  return e == cudaSuccess ? FRACTAL_OK : FRACTAL_ECUDA;
}

int fractal_batch_autotune(fractal_batch_t b, float a, int reps, float* best_us, void* stream) {
  if (!b || !b->bound || reps < 1 || !std::isfinite(a)) return FRACTAL_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return FRACTAL_ENOMEM;
  }
  const int old_T = b->T, old_spl = b->spl;
  float best = -1.f;
  int best_T = old_T, best_spl = old_spl;
  int status = FRACTAL_OK;
  const int spls[4] = {8, 16, 32, 50};
  for (int T = 16; T <= 512 && status == FRACTAL_OK; T *= 2) {
    for (int si = 0; si < 4 && status == FRACTAL_OK; ++si) {
      if (fractal_batch_configure(b, T, spls[si]) != FRACTAL_OK) continue;
      // launches of spl steps, dev_a -> dev_b only (which = 0)
      auto one = [&]() -> int {
        return launch_diffusion_batch(b->d_inst, b->count, b->items, 0, a, b->spl, b->margin, b->spl, b->T, b->ctas,
                                      b->threads, st, nullptr, nullptr, b->desc_ok ? b->d_desc : nullptr) ==
                       cudaSuccess
                   ? FRACTAL_OK
                   : FRACTAL_ECUDA;
      };
      for (int i = 0; i < 2 && status == FRACTAL_OK; ++i) status = one();
      if (status != FRACTAL_OK || cudaEventRecord(e0, st) != cudaSuccess) {
        status = FRACTAL_ECUDA;
        break;
      }
      for (int i = 0; i < reps && status == FRACTAL_OK; ++i) status = one();
      float ms = 0.f;
      if (status != FRACTAL_OK || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        status = FRACTAL_ECUDA;
        break;
      }
      const float us = 1000.f * ms / (float)(reps * b->spl);
      if (best < 0.f || us < best) {
        best = us;
        best_T = T;
        best_spl = spls[si];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != FRACTAL_OK) cudaGetLastError();
  const bool ok = status == FRACTAL_OK && best >= 0.f;
  const int st2 = fractal_batch_configure(b, ok ? best_T : old_T, ok ? best_spl : old_spl);
  if (ok && best_us) *best_us = best;
  return status != FRACTAL_OK ? status : st2;
}

int fractal_batch_graph_capture(fractal_batch_t b, float a, int steps) {
  if (!b || !b->bound || steps < 1 || !std::isfinite(a)) return FRACTAL_EINVAL;
  drop_graph(b);
  if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return FRACTAL_ECUDA;
  }
  const int st = launch_steps(b, a, steps, b->capture);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
  if (st != FRACTAL_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return FRACTAL_ECUDA;
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    b->exec = nullptr;
    cudaGetLastError();
    return FRACTAL_ECUDA;
  }
  b->graph = g;
  b->graph_steps = steps;
  return FRACTAL_OK;
}

int fractal_batch_graph_launch(fractal_batch_t b, void* stream) {
  if (!b || !b->exec) return FRACTAL_EINVAL;
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? FRACTAL_OK : FRACTAL_ECUDA;
}

int fractal_batch_get_info(fractal_batch_t b, fractal_batch_info* info) {
  if (!b || !info) return FRACTAL_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->count = b->count;
  info->k_min = b->kmin;
  info->k_max = b->kmax;
  info->supertile = b->T;
  info->steps_per_launch = b->spl;
  info->ctas = b->ctas;
  info->threads = b->threads;
  info->smem_bytes = fused_batch_smem_bytes(b->threads);
  info->supertiles = b->items;
  info->members = b->members;
  info->bound = b->bound ? 1 : 0;
  info->graph_steps = b->graph_steps;
  return FRACTAL_OK;
}

}  // extern "C"
