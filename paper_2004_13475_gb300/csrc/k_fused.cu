// Temporally fused diffusion: one CTA advances its member super-tile by up to
// M steps per launch, each thread holding one 8 x 8-cell block of the gasket
// in registers.
//
// Blocks and ports.  Split the array into 8 x 8 blocks.  A block (BX, BY) with
// BX & BY == 0 holds the 27 members (i, j), i & j == 0, of a level-3 gasket;
// every other block holds none.  Its members touch cells of other blocks at
// four links only, through three corner cells ("ports"):
//   (0,0) <-> (0,7) of the block above      (0,0) <-> (7,0) of the block left
//   (7,0) <-> (0,0) of the block right      (0,7) <-> (0,0) of the block below
// (any other member (i, 0) or (0, j) on the near edges faces a cell (i, 7) or
// (7, j) of the neighbour with i & 7 or 7 & j nonzero, a non-member; the far
// edges (7, j) and (i, 7) hold members only at j = 0 and i = 0).  So a step
// needs, besides the block's own 27 values, four values of its neighbours:
// each thread publishes its three port values per step in shared memory and
// reads four.
//
// Margin boxes.  The gasket outside a member super-tile of side T touches it
// only near (0, 0), (T-1, 0) and (0, T-1); for s <= M <= T/2 every member that
// can reach the super-tile within s steps of the 4-neighbour stencil lies in
//   left   [-M, 0) x [0, M)        top    [0, M) x [-M, 0)
//   right  [T, T+M) x [-M, M)      bottom [-M, M) x [T, T+M)
// With M a multiple of 8 these are whole blocks; they are evolved with the
// super-tile (a box block whose neighbour was not staged goes wrong from the
// box edge inwards, one cell per step, and never reaches the super-tile) and
// are not written back.
//
// A launch reads the member blocks' member 16-byte chunks once, runs the steps
// with one barrier each, and writes the member blocks back; for rho >= 8 it
// also writes the zeros of the non-member cells of member tiles, so that every
// write covers whole 32-byte sectors.
#include <atomic>

#include "blocks.cuh"
#include "launch.h"
#include "tma.cuh"

namespace fractal {
namespace {

// CTA sizes of a fused launch, each compiled with its own register budget:
// up to 288 threads (super-tile side 256 with 32-cell margins: 243 + 27
// blocks), four CTAs per SM; up to 352 (64-cell margins: 243 + 81), three;
// up to 512 (128-cell margins: 243 + 243), two.
constexpr int kFusedMaxThreads = 512;

// Per-CTA geometry of a fused launch.
struct FGeo {
  int n;        // array side
  int L;        // block levels of the super-tile: T / 8 = 2^L
  int lw;       // 3^ceil(L/2): width of the level-L packed grid
  int nb;       // member blocks of the super-tile: 3^L
  int W;        // box width in blocks: M / 8
  int lW;       // log2 W
  int nbox;     // box blocks: 6 W^2
  int reach;    // steps per launch served: box blocks further than this are not staged
  int log_rho;  // the plan's tile side (write-back of whole member tiles)
  int R;        // super-tile levels of the array: (k - 3) - L
  int lwR;      // 3^ceil(R/2): width of the level-R packed grid of super-tiles
  int64_t rec0; // records before this array's (batches: earlier instances')
};

// Compact records between the launches of one call: the 27 members of a
// member 8 x 8 block (row-major order of the member cells) and one pad, 7
// float4s; record s * 3^L + t for member block t (lambda or BB rank order)
// of member super-tile s (its index in the level-R packed grid, or its BB
// rank).  The records of one super-tile form a group stored float4 by
// float4: float4 i of its block t at (group start) + i * 3^L + t, so that
// the threads of a warp, taking consecutive blocks, read and write 16
// consecutive bytes each.  3^(k-3) records hold the whole gasket; a launch
// reads and writes them instead of eight scattered 32-byte rows per block.
constexpr int kRecF4 = 7;

// Float4 index of float4 0 of record `rec` (a record's float4s are nb apart).
__device__ __forceinline__ int64_t rec_base(int64_t rec, int nb) {
  const int64_t t = rec % nb;
  return (rec - t) * kRecF4 + t;
}

// Record of the member block (GX, GY) (block coordinates in the array).
template <int MODE>
__device__ __forceinline__ int64_t block_record(int GX, int GY, const FGeo& f) {
  const int mask = (1 << f.L) - 1;
  const int ssx = GX >> f.L, ssy = GY >> f.L, lx = GX & mask, ly = GY & mask;
  const int64_t s = MODE == kLambda ? lambda_inverse(ssx, ssy, f.R, f.lwR) : bb_rank(ssx, ssy, f.R);
  const int t = MODE == kLambda ? lambda_inverse(lx, ly, f.L, f.lw) : bb_rank(lx, ly, f.L);
  return f.rec0 + s * f.nb + t;
}

// Member m of a record -> float m%4 of float4 m/4 (compile-time m).
__device__ __forceinline__ float rec_get(const float4 (&r)[kRecF4], int m) {
  const float4 v = r[m >> 2];
  return (m & 3) == 0 ? v.x : (m & 3) == 1 ? v.y : (m & 3) == 2 ? v.z : v.w;
}
__device__ __forceinline__ void rec_set(float4 (&r)[kRecF4], int m, float x) {
  float4& v = r[m >> 2];
  if ((m & 3) == 0) v.x = x; else if ((m & 3) == 1) v.y = x; else if ((m & 3) == 2) v.z = x; else v.w = x;
}

// Member blocks the margin boxes can hold: a gasket fragment of side M at
// each of the three contacts, 3 * 3^log2(W) (tests/test_fusion_boxes.py
// checks every super-tile position); a launch gives threads to those only.
__host__ __device__ inline int box_cap(int W) {
  int c = 3;
  for (int w = W; w > 1; w >>= 1) c *= 3;
  return c < 6 * W * W ? c : 6 * W * W;
}
constexpr int kMaxW = 16;                    // margins up to 128 cells
constexpr int kMaxBox = 6 * kMaxW * kMaxW;   // box blocks: 6 W^2
constexpr int kMaxBoxMembers = 243;          // box_cap(16)
constexpr int kMaxSide = 32;                 // blocks per super-tile side (T <= 256)

// Member block t of the super-tile (lambda order, or BB rank order via tab).
template <int MODE>
__device__ __forceinline__ void member_block(int t, const FGeo& f, const int* tab, int& bx, int& by) {
  if (MODE == kLambda) {
    lambda_scalar((uint32_t)(t % f.lw), (uint32_t)(t / f.lw), f.L, bx, by);
  } else {
    const int j = tab[t];
    bx = j & ((1 << f.L) - 1);
    by = j >> f.L;
  }
}

// Box block b (0 <= b < 6 W^2): left, top, right, bottom boxes in row order.
// Block coordinates relative to the super-tile.
__device__ __forceinline__ void box_block(int b, const FGeo& f, int& bx, int& by) {
  const int W = f.W, lW = f.lW, W2 = W * W, side = 1 << f.L;
  if (b < W2) {  // left
    bx = -W + (b & (W - 1));
    by = b >> lW;
    return;
  }
  b -= W2;
  if (b < W2) {  // top
    bx = b & (W - 1);
    by = -W + (b >> lW);
    return;
  }
  b -= W2;
  if (b < 2 * W2) {  // right
    bx = side + (b & (W - 1));
    by = -W + (b >> lW);
    return;
  }
  b -= 2 * W2;  // bottom
  bx = -W + (b & (2 * W - 1));
  by = side + (b >> (lW + 1));
}

// Thread that owns block (bx, by), or `none` if no staged member block is
// there; own: the thread of each member block of the super-tile (slot
// by * side + bx); boxrank: compacted rank of each box block, -1 for
// non-members.
__device__ __forceinline__ int fused_owner(int bx, int by, const FGeo& f, const short* own, const int* boxrank,
                                           int none) {
  const int side = 1 << f.L, W = f.W, W2 = W * W;
  if (bx >= 0 && by >= 0 && bx < side && by < side) {
    if (bx & by) return none;
    return own[(by << f.L) + bx];
  }
  int b = -1;
  if (bx >= -W && bx < 0 && by >= 0 && by < W) b = by * W + (bx + W);
  else if (bx >= 0 && bx < W && by >= -W && by < 0) b = W2 + (by + W) * W + bx;
  else if (bx >= side && bx < side + W && by >= -W && by < W) b = 2 * W2 + (by + W) * W + (bx - side);
  else if (bx >= -W && bx < W && by >= side && by < side + W) b = 4 * W2 + (by - side) * 2 * W + (bx + W);
  if (b < 0 || boxrank[b] < 0) return none;
  return f.nb + boxrank[b];
}

__device__ __forceinline__ bool block_member(int gx, int gy, int nblk) {
  return (unsigned)gx < (unsigned)nblk && (unsigned)gy < (unsigned)nblk && (gx & gy) == 0;
}

// Manhattan distance from the nearest cell of block (qx, qy) (block
// coordinates relative to the super-tile) to the super-tile [0, 8 side)^2.
// Influence moves one cell per step along 4-neighbour links, so a launch of
// s steps needs no box block further than s: a block it leaves out is read
// as 0 by its neighbours, and the error that starts there (at distance >= s)
// reaches the super-tile only after more than s steps.
__host__ __device__ inline int box_distance(int qx, int qy, int side) {
  const int dx = qx < 0 ? -kB * qx - kB + 1 : qx >= side ? kB * (qx - side) + 1 : 0;
  const int dy = qy < 0 ? -kB * qy - kB + 1 : qy >= side ? kB * (qy - side) + 1 : 0;
  return dx + dy;
}

// Port slots: P0 = (0,0), PR = (7,0), PD = (0,7) of every block, double-
// buffered by step parity, plus a zero slot at index `threads`.
__host__ __device__ inline int fused_slots(int threads) { return threads + 1; }

// CTA size classes of the fused kernel (launch bounds and, as the port
// arrays' stride, slots = class + 1, a compile-time constant so that the two
// parities' offsets are immediates): 288 threads, four CTAs per SM; 352,
// three; 512, two.
__host__ __device__ inline int fused_class(int threads) { return threads <= 288 ? 288 : threads <= 352 ? 352 : 512; }

// Write back one member block of the super-tile from its values u (members;
// other entries unused): to the embedded array out (whole 32-byte rows, 0 at
// non-members, and the non-member cells of its tile row for rho >= 16), or to
// record `rec` of pout when that is not null.  Returns the block's member sum
// (FP32 within a row, FP64 over the rows) when want_sum, else 0.
__device__ __forceinline__ double write_block(const float (&u)[kB * kB], const FGeo& f, int GX, int GY,
                                              bool want_sum, float* __restrict__ out, float* __restrict__ pout,
                                              int64_t rec) {
  double sum = 0.0;
  if (want_sum) {
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      float r = 0.f;
      bool first = true;
#pragma unroll
      for (int i = 0; i < kB; ++i) {
        if (!amem(i, j)) continue;
        r = first ? u[j * kB + i] : r + u[j * kB + i];
        first = false;
      }
      sum += (double)r;
    }
  }
  if (pout) {
    float4 r[kRecF4];
    r[kRecF4 - 1].w = 0.f;  // the pad
    int m = 0;
#pragma unroll
    for (int q = 0; q < kB * kB; ++q)
      if (amem(q % kB, q / kB)) rec_set(r, m++, u[q]);
    float4* p = reinterpret_cast<float4*>(pout) + rec_base(rec, f.nb);
#pragma unroll
    for (int i = 0; i < kRecF4; ++i) p[(int64_t)i * f.nb] = r[i];
    return sum;
  }
  float* o = out + (size_t)GY * kB * (size_t)f.n + (size_t)GX * kB;
#pragma unroll
  for (int j = 0; j < kB; ++j)
    *reinterpret_cast<float4*>(o + (size_t)j * f.n) =
        make_float4(u[j * kB + 0], u[j * kB + 1], u[j * kB + 2], u[j * kB + 3]);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    *reinterpret_cast<float4*>(o + (size_t)j * f.n + 4) =
        make_float4(u[j * kB + 4], u[j * kB + 5], u[j * kB + 6], u[j * kB + 7]);
  if (f.log_rho >= 3) {
    // non-member cells of member tiles: the block's lower right quarter,
    // and (rho >= 16) the non-member blocks right of this one in its tile
    // row, up to the next member block
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 4; j < kB; ++j) *reinterpret_cast<float4*>(o + (size_t)j * f.n + 4) = z;
    const int bpt = 1 << (f.log_rho - 3);  // blocks per tile side
    const int tx = GX & (bpt - 1), ty = GY & (bpt - 1);
    for (int q = tx + 1; q < bpt && (q & ty) != 0; ++q) {
      float* p = o + (size_t)(q - tx) * kB;
      for (int j = 0; j < kB; ++j) {
        *reinterpret_cast<float4*>(p + (size_t)j * f.n) = z;
        *reinterpret_cast<float4*>(p + (size_t)j * f.n + 4) = z;
      }
    }
  }
  return sum;
}

// The block of one staged slot into u (members; other entries 0): record
// `rec` of pin when that is not null, else the block (GX, GY) of in.
__device__ __forceinline__ void stage_block(float (&u)[kB * kB], const FGeo& f, int GX, int GY,
                                            const float* __restrict__ in, const float* __restrict__ pin, int64_t rec) {
#pragma unroll
  for (int q = 0; q < kB * kB; ++q) u[q] = 0.f;
  if (pin) {
    const float4* p = reinterpret_cast<const float4*>(pin) + rec_base(rec, f.nb);
    float4 r[kRecF4];
#pragma unroll
    for (int i = 0; i < kRecF4; ++i) r[i] = __ldg(p + (int64_t)i * f.nb);
    int m = 0;
#pragma unroll
    for (int q = 0; q < kB * kB; ++q)
      if (amem(q % kB, q / kB)) u[q] = rec_get(r, m++);
    return;
  }
  const float* b = in + (size_t)GY * kB * (size_t)f.n + (size_t)GX * kB;
  float4 c[12];
#pragma unroll
  for (int j = 0; j < kB; ++j) c[j] = __ldg(reinterpret_cast<const float4*>(b + (size_t)j * f.n));
#pragma unroll
  for (int j = 0; j < 4; ++j) c[8 + j] = __ldg(reinterpret_cast<const float4*>(b + (size_t)j * f.n + 4));
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    const float4 v = mask_chunk(c[j], 0, j);
    u[j * kB + 0] = v.x;
    u[j * kB + 1] = v.y;
    u[j * kB + 2] = v.z;
    u[j * kB + 3] = v.w;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 v = mask_chunk(c[8 + j], 4, j);
    u[j * kB + 4] = v.x;
    u[j * kB + 5] = v.y;
    u[j * kB + 6] = v.z;
    u[j * kB + 7] = v.w;
  }
}

// One super-tile whose block origin is (OX, OY) (in blocks).  All threads of
// the CTA call it; it ends after the write-back.  ports: 6 * slots floats.
// The state comes from the embedded array `in`, or from the records `pin`
// when that is not null; it goes to the embedded array `out`, or to the
// records `pout` when that is not null (srec: the super-tile's first record).
// Returns this thread's share of the sum of the written members (its block's
// rows in FP32, the rows in FP64; 0 for box blocks and idle threads, and 0
// unless want_sum).
// Per-thread setup of a fused launch, the same for every launch of one fused
// configuration (array, super-tile, margin, CTA size): the thread's block
// (bx, by, relative to the super-tile origin; a member block of the
// super-tile, a member block of a margin box, or none), the threads that own
// its four ports' neighbours (`zero`: the zero slot), which of those
// neighbours are members, and for a box block its record.
struct FSetup {
  int bx, by;
  bool active;
  int up, lf, rt, dn;
  bool fu, fl, fr, fd;
  int rec;  // a box block's record (records launches), -1 otherwise
};

template <int MODE>
__device__ __forceinline__ FSetup fused_setup(const FGeo& f, int OX, int OY, const int* tab) {
  const int t = threadIdx.x, nthreads = blockDim.x;
  const int zero = nthreads;
  const int nblk = f.n / kB;
  // the margin boxes' member blocks, compacted in box order: boxrank[b] is
  // the rank of box block b among them (-1 if not a member), boxlist the list
  __shared__ int boxrank[kMaxBox], boxlist[kMaxBoxMembers], wcnt[16];
  __shared__ short own[kMaxSide * kMaxSide];
  FSetup s;
  s.bx = s.by = 0;
  s.active = false;
  s.rec = -1;
  if (t < f.nb) {
    member_block<MODE>(t, f, tab, s.bx, s.by);
    own[(s.by << f.L) + s.bx] = (short)t;  // every member slot is some thread's
    s.active = true;
  }
  int nbox_member = 0;
  for (int b0 = 0; b0 < f.nbox; b0 += nthreads) {  // its barriers also publish own[]
    const int b = b0 + t;
    bool m = false;
    if (b < f.nbox) {
      int qx, qy;
      box_block(b, f, qx, qy);
      m = block_member(OX + qx, OY + qy, nblk) && box_distance(qx, qy, 1 << f.L) <= f.reach;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if ((t & 31) == 0) wcnt[t >> 5] = __popc(bal);
    __syncthreads();
    // lane l holds warp l's count: the warps before this one, and all
    const int lane = t & 31, nw = nthreads >> 5;
    const unsigned c = lane < nw ? (unsigned)wcnt[lane] : 0u;
    int rank = nbox_member + (int)__reduce_add_sync(0xffffffffu, lane < (t >> 5) ? c : 0u);
    const int total = (int)__reduce_add_sync(0xffffffffu, c);
    rank += __popc(bal & ((1u << lane) - 1u));
    if (b < f.nbox) {
      boxrank[b] = m ? rank : -1;
      if (m) boxlist[rank] = b;
    }
    nbox_member += total;
    __syncthreads();
  }
  if (t >= f.nb && t - f.nb < nbox_member) {
    box_block(boxlist[t - f.nb], f, s.bx, s.by);
    s.active = true;
    s.rec = (int)block_record<MODE>(OX + s.bx, OY + s.by, f);
  }
  const int GX = OX + s.bx, GY = OY + s.by;
  s.up = s.lf = s.rt = s.dn = zero;
  s.fu = s.fl = s.fr = s.fd = false;
  if (s.active) {
    s.fu = block_member(GX, GY - 1, nblk);
    s.fl = block_member(GX - 1, GY, nblk);
    s.fr = block_member(GX + 1, GY, nblk);
    s.fd = block_member(GX, GY + 1, nblk);
    if (s.fu) s.up = fused_owner(s.bx, s.by - 1, f, own, boxrank, zero);
    if (s.fl) s.lf = fused_owner(s.bx - 1, s.by, f, own, boxrank, zero);
    if (s.fr) s.rt = fused_owner(s.bx + 1, s.by, f, own, boxrank, zero);
    if (s.fd) s.dn = fused_owner(s.bx, s.by + 1, f, own, boxrank, zero);
  }
  return s;
}

// A setup in 16 bytes: x = flags (active, fu, fl, fr, fd) | bx << 8 | by << 16
// (bytes, two's complement), y = up | lf << 16, z = rt | dn << 16, w = rec.
__device__ __forceinline__ int4 pack_setup(const FSetup& s) {
  const int flags = (s.active ? 1 : 0) | (s.fu ? 2 : 0) | (s.fl ? 4 : 0) | (s.fr ? 8 : 0) | (s.fd ? 16 : 0);
  return make_int4(flags | ((s.bx & 0xff) << 8) | ((s.by & 0xff) << 16), s.up | (s.lf << 16), s.rt | (s.dn << 16),
                   s.rec);
}
__device__ __forceinline__ FSetup unpack_setup(int4 q) {
  FSetup s;
  s.active = q.x & 1;
  s.fu = q.x & 2;
  s.fl = q.x & 4;
  s.fr = q.x & 8;
  s.fd = q.x & 16;
  s.bx = (int)(signed char)((q.x >> 8) & 0xff);
  s.by = (int)(signed char)((q.x >> 16) & 0xff);
  s.up = q.y & 0xffff;
  s.lf = (q.y >> 16) & 0xffff;
  s.rt = q.z & 0xffff;
  s.dn = (q.z >> 16) & 0xffff;
  s.rec = q.w;
  return s;
}

template <int MODE, int SLOTS>
__device__ __forceinline__ double fused_supertile(const float* __restrict__ in, float* __restrict__ out, float a,
                                                  int nsteps, const FGeo& f, int OX, int OY, const int* tab,
                                                  float* ports, bool want_sum, const float* __restrict__ pin,
                                                  float* __restrict__ pout, int64_t srec,
                                                  const int4* __restrict__ desc) {
  const int t = threadIdx.x, nthreads = blockDim.x;
  constexpr int slots = SLOTS;  // >= nthreads + 1
  const int zero = nthreads;
  float* P0 = ports;  // [2][slots] each
  float* PR = ports + 2 * slots;
  float* PD = ports + 4 * slots;

  // this thread's setup: from the launch's descriptors, else computed here
  const FSetup su = desc ? unpack_setup(__ldg(desc + t)) : fused_setup<MODE>(f, OX, OY, tab);
  const int bx = su.bx, by = su.by;
  const bool active = su.active;
  const int GX = OX + bx, GY = OY + by;
  const int up = su.up, lf = su.lf, rt = su.rt, dn = su.dn;
  // the ports' degrees: 2, 1, 1 inside the block plus the member neighbour blocks
  const float d0 = 2.f + (su.fu ? 1.f : 0.f) + (su.fl ? 1.f : 0.f), dr = 1.f + (su.fr ? 1.f : 0.f),
              dd = 1.f + (su.fd ? 1.f : 0.f);

  // stage: the block's members straight into registers
  float u[kB * kB];
  if (active) {
    stage_block(u, f, GX, GY, in, pin, t < f.nb ? srec + t : (int64_t)su.rec);
  } else {
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) u[q] = 0.f;
  }
  P0[t] = u[0];
  PR[t] = u[kB - 1];
  PD[t] = u[(kB - 1) * kB];
  if (t == 0) {
    P0[zero] = P0[slots + zero] = 0.f;
    PR[zero] = PR[slots + zero] = 0.f;
    PD[zero] = PD[slots + zero] = 0.f;
  }
  __syncthreads();

  // two steps per iteration: the port offsets of both parities are fixed
#pragma unroll 2
  for (int s = 0; s < nsteps; ++s) {
    const int cur = (s & 1) * slots, nxt = slots - cur;
    if (active) {
      const float vu = PD[cur + up], vl = PR[cur + lf], vr = P0[cur + rt], vd = P0[cur + dn];
      block_step(u, a, vu, vl, vr, vd, d0, dr, dd);
    }
    P0[nxt + t] = u[0];
    PR[nxt + t] = u[kB - 1];
    PD[nxt + t] = u[(kB - 1) * kB];
    __syncthreads();
  }

  // write back the super-tile's member blocks (not the boxes)
  if (!(active && t < f.nb)) return 0.0;
  return write_block(u, f, GX, GY, want_sum, out, pout, srec + t);
}

// Two blocks per thread: slots 2t and 2t + 1 of the launch's descriptors
// (written for 2 * blockDim.x slots per CTA), every operation of the step
// paired across the two (block_step2); otherwise as fused_supertile.  The
// port arrays hold one value per slot, `slots` (even: the paired port stores
// are 8-byte aligned) per parity.
template <int MODE, int SLOTS>
__device__ __forceinline__ double fused_supertile2(const float* __restrict__ in, float* __restrict__ out, float a,
                                                   int nsteps, const FGeo& f, int OX, int OY, float* ports,
                                                   bool want_sum, const float* __restrict__ pin,
                                                   float* __restrict__ pout, int64_t srec,
                                                   const int4* __restrict__ desc) {
  const int t = threadIdx.x, zero = 2 * blockDim.x;
  constexpr int slots = SLOTS;  // >= zero + 1, even
  float* P0 = ports;
  float* PR = ports + 2 * slots;
  float* PD = ports + 4 * slots;
  const FSetup s0 = unpack_setup(__ldg(desc + 2 * t)), s1 = unpack_setup(__ldg(desc + 2 * t + 1));
  float2 u[kB * kB];
  {
    float w0[kB * kB], w1[kB * kB];
    if (s0.active) {
      stage_block(w0, f, OX + s0.bx, OY + s0.by, in, pin, 2 * t < f.nb ? srec + 2 * t : (int64_t)s0.rec);
    } else {
#pragma unroll
      for (int q = 0; q < kB * kB; ++q) w0[q] = 0.f;
    }
    if (s1.active) {
      stage_block(w1, f, OX + s1.bx, OY + s1.by, in, pin, 2 * t + 1 < f.nb ? srec + 2 * t + 1 : (int64_t)s1.rec);
    } else {
#pragma unroll
      for (int q = 0; q < kB * kB; ++q) w1[q] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) u[q] = make_float2(w0[q], w1[q]);
  }
  // the ports' degrees, negated: 2, 1, 1 inside the block plus the member neighbour blocks
  const float2 nd0 = make_float2(-(2.f + (s0.fu ? 1.f : 0.f) + (s0.fl ? 1.f : 0.f)),
                                 -(2.f + (s1.fu ? 1.f : 0.f) + (s1.fl ? 1.f : 0.f)));
  const float2 ndr = make_float2(-(1.f + (s0.fr ? 1.f : 0.f)), -(1.f + (s1.fr ? 1.f : 0.f)));
  const float2 ndd = make_float2(-(1.f + (s0.fd ? 1.f : 0.f)), -(1.f + (s1.fd ? 1.f : 0.f)));
  const bool active = s0.active || s1.active;
  const float2 a2 = make_float2(a, a);
  *reinterpret_cast<float2*>(P0 + 2 * t) = u[0];
  *reinterpret_cast<float2*>(PR + 2 * t) = u[kB - 1];
  *reinterpret_cast<float2*>(PD + 2 * t) = u[(kB - 1) * kB];
  if (t == 0) {
    P0[zero] = P0[slots + zero] = 0.f;
    PR[zero] = PR[slots + zero] = 0.f;
    PD[zero] = PD[slots + zero] = 0.f;
  }
  __syncthreads();

  // two steps per iteration: the port offsets of both parities are fixed
#pragma unroll 2
  for (int s = 0; s < nsteps; ++s) {
    const int cur = (s & 1) * slots, nxt = slots - cur;
    if (active) {
      const float2 vu = make_float2(PD[cur + s0.up], PD[cur + s1.up]);
      const float2 vl = make_float2(PR[cur + s0.lf], PR[cur + s1.lf]);
      const float2 vr = make_float2(P0[cur + s0.rt], P0[cur + s1.rt]);
      const float2 vd = make_float2(P0[cur + s0.dn], P0[cur + s1.dn]);
      block_step2(u, a2, vu, vl, vr, vd, nd0, ndr, ndd);
    }
    *reinterpret_cast<float2*>(P0 + nxt + 2 * t) = u[0];
    *reinterpret_cast<float2*>(PR + nxt + 2 * t) = u[kB - 1];
    *reinterpret_cast<float2*>(PD + nxt + 2 * t) = u[(kB - 1) * kB];
    __syncthreads();
  }

  // write back the super-tile's member blocks (not the boxes)
  double sum = 0.0;
  if (s0.active && 2 * t < f.nb) {
    float w[kB * kB];
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) w[q] = u[q].x;
    sum += write_block(w, f, OX + s0.bx, OY + s0.by, want_sum, out, pout, srec + 2 * t);
  }
  if (s1.active && 2 * t + 1 < f.nb) {
    float w[kB * kB];
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) w[q] = u[q].y;
    sum += write_block(w, f, OX + s1.bx, OY + s1.by, want_sum, out, pout, srec + 2 * t + 1);
  }
  return sum;
}

// One warp per CTA: super-tiles of side 128 (81 member blocks) with margins
// of at most 16 cells (at most 9 box blocks within reach), 96 block slots,
// three per lane (slots t, t + 32 and t + 64 of lane t: the first two paired
// in float2 as in fused_supertile2, the third on its own).  With a single
// warp the per-step port exchange needs only __syncwarp: no CTA waits on a
// slower warp of its own, and the CTAs, one warp each, spread evenly over the
// SM's four sub-partitions whatever their number.  The port arrays hold
// 96 + 2 slots per parity (the zero slot at 96).  Descriptors as for the
// other fused launches (96 per super-tile).
constexpr int kWarpSlots = 96;
constexpr int kWarpSide = 128;

template <int MODE>
__device__ __forceinline__ double fused_supertile_w(const float* __restrict__ in, float* __restrict__ out, float a,
                                                    int nsteps, const FGeo& f, int OX, int OY, float* ports,
                                                    bool want_sum, const float* __restrict__ pin,
                                                    float* __restrict__ pout, int64_t srec,
                                                    const int4* __restrict__ desc) {
  constexpr int kSl = kWarpSlots + 2;
  constexpr int zero = kWarpSlots;
  const int t = threadIdx.x;
  float* P0 = ports;
  float* PR = ports + 2 * kSl;
  float* PD = ports + 4 * kSl;
  const FSetup s0 = unpack_setup(__ldg(desc + t)), s1 = unpack_setup(__ldg(desc + t + 32)),
               s2 = unpack_setup(__ldg(desc + t + 64));
  float2 u[kB * kB];
  float v[kB * kB];
  {
    float w0[kB * kB], w1[kB * kB];
    if (s0.active) {
      stage_block(w0, f, OX + s0.bx, OY + s0.by, in, pin, t < f.nb ? srec + t : (int64_t)s0.rec);
    } else {
#pragma unroll
      for (int q = 0; q < kB * kB; ++q) w0[q] = 0.f;
    }
    if (s1.active) {
      stage_block(w1, f, OX + s1.bx, OY + s1.by, in, pin, t + 32 < f.nb ? srec + t + 32 : (int64_t)s1.rec);
    } else {
#pragma unroll
      for (int q = 0; q < kB * kB; ++q) w1[q] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) u[q] = make_float2(w0[q], w1[q]);
  }
  if (s2.active) {
    stage_block(v, f, OX + s2.bx, OY + s2.by, in, pin, t + 64 < f.nb ? srec + t + 64 : (int64_t)s2.rec);
  } else {
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) v[q] = 0.f;
  }
  // the ports' degrees: 2, 1, 1 inside the block plus the member neighbour
  // blocks (negated for the paired step)
  const float2 nd0 = make_float2(-(2.f + (s0.fu ? 1.f : 0.f) + (s0.fl ? 1.f : 0.f)),
                                 -(2.f + (s1.fu ? 1.f : 0.f) + (s1.fl ? 1.f : 0.f)));
  const float2 ndr = make_float2(-(1.f + (s0.fr ? 1.f : 0.f)), -(1.f + (s1.fr ? 1.f : 0.f)));
  const float2 ndd = make_float2(-(1.f + (s0.fd ? 1.f : 0.f)), -(1.f + (s1.fd ? 1.f : 0.f)));
  const float d0 = 2.f + (s2.fu ? 1.f : 0.f) + (s2.fl ? 1.f : 0.f), dr = 1.f + (s2.fr ? 1.f : 0.f),
              dd = 1.f + (s2.fd ? 1.f : 0.f);
  const float2 a2 = make_float2(a, a);
  const bool act01 = s0.active || s1.active;
  P0[t] = u[0].x;
  P0[t + 32] = u[0].y;
  P0[t + 64] = v[0];
  PR[t] = u[kB - 1].x;
  PR[t + 32] = u[kB - 1].y;
  PR[t + 64] = v[kB - 1];
  PD[t] = u[(kB - 1) * kB].x;
  PD[t + 32] = u[(kB - 1) * kB].y;
  PD[t + 64] = v[(kB - 1) * kB];
  if (t == 0) {
    P0[zero] = P0[kSl + zero] = 0.f;
    PR[zero] = PR[kSl + zero] = 0.f;
    PD[zero] = PD[kSl + zero] = 0.f;
  }
  __syncwarp();

  // two steps per iteration: the port offsets of both parities are fixed
#pragma unroll 2
  for (int s = 0; s < nsteps; ++s) {
    const int cur = (s & 1) * kSl, nxt = kSl - cur;
    if (act01) {
      const float2 vu = make_float2(PD[cur + s0.up], PD[cur + s1.up]);
      const float2 vl = make_float2(PR[cur + s0.lf], PR[cur + s1.lf]);
      const float2 vr = make_float2(P0[cur + s0.rt], P0[cur + s1.rt]);
      const float2 vd = make_float2(P0[cur + s0.dn], P0[cur + s1.dn]);
      block_step2(u, a2, vu, vl, vr, vd, nd0, ndr, ndd);
    }
    if (s2.active)
      block_step(v, a, PD[cur + s2.up], PR[cur + s2.lf], P0[cur + s2.rt], P0[cur + s2.dn], d0, dr, dd);
    P0[nxt + t] = u[0].x;
    P0[nxt + t + 32] = u[0].y;
    P0[nxt + t + 64] = v[0];
    PR[nxt + t] = u[kB - 1].x;
    PR[nxt + t + 32] = u[kB - 1].y;
    PR[nxt + t + 64] = v[kB - 1];
    PD[nxt + t] = u[(kB - 1) * kB].x;
    PD[nxt + t + 32] = u[(kB - 1) * kB].y;
    PD[nxt + t + 64] = v[(kB - 1) * kB];
    __syncwarp();
  }

  // write back the super-tile's member blocks (not the boxes)
  double sum = 0.0;
  if (s0.active && t < f.nb) {
    float w[kB * kB];
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) w[q] = u[q].x;
    sum += write_block(w, f, OX + s0.bx, OY + s0.by, want_sum, out, pout, srec + t);
  }
  if (s1.active && t + 32 < f.nb) {
    float w[kB * kB];
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) w[q] = u[q].y;
    sum += write_block(w, f, OX + s1.bx, OY + s1.by, want_sum, out, pout, srec + t + 32);
  }
  if (s2.active && t + 64 < f.nb) sum += write_block(v, f, OX + s2.bx, OY + s2.by, want_sum, out, pout, srec + t + 64);
  return sum;
}

// Four warps, 320 slots (super-tile side 256 with margins of 33 to 64 cells,
// at most 71 box blocks within a reach of 56): every thread takes slots t
// and t + 128 (paired as in fused_supertile2), and the lanes of two of the
// four warps a third slot 256 + 32 k + lane (k = 0, 1), stepped on its own.
// A CTA of five warps (two slots each) would put two of its warps on one SM
// sub-partition, which then sets the pace of every per-step barrier; with
// four warps each sub-partition holds one warp of the CTA.  The warps with a
// third slot are 0 and 2 or 1 and 3 by the parity of the CTA, so that the
// CTAs resident on one SM spread the heavier warps over all four
// sub-partitions.
constexpr int kQ3Threads = 128;
constexpr int kQ3Slots = 320;

template <int MODE>
__device__ __forceinline__ double fused_supertile3(const float* __restrict__ in, float* __restrict__ out, float a,
                                                   int nsteps, const FGeo& f, int OX, int OY, float* ports,
                                                   bool want_sum, const float* __restrict__ pin,
                                                   float* __restrict__ pout, int64_t srec,
                                                   const int4* __restrict__ desc, int heavy) {
  constexpr int kSl = kQ3Slots + 2;
  constexpr int zero = kQ3Slots;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int k3 = warp == heavy ? 0 : warp == (heavy ^ 2) ? 1 : -1;  // warp-uniform
  const int q0 = t, q1 = t + kQ3Threads, q2 = 2 * kQ3Threads + 32 * (k3 < 0 ? 0 : k3) + lane;
  float* P0 = ports;
  float* PR = ports + 2 * kSl;
  float* PD = ports + 4 * kSl;
  const FSetup s0 = unpack_setup(__ldg(desc + q0)), s1 = unpack_setup(__ldg(desc + q1));
  FSetup s2 = s0;
  s2.active = false;
  if (k3 >= 0) s2 = unpack_setup(__ldg(desc + q2));
  float2 u[kB * kB];
  float v[kB * kB];
  {
    float w0[kB * kB], w1[kB * kB];
    if (s0.active) {
      stage_block(w0, f, OX + s0.bx, OY + s0.by, in, pin, q0 < f.nb ? srec + q0 : (int64_t)s0.rec);
    } else {
#pragma unroll
      for (int q = 0; q < kB * kB; ++q) w0[q] = 0.f;
    }
    if (s1.active) {
      stage_block(w1, f, OX + s1.bx, OY + s1.by, in, pin, q1 < f.nb ? srec + q1 : (int64_t)s1.rec);
    } else {
#pragma unroll
      for (int q = 0; q < kB * kB; ++q) w1[q] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) u[q] = make_float2(w0[q], w1[q]);
  }
  if (s2.active) {
    stage_block(v, f, OX + s2.bx, OY + s2.by, in, pin, q2 < f.nb ? srec + q2 : (int64_t)s2.rec);
  } else {
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) v[q] = 0.f;
  }
  const float2 nd0 = make_float2(-(2.f + (s0.fu ? 1.f : 0.f) + (s0.fl ? 1.f : 0.f)),
                                 -(2.f + (s1.fu ? 1.f : 0.f) + (s1.fl ? 1.f : 0.f)));
  const float2 ndr = make_float2(-(1.f + (s0.fr ? 1.f : 0.f)), -(1.f + (s1.fr ? 1.f : 0.f)));
  const float2 ndd = make_float2(-(1.f + (s0.fd ? 1.f : 0.f)), -(1.f + (s1.fd ? 1.f : 0.f)));
  const float d0 = 2.f + (s2.fu ? 1.f : 0.f) + (s2.fl ? 1.f : 0.f), dr = 1.f + (s2.fr ? 1.f : 0.f),
              dd = 1.f + (s2.fd ? 1.f : 0.f);
  const float2 a2 = make_float2(a, a);
  const bool act01 = s0.active || s1.active;
  P0[q0] = u[0].x;
  P0[q1] = u[0].y;
  PR[q0] = u[kB - 1].x;
  PR[q1] = u[kB - 1].y;
  PD[q0] = u[(kB - 1) * kB].x;
  PD[q1] = u[(kB - 1) * kB].y;
  if (k3 >= 0) {
    P0[q2] = v[0];
    PR[q2] = v[kB - 1];
    PD[q2] = v[(kB - 1) * kB];
  }
  if (t == 0) {
    P0[zero] = P0[kSl + zero] = 0.f;
    PR[zero] = PR[kSl + zero] = 0.f;
    PD[zero] = PD[kSl + zero] = 0.f;
  }
  __syncthreads();

  // two steps per iteration: the port offsets of both parities are fixed
#pragma unroll 2
  for (int s = 0; s < nsteps; ++s) {
    const int cur = (s & 1) * kSl, nxt = kSl - cur;
    if (act01) {
      const float2 vu = make_float2(PD[cur + s0.up], PD[cur + s1.up]);
      const float2 vl = make_float2(PR[cur + s0.lf], PR[cur + s1.lf]);
      const float2 vr = make_float2(P0[cur + s0.rt], P0[cur + s1.rt]);
      const float2 vd = make_float2(P0[cur + s0.dn], P0[cur + s1.dn]);
      block_step2(u, a2, vu, vl, vr, vd, nd0, ndr, ndd);
    }
    if (k3 >= 0) {
      if (s2.active)
        block_step(v, a, PD[cur + s2.up], PR[cur + s2.lf], P0[cur + s2.rt], P0[cur + s2.dn], d0, dr, dd);
      P0[nxt + q2] = v[0];
      PR[nxt + q2] = v[kB - 1];
      PD[nxt + q2] = v[(kB - 1) * kB];
    }
    P0[nxt + q0] = u[0].x;
    P0[nxt + q1] = u[0].y;
    PR[nxt + q0] = u[kB - 1].x;
    PR[nxt + q1] = u[kB - 1].y;
    PD[nxt + q0] = u[(kB - 1) * kB].x;
    PD[nxt + q1] = u[(kB - 1) * kB].y;
    __syncthreads();
  }

  // write back the super-tile's member blocks (slots 256 and up are box blocks)
  double sum = 0.0;
  if (s0.active && q0 < f.nb) {
    float w[kB * kB];
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) w[q] = u[q].x;
    sum += write_block(w, f, OX + s0.bx, OY + s0.by, want_sum, out, pout, srec + q0);
  }
  if (s1.active && q1 < f.nb) {
    float w[kB * kB];
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) w[q] = u[q].y;
    sum += write_block(w, f, OX + s1.bx, OY + s1.by, want_sum, out, pout, srec + q1);
  }
  return sum;
}

__device__ __forceinline__ FGeo make_fgeo(int n, int T, int M, int reach, int log_rho, int R) {
  FGeo f;
  f.n = n;
  f.L = ilog2c(T) - 3;
  int lw = 1, nb = 1;
  for (int i = 0; i < f.L; ++i) nb *= 3;
  for (int i = 0; i < (f.L + 1) / 2; ++i) lw *= 3;
  f.lw = lw;
  f.nb = nb;
  f.W = M / kB;
  f.lW = ilog2c(f.W);
  f.nbox = 6 * f.W * f.W;
  f.reach = reach;
  f.log_rho = log_rho;
  f.R = R;
  f.rec0 = 0;
  int lwR = 1;
  for (int i = 0; i < (R + 1) / 2; ++i) lwR *= 3;
  f.lwR = lwR;
  return f;
}

// BB: member block slots of the 2^L x 2^L box, in row-major order.
__device__ __forceinline__ void bb_table(int* tab, const FGeo& f) {
  const int side = 1 << f.L;
  for (int j = threadIdx.x; j < side * side; j += blockDim.x) {
    const int x = j & (side - 1), y = j >> f.L;
    if ((x & y) == 0) tab[bb_rank(x, y, f.L)] = j;
  }
}

template <int MODE, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) diffusion_fused_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                              float a, int nsteps, int M, int reach, int log_rho,
                                                              Geo g,
                                                              double* __restrict__ partials,
                                                              const float* __restrict__ pin,
                                                              float* __restrict__ pout,
                                                              const int4* __restrict__ desc) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ double red[32];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (partials && threadIdx.x == 0) partials[cta_id()] = 0.0;
    return;
  }
  const FGeo f = make_fgeo(g.n, g.T, M, reach, log_rho, g.R);
  float* ports = fsm;
  int* tab = reinterpret_cast<int*>(fsm + 6 * fused_slots(MAXT));
  if (MODE == kBB && !desc) {
    bb_table(tab, f);
    __syncthreads();
  }
  // the super-tile's index among the member super-tiles (lambda: the CTA's
  // packed index; BB: its rank): its records and its threads' descriptors
  const int64_t st = MODE == kLambda ? cta_id() : (int64_t)bb_rank(sx, sy, f.R);
  const double mine = fused_supertile<MODE, MAXT + 1>(in, out, a, nsteps, f, sx << f.L, sy << f.L, tab, ports,
                                            partials != nullptr, pin, pout, st * f.nb,
                                            desc ? desc + st * blockDim.x : nullptr);
  if (partials) {  // the sum of the result's members, per CTA (uniform branch)
    const double s = block_sum<double>(mine, red);
    if (threadIdx.x == 0) partials[cta_id()] = s;
  }
}

// The same launch with two blocks per thread (fused_supertile2): PMAX
// threads at most, 2 * blockDim.x descriptor slots per CTA.
template <int MODE, int PMAX, int MINB>
__global__ void __launch_bounds__(PMAX, MINB) diffusion_fused2_kernel(const float* __restrict__ in,
                                                                   float* __restrict__ out, float a, int nsteps, int M,
                                                                   int reach, int log_rho, Geo g, double* __restrict__ partials,
                                                                   const float* __restrict__ pin,
                                                                   float* __restrict__ pout,
                                                                   const int4* __restrict__ desc) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ double red[32];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (partials && threadIdx.x == 0) partials[cta_id()] = 0.0;
    return;
  }
  const FGeo f = make_fgeo(g.n, g.T, M, reach, log_rho, g.R);
  const int64_t st = MODE == kLambda ? cta_id() : (int64_t)bb_rank(sx, sy, f.R);
  const double mine = fused_supertile2<MODE, 2 * PMAX + 2>(in, out, a, nsteps, f, sx << f.L, sy << f.L, fsm,
                                                           partials != nullptr, pin, pout, st * f.nb,
                                                           desc + st * 2 * blockDim.x);
  if (partials) {
    const double s = block_sum<double>(mine, red);
    if (threadIdx.x == 0) partials[cta_id()] = s;
  }
}

// One super-tile per CTA of four warps and 320 slots (fused_supertile3);
// three CTAs per SM, so that a thread with three blocks keeps them in
// registers without spilling (7.7 -> 7.4 us per step at k = 16 against four
// CTAs per SM at 128 registers).
template <int MODE>
__global__ void __launch_bounds__(kQ3Threads, 3) diffusion_fused3_kernel(const float* __restrict__ in,
                                                                         float* __restrict__ out, float a, int nsteps,
                                                                         int M, int reach, int log_rho, Geo g,
                                                                         double* __restrict__ partials,
                                                                         const float* __restrict__ pin,
                                                                         float* __restrict__ pout,
                                                                         const int4* __restrict__ desc) {
  __shared__ __align__(16) float ports[6 * (kQ3Slots + 2)];
  __shared__ double red[32];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (partials && threadIdx.x == 0) partials[cta_id()] = 0.0;
    return;
  }
  const FGeo f = make_fgeo(g.n, g.T, M, reach, log_rho, g.R);
  const int64_t st = MODE == kLambda ? cta_id() : (int64_t)bb_rank(sx, sy, f.R);
  const double mine = fused_supertile3<MODE>(in, out, a, nsteps, f, sx << f.L, sy << f.L, ports, partials != nullptr,
                                             pin, pout, st * f.nb, desc + st * kQ3Slots, (int)(cta_id() & 1));
  if (partials) {
    const double s = block_sum<double>(mine, red);
    if (threadIdx.x == 0) partials[cta_id()] = s;
  }
}

// One super-tile of side 128 per CTA of one warp (fused_supertile_w).
template <int MODE, int MINB>
__global__ void __launch_bounds__(32, MINB) diffusion_fused_warp_kernel(const float* __restrict__ in,
                                                                         float* __restrict__ out, float a, int nsteps,
                                                                         int M, int reach, int log_rho, Geo g,
                                                                         double* __restrict__ partials,
                                                                         const float* __restrict__ pin,
                                                                         float* __restrict__ pout,
                                                                         const int4* __restrict__ desc) {
  __shared__ __align__(16) float ports[6 * (kWarpSlots + 2)];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (partials && threadIdx.x == 0) partials[cta_id()] = 0.0;
    return;
  }
  const FGeo f = make_fgeo(g.n, g.T, M, reach, log_rho, g.R);
  const int64_t st = MODE == kLambda ? cta_id() : (int64_t)bb_rank(sx, sy, f.R);
  const double mine = fused_supertile_w<MODE>(in, out, a, nsteps, f, sx << f.L, sy << f.L, ports, partials != nullptr,
                                              pin, pout, st * f.nb, desc + st * kWarpSlots);
  if (partials) {
    const double s = warp_sum(mine);
    if (threadIdx.x == 0) partials[cta_id()] = s;
  }
}

// ------------------------------------- conductivity steps in double-float ---
// The gradient path's state u (and the adjoint state p) in double-float,
// advanced up to `margin` steps per launch like the float32 fused kernels:
// one 8 x 8 block per thread, the super-tile (side 128 at most) and the
// member blocks of its margin boxes within reach, ports exchanged through
// shared memory once per step.  The step is u'_c = u_c + sum_nb c_{c,nb}
// (u_nb - u_c) with c = (a / 2) (kappa_c + kappa_nb) (the edge conductance
// of the gradient path), formed once per launch per link in double-float.
// The flux of a link is computed once and given to both ends: the block's
// 26 links form the tree of bparent, updated in place children first (a
// child's flux with its parent enters the parent's sum before the parent is
// overwritten), the four links to other blocks at the ports.  A launch may
// record the state of its own blocks before every step (and after the last)
// in compact records: 27 members x (hi, lo) and a pad, 14 float4s per block,
// stored float4 by float4 per super-tile like the float32 records.  The
// reverse step of the gradient is the same operator applied to p (it is
// symmetric), so the same kernel carries p back through a segment; the
// kappa gradient is then summed over the segment from the two recorded
// trajectories (kappa_grad_df_kernel).
constexpr int kKapThreads = 128;
constexpr int kKRecF4 = 14;

struct DfSum {
  dfloat s = dfloat(0.f, 0.f);
  bool any = false;
  __device__ __forceinline__ void add(dfloat v) {
    s = any ? s + v : v;
    any = true;
  }
  __device__ __forceinline__ void sub(dfloat v) {
    s = any ? s - v : -v;
    any = true;
  }
};

// One step of a block: c[q] is the coefficient of the link from member q to
// its parent; cu, cl, cr, cd those of the port links (0 where the neighbour
// block is not a member) and vu, vl, vr, vd the neighbour values there.
__device__ __forceinline__ void kblock_step(dfloat (&u)[kB * kB], const dfloat (&c)[kB * kB], dfloat cu, dfloat cl,
                                            dfloat cr, dfloat cd, dfloat vu, dfloat vl, dfloat vr, dfloat vd) {
  DfSum acc[kB * kB];  // fluxes of the children's links, per cell
#pragma unroll
  for (int s = 2 * (kB - 1); s >= 0; --s) {
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int i = s - j;
      if (i < 0 || i >= kB || !amem(i, j)) continue;
      const int q = j * kB + i;
      DfSum f = acc[q];
      if (q != 0) {
        const int pq = bparent(i, j);
        const dfloat fl = c[q] * (u[pq] - u[q]);
        f.add(fl);
        acc[pq].sub(fl);
      } else {
        f.add(cu * (vu - u[0]));
        f.add(cl * (vl - u[0]));
      }
      if (q == kB - 1) f.add(cr * (vr - u[q]));
      if (q == (kB - 1) * kB) f.add(cd * (vd - u[q]));
      u[q] = u[q] + f.s;
    }
  }
}

// Float4 0 of the record of block `rec` (a record's float4s are nb apart).
__device__ __forceinline__ int64_t krec_base(int64_t rec, int nb) {
  const int64_t t = rec % nb;
  return (rec - t) * kKRecF4 + t;
}

__device__ __forceinline__ void krec_write(float4* __restrict__ p, int nb, const dfloat (&u)[kB * kB]) {
  float v[4 * kKRecF4];
  int m = 0;
#pragma unroll
  for (int q = 0; q < kB * kB; ++q) {
    if (!amem(q % kB, q / kB)) continue;
    v[2 * m] = u[q].hi;
    v[2 * m + 1] = u[q].lo;
    ++m;
  }
  v[4 * kKRecF4 - 2] = v[4 * kKRecF4 - 1] = 0.f;
#pragma unroll
  for (int i = 0; i < kKRecF4; ++i) p[(int64_t)i * nb] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

__device__ __forceinline__ void krec_read(const float4* __restrict__ p, int nb, dfloat (&u)[kB * kB]) {
  float v[4 * kKRecF4];
#pragma unroll
  for (int i = 0; i < kKRecF4; ++i) {
    const float4 r = __ldg(p + (int64_t)i * nb);
    v[4 * i] = r.x;
    v[4 * i + 1] = r.y;
    v[4 * i + 2] = r.z;
    v[4 * i + 3] = r.w;
  }
  int m = 0;
#pragma unroll
  for (int q = 0; q < kB * kB; ++q) {
    if (!amem(q % kB, q / kB)) {
      u[q] = dfloat(0.f, 0.f);
      continue;
    }
    u[q] = dfloat(v[2 * m], v[2 * m + 1]);
    ++m;
  }
}

// A record in shared memory (float4s nb apart, as in the trajectory).
__device__ __forceinline__ void krec_read_shared(const float4* p, int nb, dfloat (&u)[kB * kB]) {
  float v[4 * kKRecF4];
#pragma unroll
  for (int i = 0; i < kKRecF4; ++i) {
    const float4 r = p[i * nb];
    v[4 * i] = r.x;
    v[4 * i + 1] = r.y;
    v[4 * i + 2] = r.z;
    v[4 * i + 3] = r.w;
  }
  int m = 0;
#pragma unroll
  for (int q = 0; q < kB * kB; ++q) {
    if (!amem(q % kB, q / kB)) {
      u[q] = dfloat(0.f, 0.f);
      continue;
    }
    u[q] = dfloat(v[2 * m], v[2 * m + 1]);
    ++m;
  }
}

// Member m of a record (its two floats lie in one float4: 2m is even).
__device__ __forceinline__ dfloat krec_member(const float4* __restrict__ p, int nb, int m) {
  const float4 r = __ldg(p + (int64_t)((2 * m) >> 2) * nb);
  return ((2 * m) & 3) ? dfloat(r.z, r.w) : dfloat(r.x, r.y);
}

// A launch of nsteps <= reach <= M steps: `in` -> `out` (embedded double-
// float arrays; out may be null), the state before each step into the
// records traj + s * stride (s = 0 .. nsteps - 1) and, when out is null,
// the final state into record nsteps (traj may be null).
template <int MODE>
__global__ void __launch_bounds__(kKapThreads, 3) kappa_fused_df_kernel(const dfloat* __restrict__ in,
                                                                         dfloat* __restrict__ out,
                                                                         float4* __restrict__ traj, int64_t stride,
                                                                         const float* __restrict__ kappa, dfloat ha,
                                                                         int nsteps, int M, int reach, Geo g,
                                                                         const float* __restrict__ in_f32,
                                                                         float* __restrict__ out_f32) {
  __shared__ __align__(16) float2 kports[6 * (kKapThreads + 1)];
  __shared__ int tab[81];  // BB: member block slots of the super-tile (side <= 128)
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const FGeo f = make_fgeo(g.n, g.T, M, reach, 3, g.R);
  if (MODE == kBB) {
    bb_table(tab, f);
    __syncthreads();
  }
  const int OX = sx << f.L, OY = sy << f.L;
  const FSetup su = fused_setup<MODE>(f, OX, OY, tab);
  const int t = threadIdx.x, SL = blockDim.x + 1, zero = blockDim.x;
  float2* P0 = kports;
  float2* PR = kports + 2 * SL;
  float2* PD = kports + 4 * SL;
  const bool own = su.active && t < f.nb;
  const int64_t st = MODE == kLambda ? cta_id() : (int64_t)bb_rank(sx, sy, f.R);
  float4* rec = traj ? traj + krec_base(st * f.nb + t, f.nb) : nullptr;
  dfloat u[kB * kB], c[kB * kB];
  dfloat cu(0.f), cl(0.f), cr(0.f), cd(0.f);
  size_t base = 0;
#pragma unroll
  for (int q = 0; q < kB * kB; ++q) c[q] = dfloat(0.f, 0.f);
  if (su.active) {
    base = (size_t)(OY + su.by) * kB * (size_t)f.n + (size_t)(OX + su.bx) * kB;
    if (in_f32) {  // a float32 state: each member x as the pair (x, 0)
      float x[kB * kB];
      load_block(x, in_f32 + base, f.n);
#pragma unroll
      for (int q = 0; q < kB * kB; ++q) u[q] = dfloat(x[q], 0.f);
    } else {
      load_block(u, in + base, f.n);
    }
    float kk[kB * kB];
    load_block(kk, kappa + base, f.n);
#pragma unroll
    for (int q = 1; q < kB * kB; ++q)
      if (amem(q % kB, q / kB)) c[q] = ha * two_sum(kk[q], kk[bparent(q % kB, q / kB)]);
    if (su.fu) cu = ha * two_sum(kk[0], __ldg(kappa + base - f.n));
    if (su.fl) cl = ha * two_sum(kk[0], __ldg(kappa + base - 1));
    if (su.fr) cr = ha * two_sum(kk[kB - 1], __ldg(kappa + base + kB));
    if (su.fd) cd = ha * two_sum(kk[(kB - 1) * kB], __ldg(kappa + base + (size_t)kB * f.n));
  } else {
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) u[q] = dfloat(0.f, 0.f);
  }
  P0[t] = make_float2(u[0].hi, u[0].lo);
  PR[t] = make_float2(u[kB - 1].hi, u[kB - 1].lo);
  PD[t] = make_float2(u[(kB - 1) * kB].hi, u[(kB - 1) * kB].lo);
  if (t == 0) {
    P0[zero] = P0[SL + zero] = make_float2(0.f, 0.f);
    PR[zero] = PR[SL + zero] = make_float2(0.f, 0.f);
    PD[zero] = PD[SL + zero] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int s = 0; s < nsteps; ++s) {
    const int cur = (s & 1) * SL, nxt = SL - cur;
    if (rec && own) krec_write(rec + (int64_t)s * stride, f.nb, u);
    if (su.active) {
      const float2 vu = PD[cur + su.up], vl = PR[cur + su.lf], vr = P0[cur + su.rt], vd = P0[cur + su.dn];
      kblock_step(u, c, cu, cl, cr, cd, dfloat(vu.x, vu.y), dfloat(vl.x, vl.y), dfloat(vr.x, vr.y),
                  dfloat(vd.x, vd.y));
    }
    P0[nxt + t] = make_float2(u[0].hi, u[0].lo);
    PR[nxt + t] = make_float2(u[kB - 1].hi, u[kB - 1].lo);
    PD[nxt + t] = make_float2(u[(kB - 1) * kB].hi, u[(kB - 1) * kB].lo);
    __syncthreads();
  }
  if (!own) return;
  if (rec && !out && !out_f32) krec_write(rec + (int64_t)nsteps * stride, f.nb, u);
  if (out_f32) {  // float32: hi + lo rounded once
    float w[kB * kB];
#pragma unroll
    for (int q = 0; q < kB * kB; ++q) w[q] = u[q].hi + u[q].lo;
    store_block(out_f32 + base, f.n, w);
  } else if (out) {
    store_block(out + base, f.n, u);
  }
}

// dJ/dkappa over a segment of nsteps steps from the recorded trajectories:
// utraj record s = u_(t0 + s), ptraj record s = p_(t0 + nsteps - s), so the
// step t0 + s pairs utraj[s] with ptraj[nsteps - 1 - s].  Per link (c, nb)
// and step, (u_nb - u_c) (p_c - p_nb) enters the sums of both ends (the same
// value); at the end gkappa += (a / 2) * sum at every member (read-modify-
// write of the embedded double-float array).  One CTA per super-tile (side
// as the fused launch), one thread per member block; the super-tile's two
// records of a step (contiguous) and the port neighbours' values are copied
// into shared memory (cp.async) before the step's sums.  One stage of 41 KB
// lets four CTAs share an SM, whose copies and sums overlap one another's
// (205 against 221 us per 20-step segment at k = 13 for two stages and two
// CTAs per SM).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kGradThreads = 96;

// Shared memory of one stage: the u and p records of the super-tile
// (2 nb kKRecF4 float4) and eight port values per block (float2).
__host__ __device__ inline int kgrad_stage_bytes(int nb) { return 2 * nb * kKRecF4 * 16 + nb * 8 * 8; }

template <int MODE>
__global__ void __launch_bounds__(kGradThreads, 4) kappa_grad_df_kernel(const float4* __restrict__ utraj,
                                                                          const float4* __restrict__ ptraj,
                                                                          int64_t stride, dfloat* __restrict__ gk,
                                                                          dfloat ha, int nsteps, Geo g, int accumulate,
                                                                          float* __restrict__ out_f32) {
  extern __shared__ __align__(16) float4 gsm[];
  __shared__ int tab[81];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const FGeo f = make_fgeo(g.n, g.T, kB, 1, 3, g.R);
  if (MODE == kBB) {
    bb_table(tab, f);
    __syncthreads();
  }
  const int t = threadIdx.x, nb = f.nb;
  const bool act = t < nb;
  const int64_t st = MODE == kLambda ? cta_id() : (int64_t)bb_rank(sx, sy, f.R);
  const int64_t tile0 = st * nb * kKRecF4;  // the super-tile's records: float4 [tile0, tile0 + nb * 14)
  int GX = 0, GY = 0;
  bool fu = false, fl = false, fr = false, fd = false;
  int64_t nbr[4] = {0, 0, 0, 0};  // float4 holding the port neighbour's member (up, left, right, down)
  if (act) {
    int bx, by;
    member_block<MODE>(t, f, tab, bx, by);
    GX = (sx << f.L) + bx;
    GY = (sy << f.L) + by;
    const int nblk = f.n / kB;
    fu = block_member(GX, GY - 1, nblk);
    fl = block_member(GX - 1, GY, nblk);
    fr = block_member(GX + 1, GY, nblk);
    fd = block_member(GX, GY + 1, nblk);
    // members 26 ((0,7)), 7 ((7,0)), 0, 0: float4 (2m) / 4 of the record
    if (fu) nbr[0] = krec_base(block_record<MODE>(GX, GY - 1, f), nb) + (int64_t)13 * nb;
    if (fl) nbr[1] = krec_base(block_record<MODE>(GX - 1, GY, f), nb) + (int64_t)3 * nb;
    if (fr) nbr[2] = krec_base(block_record<MODE>(GX + 1, GY, f), nb);
    if (fd) nbr[3] = krec_base(block_record<MODE>(GX, GY + 1, f), nb);
  }
  const int sb = kgrad_stage_bytes(nb) / 16;  // float4 per stage
  auto stage_u = [&](int b) { return gsm + b * sb; };
  auto stage_p = [&](int b) { return gsm + b * sb + nb * kKRecF4; };
  auto stage_n = [&](int b) { return reinterpret_cast<float2*>(gsm + b * sb + 2 * nb * kKRecF4); };
  // copy step s's records and port values into stage b (one commit group)
  auto load = [&](int b, int s) {
    const float4* U = utraj + (int64_t)s * stride + tile0;
    const float4* P = ptraj + (int64_t)(nsteps - 1 - s) * stride + tile0;
    float4* du = stage_u(b);
    float4* dp = stage_p(b);
    for (int i = t; i < nb * kKRecF4; i += kGradThreads) {
      cp_async16(du + i, U + i);
      cp_async16(dp + i, P + i);
    }
    if (act) {
      const float4* Ua = utraj + (int64_t)s * stride;
      const float4* Pa = ptraj + (int64_t)(nsteps - 1 - s) * stride;
      float2* dn = stage_n(b) + t * 8;
      // the member's float2: member m is floats 2m, 2m + 1: (0,7) = member 26 -> .x.y of float4 13,
      // (7,0) = member 7 -> .z.w of float4 3, (0,0) = member 0 -> .x.y of float4 0
      const int off[4] = {0, 2, 0, 0};
      const bool has[4] = {fu, fl, fr, fd};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!has[q]) continue;
        cp_async8(dn + q, reinterpret_cast<const float*>(Ua + nbr[q]) + off[q]);
        cp_async8(dn + 4 + q, reinterpret_cast<const float*>(Pa + nbr[q]) + off[q]);
      }
    }
    cp_async_commit();
  };
  DfSum gs[kB * kB];
  for (int s = 0; s < nsteps; ++s) {
    const int b = 0;  // one stage
    load(b, s);
    cp_async_wait<0>();
    __syncthreads();
    if (act) {
      dfloat u[kB * kB], p[kB * kB];
      krec_read_shared(stage_u(b) + t, nb, u);
      krec_read_shared(stage_p(b) + t, nb, p);
#pragma unroll
      for (int q = 1; q < kB * kB; ++q) {
        if (!amem(q % kB, q / kB)) continue;
        const int pq = bparent(q % kB, q / kB);
        const dfloat w = (u[pq] - u[q]) * (p[q] - p[pq]);
        gs[q].add(w);
        gs[pq].add(w);
      }
      const float2* dn = stage_n(b) + t * 8;
      if (fu) {
        const float2 a = dn[0], c = dn[4];
        gs[0].add((dfloat(a.x, a.y) - u[0]) * (p[0] - dfloat(c.x, c.y)));
      }
      if (fl) {
        const float2 a = dn[1], c = dn[5];
        gs[0].add((dfloat(a.x, a.y) - u[0]) * (p[0] - dfloat(c.x, c.y)));
      }
      if (fr) {
        const float2 a = dn[2], c = dn[6];
        gs[kB - 1].add((dfloat(a.x, a.y) - u[kB - 1]) * (p[kB - 1] - dfloat(c.x, c.y)));
      }
      if (fd) {
        const float2 a = dn[3], c = dn[7];
        const int q = (kB - 1) * kB;
        gs[q].add((dfloat(a.x, a.y) - u[q]) * (p[q] - dfloat(c.x, c.y)));
      }
    }
    __syncthreads();  // the stage is refilled by the next step's copies
  }
  if (!act) return;
  // gk += (a / 2) sums (gk taken as 0 without `accumulate`), into gk, or
  // into out_f32 as float32 (hi + lo rounded once) when that is not null
  const size_t off = (size_t)GY * kB * (size_t)f.n + (size_t)GX * kB;
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    dfloat v[kB];
    if (accumulate) {
      ld4(gk + off + (size_t)j * f.n, v);
      ld4(gk + off + (size_t)j * f.n + 4, v + 4);
    } else {
#pragma unroll
      for (int i = 0; i < kB; ++i) v[i] = dfloat(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kB; ++i) v[i] = amem(i, j) && gs[j * kB + i].any ? v[i] + ha * gs[j * kB + i].s
                                                                           : (amem(i, j) ? v[i] : dfloat(0.f, 0.f));
    if (out_f32) {
      float o[kB];
#pragma unroll
      for (int i = 0; i < kB; ++i) o[i] = v[i].hi + v[i].lo;
      st4(out_f32 + off + (size_t)j * f.n, o);
      st4(out_f32 + off + (size_t)j * f.n + 4, o + 4);
    } else {
      st4(gk + off + (size_t)j * f.n, v);
      st4(gk + off + (size_t)j * f.n + 4, v + 4);
    }
  }
}

// ---------------------------------------------------------------- batches ---
// Persistent launch over the member super-tiles of many instances: CTA c
// takes items c, c + gridDim.x, ...; item w belongs to the last instance
// whose first item is <= w (binary search on the prefix table), and is that
// instance's super-tile lambda(w - first) at level R (Theorem 1).
__device__ __forceinline__ int batch_instance(const BatchInst* __restrict__ inst, int count, int64_t w) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].first <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(288, 4) diffusion_batch_kernel(const BatchInst* __restrict__ inst, int count,
                                                              int64_t items, int which, float a, int nsteps, int M,
                                                              int reach, int T, const float* __restrict__ pin,
                                                              float* __restrict__ pout,
                                                              const int4* __restrict__ desc) {
  extern __shared__ __align__(16) float fsm[];
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const BatchInst I = inst[batch_instance(inst, count, w)];
    const int64_t om = w - I.first;
    int sx, sy;
    warp_lambda((uint32_t)(om % I.lwR), (uint32_t)(om / I.lwR), I.R, sx, sy);
    FGeo f = make_fgeo(I.n, T, M, reach, 3, I.R);
    f.rec0 = I.first * f.nb;  // item w's records start at w * nb
    fused_supertile<kLambda, 289>(pin ? nullptr : (which ? I.b : I.a), pout ? nullptr : (which ? I.a : I.b), a, nsteps,
                              f, sx << f.L, sy << f.L, nullptr, fsm, false, pin, pout, w * f.nb,
                              desc ? desc + w * blockDim.x : nullptr);
  }
}

// Batches in the four-warp layout of fused_supertile3 (super-tile side 256,
// 320 slots): one CTA per item (its instance by binary search, its
// super-tile by lambda at the instance's level), three CTAs per SM.
__global__ void __launch_bounds__(kQ3Threads, 3) diffusion_batch3_kernel(const BatchInst* __restrict__ inst,
                                                                         int count, int which, float a, int nsteps,
                                                                         int M, int reach, int T,
                                                                         const float* __restrict__ pin,
                                                                         float* __restrict__ pout,
                                                                         const int4* __restrict__ desc) {
  __shared__ __align__(16) float ports[6 * (kQ3Slots + 2)];
  const int64_t w = blockIdx.x;
  const BatchInst I = inst[batch_instance(inst, count, w)];
  const int64_t om = w - I.first;
  int sx, sy;
  warp_lambda((uint32_t)(om % I.lwR), (uint32_t)(om / I.lwR), I.R, sx, sy);
  FGeo f = make_fgeo(I.n, T, M, reach, 3, I.R);
  f.rec0 = I.first * f.nb;  // item w's records start at w * nb
  fused_supertile3<kLambda>(pin ? nullptr : (which ? I.b : I.a), pout ? nullptr : (which ? I.a : I.b), a, nsteps, f,
                            sx << f.L, sy << f.L, ports, false, pin, pout, w * f.nb, desc + w * kQ3Slots,
                            (int)(w & 1));
}

// The batch launch's per-thread setups, item by item (w * blockDim.x + t).
__global__ void __launch_bounds__(512) batch_describe_kernel(const BatchInst* __restrict__ inst, int count,
                                                             int64_t items, int M, int reach, int T,
                                                             int4* __restrict__ desc) {
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const BatchInst I = inst[batch_instance(inst, count, w)];
    const int64_t om = w - I.first;
    int sx, sy;
    warp_lambda((uint32_t)(om % I.lwR), (uint32_t)(om / I.lwR), I.R, sx, sy);
    FGeo f = make_fgeo(I.n, T, M, reach, 3, I.R);
    f.rec0 = I.first * f.nb;
    const FSetup s = fused_setup<kLambda>(f, sx << f.L, sy << f.L, nullptr);
    desc[w * blockDim.x + threadIdx.x] = pack_setup(s);
    __syncthreads();  // the setup's shared tables are rewritten for the next item
  }
}

// Per-super-tile sums of the member cells (FP32 within a 16-byte chunk, FP64
// above; fixed order), then per instance in item order.
__global__ void __launch_bounds__(512) batch_partials_kernel(const BatchInst* __restrict__ inst, int count,
                                                             int64_t items, int which, int T,
                                                             double* __restrict__ partials) {
  __shared__ double warp_sum[16];
  const int L = ilog2c(T) - 3;
  int nb = 1, lw = 1;
  for (int i = 0; i < L; ++i) nb *= 3;
  for (int i = 0; i < (L + 1) / 2; ++i) lw *= 3;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const BatchInst I = inst[batch_instance(inst, count, w)];
    const int64_t om = w - I.first;
    int sx, sy;
    warp_lambda((uint32_t)(om % I.lwR), (uint32_t)(om / I.lwR), I.R, sx, sy);
    const float* buf = which ? I.b : I.a;
    double acc = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      int bx, by;
      lambda_scalar((uint32_t)(t % lw), (uint32_t)(t / lw), L, bx, by);
      const float* p = buf + ((size_t)((sy << L) + by) * kB) * (size_t)I.n + (size_t)((sx << L) + bx) * kB;
#pragma unroll
      for (int j = 0; j < kB; ++j) {
        const float4 v = mask_chunk(__ldg(reinterpret_cast<const float4*>(p + (size_t)j * I.n)), 0, j);
        acc += (double)((v.x + v.y) + (v.z + v.w));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 v = mask_chunk(__ldg(reinterpret_cast<const float4*>(p + (size_t)j * I.n + 4)), 4, j);
        acc += (double)((v.x + v.y) + (v.z + v.w));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += warp_sum[i];
      partials[w] = s;
    }
    __syncthreads();
  }
}

__global__ void batch_sums_kernel(const BatchInst* __restrict__ inst, int count, int64_t items,
                                  const double* __restrict__ partials, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t e = i + 1 < count ? inst[i + 1].first : items;
  double s = 0.0;
  for (int64_t w = inst[i].first; w < e; ++w) s += partials[w];
  out[i] = s;
}

// One descriptor per thread of a fused launch (the launch's geometry, one
// CTA per member super-tile): the setup every launch of the configuration
// would compute, written once.
template <int MODE>
__global__ void __launch_bounds__(512) fused_describe_kernel(Geo g, int M, int reach, int log_rho,
                                                             int4* __restrict__ desc) {
  extern __shared__ __align__(16) float fsm[];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) return;
  const FGeo f = make_fgeo(g.n, g.T, M, reach, log_rho, g.R);
  int* tab = reinterpret_cast<int*>(fsm);
  if (MODE == kBB) {
    bb_table(tab, f);
    __syncthreads();
  }
  const int64_t st = MODE == kLambda ? cta_id() : (int64_t)bb_rank(sx, sy, f.R);
  const FSetup s = fused_setup<MODE>(f, sx << f.L, sy << f.L, tab);
  desc[st * blockDim.x + threadIdx.x] = pack_setup(s);
}

template <int MODE>
cudaError_t go(const Launch& L, const float* in, float* out, float a, int nsteps, int margin, int reach, int log_rho,
               double* partials, const float* pin, float* pout, const int4* desc, cudaStream_t s) {
  // the smallest CTA class that holds the launch: more CTAs per SM
  auto run = [&](auto* k) -> cudaError_t {
    cudaError_t e = allow_smem((const void*)k, L.smem);
    if (e != cudaSuccess) return e;
    k<<<L.grid, L.threads, L.smem, s>>>(in, out, a, nsteps, margin, reach, log_rho, L.geo, partials, pin, pout, desc);
    return cudaGetLastError();
  };
  if (L.threads <= 288) return run(diffusion_fused_kernel<MODE, 288, 4>);
  if (L.threads <= 352) return run(diffusion_fused_kernel<MODE, 352, 3>);
  return run(diffusion_fused_kernel<MODE, 512, 2>);
}

// Two blocks per thread (with descriptors): L.threads / 2 threads, in the
// class holding them; ports of 2 * class + 2 slots per parity.
template <int MODE>
cudaError_t go2(const Launch& L, const float* in, float* out, float a, int nsteps, int margin, int reach, int log_rho,
                double* partials, const float* pin, float* pout, const int4* desc, cudaStream_t s) {
  const int threads = L.threads / 2;
  auto run = [&](auto* k, int pmax) -> cudaError_t {
    const int smem = 6 * (2 * pmax + 2) * 4;
    cudaError_t e = allow_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<L.grid, threads, smem, s>>>(in, out, a, nsteps, margin, reach, log_rho, L.geo, partials, pin, pout, desc);
    return cudaGetLastError();
  };
  if (threads <= 160) return run(diffusion_fused2_kernel<MODE, 160, 4>, 160);
  if (threads <= 176) return run(diffusion_fused2_kernel<MODE, 176, 3>, 176);
  return run(diffusion_fused2_kernel<MODE, 256, 2>, 256);
}


// One warp per CTA (super-tile side 128, 96 slots, with descriptors).
template <int MODE>
cudaError_t gow(const Launch& L, const float* in, float* out, float a, int nsteps, int margin, int reach, int log_rho,
                double* partials, const float* pin, float* pout, const int4* desc, cudaStream_t s) {
  diffusion_fused_warp_kernel<MODE, 16><<<L.grid, 32, 0, s>>>(in, out, a, nsteps, margin, reach, log_rho, L.geo,
                                                                partials, pin, pout, desc);
  return cudaGetLastError();
}

int member_blocks(int T) {
  int nb = 1;
  for (int i = 0; i < ilog2c(T) - 3; ++i) nb *= 3;
  return nb;
}

}  // namespace

// Margin of a fused launch: the smallest power of two >= spl, at least the
// block side (8, 16, 32, 64 or 128 cells: whole blocks, W a power of two).
int fused_margin(int steps_per_launch) {
  int m = kB;
  while (m < steps_per_launch) m *= 2;
  return m;
}

// Member blocks of the margin boxes within `reach` of the super-tile
// (box_distance), the most any member super-tile has: counted over every
// member super-tile of a 64 x 64 grid of super-tiles.  Which box blocks are
// members depends only on which of the super-tile's eight neighbours are
// members (and on the array's edge, which only removes blocks), and every
// such neighbourhood of the gasket occurs in that grid.  Cached.
int box_cap_reach(int L, int W, int reach) {
  static std::atomic<int> cache[6][kMaxW + 1][129];
  if (L < 1 || L > 5 || W < 1 || W > kMaxW) return 0;
  reach = reach < 0 ? 0 : reach > 128 ? 128 : reach;
  const int hit = cache[L][W][reach].load(std::memory_order_relaxed);
  if (hit > 0) return hit - 1;
  const int side = 1 << L, W2 = W * W;
  constexpr int kGrid = 64;
  const int nblk = kGrid * side;
  int best = 0;
  for (int sy = 0; sy < kGrid; ++sy)
    for (int sx = 0; sx < kGrid; ++sx) {
      if (sx & sy) continue;
      int c = 0;
      for (int b = 0; b < 6 * W2; ++b) {
        int qx, qy, r = b;
        if (r < W2) { qx = -W + r % W; qy = r / W; }
        else if ((r -= W2) < W2) { qx = r % W; qy = -W + r / W; }
        else if ((r -= W2) < 2 * W2) { qx = side + r % W; qy = -W + r / W; }
        else { r -= 2 * W2; qx = -W + r % (2 * W); qy = side + r / (2 * W); }
        const int gx = sx * side + qx, gy = sy * side + qy;
        if (gx < 0 || gy < 0 || gx >= nblk || gy >= nblk || (gx & gy) != 0) continue;
        if (box_distance(qx, qy, side) <= reach) ++c;
      }
      best = c > best ? c : best;
    }
  cache[L][W][reach].store(best + 1, std::memory_order_relaxed);
  return best;
}

// Threads of a fused launch: one per member block of the super-tile and per
// member block of the margin boxes within `reach` (the steps per launch the
// configuration serves, at most the margin), rounded up to whole warps; 0 if
// the super-tile does not fit (side < 16 or < 2 M, a margin that is not 8
// times a power of two up to 128, a reach outside [1, M], more than
// kFusedMaxThreads threads).
int fused_threads(const Geo& g, int rho, int margin, int reach) {
  (void)rho;
  const int W = margin / kB;
  if (g.T < 2 * kB || g.T < 2 * margin || margin < kB || margin % kB != 0 || W > kMaxW || (W & (W - 1)) != 0 ||
      reach < 1 || reach > margin)
    return 0;
  const int t = (member_blocks(g.T) + box_cap_reach(ilog2c(g.T) - 3, W, reach) + 31) / 32 * 32;
  return t > kFusedMaxThreads ? 0 : t;
}

int fused_smem_bytes(const Geo& g, int margin, int reach) {
  return 6 * fused_slots(fused_class(fused_threads(g, 0, margin, reach))) * 4 + member_blocks(g.T) * 4;
}

int fused_batch_smem_bytes(int threads) {
  (void)threads;  // the batch kernel's class: 288 threads
  return 6 * fused_slots(288) * 4;
}

const void* fused_batch_kernel() { return (const void*)diffusion_batch_kernel; }

cudaError_t launch_batch_describe(const BatchInst* inst, int count, int64_t items, int margin, int reach, int T,
                                  int ctas, int threads, int4* desc, cudaStream_t s) {
  Geo g{};
  g.T = T;
  if (fused_threads(g, 0, margin, reach) != threads || (threads > 288 && threads != kQ3Slots) || ctas < 1)
    return cudaErrorInvalidValue;
  batch_describe_kernel<<<ctas, threads, 0, s>>>(inst, count, items, margin, reach, T, desc);
  return cudaGetLastError();
}

cudaError_t launch_diffusion_batch(const BatchInst* inst, int count, int64_t items, int which, float a, int nsteps,
                                   int margin, int reach, int T, int ctas, int threads, cudaStream_t s,
                                   const float* pin, float* pout, const int4* desc) {
  if (nsteps < 1 || nsteps > reach || ctas < 1) return cudaErrorInvalidValue;
  Geo g{};
  g.T = T;
  if (fused_threads(g, 0, margin, reach) != threads) return cudaErrorInvalidValue;
  if (threads == kQ3Slots) {  // four warps, one CTA per item (needs the descriptors)
    if (!desc || items < 1 || items > 0x7fffffff) return cudaErrorInvalidValue;
    diffusion_batch3_kernel<<<(unsigned)items, kQ3Threads, 0, s>>>(inst, count, which, a, nsteps, margin, reach, T,
                                                                    pin, pout, desc);
    return cudaGetLastError();
  }
  if (threads > 288) return cudaErrorInvalidValue;
  diffusion_batch_kernel<<<ctas, threads, fused_batch_smem_bytes(threads), s>>>(inst, count, items, which, a, nsteps,
                                                                               margin, reach, T, pin, pout, desc);
  return cudaGetLastError();
}

cudaError_t launch_batch_reduce(const BatchInst* inst, int count, int64_t items, int which, int T, int ctas,
                                double* partials, double* out, cudaStream_t s) {
  batch_partials_kernel<<<ctas, 256, 0, s>>>(inst, count, items, which, T, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_sums_kernel<<<(count + 127) / 128, 128, 0, s>>>(inst, count, items, partials, out);
  return cudaGetLastError();
}

cudaError_t launch_diffusion_fused(int mode, int log_rho, int margin, int reach, const Launch& L, const float* in,
                                   float* out, float a, int nsteps, cudaStream_t s, double* partials, const float* pin,
                                   float* pout, const int4* desc) {
  if (nsteps < 0 || nsteps > reach || log_rho < 2 || fused_threads(L.geo, 0, margin, reach) != L.threads ||
      (!in && !pin) || (!out && !pout))
    return cudaErrorInvalidValue;
  // two blocks per thread (the descriptors give each thread its two slots)
  // for the larger CTA classes (margins of 64 cells and more: launches of
  // many steps, bound by their arithmetic); short launches are bound by their
  // loads and stores, which one block per thread keeps more of in flight
  if (desc && L.geo.T == kWarpSide && L.threads == kWarpSlots)
    return mode == kLambda ? gow<kLambda>(L, in, out, a, nsteps, margin, reach, log_rho, partials, pin, pout, desc, s)
                           : gow<kBB>(L, in, out, a, nsteps, margin, reach, log_rho, partials, pin, pout, desc, s);
  if (desc && L.threads == kQ3Slots) {
    if (mode == kLambda)
      diffusion_fused3_kernel<kLambda><<<L.grid, kQ3Threads, 0, s>>>(in, out, a, nsteps, margin, reach, log_rho, L.geo,
                                                                     partials, pin, pout, desc);
    else
      diffusion_fused3_kernel<kBB><<<L.grid, kQ3Threads, 0, s>>>(in, out, a, nsteps, margin, reach, log_rho, L.geo,
                                                                 partials, pin, pout, desc);
    return cudaGetLastError();
  }
  if (desc && L.threads > 288)
    return mode == kLambda ? go2<kLambda>(L, in, out, a, nsteps, margin, reach, log_rho, partials, pin, pout, desc, s)
                           : go2<kBB>(L, in, out, a, nsteps, margin, reach, log_rho, partials, pin, pout, desc, s);
  return mode == kLambda ? go<kLambda>(L, in, out, a, nsteps, margin, reach, log_rho, partials, pin, pout, desc, s)
                         : go<kBB>(L, in, out, a, nsteps, margin, reach, log_rho, partials, pin, pout, desc, s);
}

int64_t fused_descriptors(const Launch& L) {
  int64_t st = 1;  // member super-tiles: 3^R
  for (int i = 0; i < L.geo.R; ++i) st *= 3;
  return st * L.threads;
}

cudaError_t launch_fused_describe(int mode, int log_rho, int margin, int reach, const Launch& L, int4* desc,
                                  cudaStream_t s) {
  if (fused_threads(L.geo, 0, margin, reach) != L.threads) return cudaErrorInvalidValue;
  const int smem = member_blocks(L.geo.T) * 4;  // BB slot table
  if (mode == kLambda)
    fused_describe_kernel<kLambda><<<L.grid, L.threads, smem, s>>>(L.geo, margin, reach, log_rho, desc);
  else
    fused_describe_kernel<kBB><<<L.grid, L.threads, smem, s>>>(L.geo, margin, reach, log_rho, desc);
  return cudaGetLastError();
}

int fused_warp_slots() { return kWarpSlots; }
int fused_q3_slots() { return kQ3Slots; }

// Geometry of the double-float conductivity launches: super-tiles of side
// min(128, n) (k >= 4), margins min(32, side / 2); false if unsupported.
bool kappa_fused_geometry(int k, int mode, Launch& L, int& margin) {
  if (k < 4 || k > 16) return false;
  const int T = k >= 7 ? 128 : 1 << k;
  margin = T / 2 < 32 ? T / 2 : 32;
  if (!supertile_grid(k, 3, mode, ilog2c(T) - 3, L)) return false;
  L.threads = fused_threads(L.geo, 8, margin, margin);
  L.smem = 0;
  return L.threads > 0 && L.threads <= kKapThreads;
}

int64_t kappa_record_float4s(int k) { return fused_records(k) * kKRecF4; }

cudaError_t launch_kappa_fused_df(int mode, int k, const dfloat* in, dfloat* out, float4* traj, const float* kappa,
                                  dfloat ha, int nsteps, cudaStream_t s, const float* in_f32, float* out_f32) {
  Launch L;
  int margin = 0;
  if (!kappa_fused_geometry(k, mode, L, margin) || nsteps < 1 || nsteps > margin) return cudaErrorInvalidValue;
  const int threads = fused_threads(L.geo, 8, margin, nsteps);
  const int64_t stride = kappa_record_float4s(k);
  if (mode == kLambda)
    kappa_fused_df_kernel<kLambda><<<L.grid, threads, 0, s>>>(in, out, traj, stride, kappa, ha, nsteps, margin, nsteps,
                                                              L.geo, in_f32, out_f32);
  else
    kappa_fused_df_kernel<kBB><<<L.grid, threads, 0, s>>>(in, out, traj, stride, kappa, ha, nsteps, margin, nsteps,
                                                          L.geo, in_f32, out_f32);
  return cudaGetLastError();
}

cudaError_t launch_kappa_grad_df(int mode, int k, const float4* utraj, const float4* ptraj, dfloat* gk, dfloat ha,
                                 int nsteps, cudaStream_t s, int accumulate, float* out_f32) {
  Launch L;
  int margin = 0;
  if (!kappa_fused_geometry(k, mode, L, margin) || nsteps < 1) return cudaErrorInvalidValue;
  const int64_t stride = kappa_record_float4s(k);
  const int smem = kgrad_stage_bytes(member_blocks(L.geo.T));
  auto run = [&](auto* k) -> cudaError_t {
    cudaError_t e = allow_smem((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<L.grid, kGradThreads, smem, s>>>(utraj, ptraj, stride, gk, ha, nsteps, L.geo, accumulate, out_f32);
    return cudaGetLastError();
  };
  return mode == kLambda ? run(kappa_grad_df_kernel<kLambda>) : run(kappa_grad_df_kernel<kBB>);
}

int64_t fused_records(int k) {
  int64_t r = 1;
  for (int i = 3; i < k; ++i) r *= 3;
  return k >= 3 ? r : 0;
}

int fused_record_bytes() { return kRecF4 * 16; }

}  // namespace fractal
