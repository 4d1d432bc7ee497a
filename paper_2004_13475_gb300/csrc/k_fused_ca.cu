// Temporally fused automaton: one CTA advances its member super-tile by up to
// `margin` B3/S23 steps per launch on a bit image in shared memory.
//
// Word tiles.  The state is packed one bit per cell, 32 cells of a row per
// word.  Inside a super-tile of side T (T >= 32, super-tile coordinates) the
// word of row y covering columns [32c, 32c + 32) holds members iff
// c & (y >> 5) == 0, whatever the plan's rho: the CTA works on 32 x 32-cell
// word tiles, the member ones being the level-log2(T/32) gasket of word
// tiles, enumerated with lambda (Sec. 5.1 further unrolling) or, in BB mode,
// by discarding the non-member slots of the 2^j x 2^j bounding box.  A word
// tile covers whole rho x rho tiles for rho <= 32; its 32-byte row segments
// are the sectors a rho = 32 tile reads and writes.  Cells of the segment in
// non-member rho-tiles are non-members and are written back as 0.
//
// Margin boxes.  Influence travels along member cells only (non-members are
// dead for ever), at one cell per step in the 8-neighbourhood.  For s <= M <=
// T/2 every member reached from the super-tile in s steps lies in
//   left   [-M, 0) x [0, M)        top    [0, M) x [-M, 0)
//   right  [T, T+M) x [-M, M]      bottom [-M, M] x [T, T+M)
// (the right and bottom boxes reach one row / column further than the
// diffusion's 4-neighbour ones: the corner cell (T-1, 0) reaches (T, M) by M
// diagonal moves).  For M <= 31 these are the words of column -1 (left,
// bottom), 0 (top, bottom) and T/32 (right).  The kernel stages them with
// the margin rounded up to a multiple of 8, ME8, and the right box to rows
// [-ME8, ME8 + 8), so that every box piece starts on a row that is a
// multiple of 8 and has a multiple of 8 rows (the words added belong to no
// other task: staging more of the state is always correct).  Box words are
// evolved with the tiles; cells whose
// neighbours were not staged go wrong from the box edge inwards, one cell
// per step, and never reach the super-tile within s steps.
//
// Tasks.  A task is one word column of at most 32 consecutive rows (a word
// tile, or a piece of a box), taken by eight lanes: lane i of the eight keeps
// rows 4i .. 4i + 3 of it in registers.  The bit image is stored by columns
// (a column's rows are consecutive words, every four of them one 16-byte
// group), so a lane's four words, and the four beside them in the columns
// left and right, are one 16-byte access each, and the eight lanes of a task
// read 128 consecutive bytes (no bank conflict).  Each step a lane forms the
// three-cell horizontal sums of its four rows (funnel shifts with the left
// word's top cell and the right word's bottom cell, a full adder), takes
// the sums of the rows above and below from the neighbouring lanes by
// shuffles (the first and last lane of a task form them from the image), and
// applies the rule to its four rows.  Box pieces are staged from a row that
// is a multiple of 8 with a multiple of 8 rows (the margin rounded up to
// ME8, the right box to rows [-ME8, ME8 + 8)), so that a lane holds four
// rows of its task or none; the words added belong to no other task.  Every
// staged word is the word of exactly one task lane; every other word of the
// image is 0 and stays 0.
//
// The rule modulo 4.  No member cell of the gasket has more than 5 member
// neighbours (the neighbourhood of a cell inside one of the three copies of
// the level-(j-1) gasket is that copy's, and the copies meet at two corners
// and one diagonal contact whose cells have at most 5; a brute-force count
// over levels 2 to 13 agrees), and non-members are always dead.  So the
// nine-cell sum S = neighbours + self is at most 6, and with m = S mod 4:
// alive next iff m == 3 (three neighbours, or two and alive) or m == 0 and
// alive now (S == 4: three neighbours and alive; S == 0 leaves a dead cell
// dead).  Two bits of the sum suffice.
//
// Records.  Between the launches of one call the state stays in compact
// records, one per member word tile: its 32 words (row order), 128 bytes
// instead of 32 rows of 32 bytes.  Record s * 3^wlev + j holds word tile j
// (lambda or BB rank order) of member super-tile s (its index in the level-R
// packed grid, or its BB rank); the first launch of a call reads the embedded
// array and the last one writes it.
#include "blocks.cuh"
#include "launch.h"

namespace fractal {
namespace {

constexpr int kCaRows = 4;   // rows per lane
constexpr int kCaLanes = 8;  // lanes per task (32 / kCaRows)
constexpr int kCaRow0 = 36;  // image row of super-tile row 0 (a multiple of 4)

// Image geometry: word columns [-2, T/32 + 1] of rows [-36, T + 36) whatever
// the margin (the box pieces reach rows -32 .. T + 31 and a lane reads one
// row beyond its four on each side), so that a column's stride is a
// compile-time constant and every lane's eight rows are 16-byte aligned.
// Word (c, y) is at (c + 2) * ca_col(T) + y + 36.
__host__ __device__ constexpr int ca_cols(int T) { return (T >> 5) + 4; }
__host__ __device__ constexpr int ca_col(int T) { return T + 2 * kCaRow0; }
__host__ __device__ constexpr int ca_image_words(int T) { return ca_cols(T) * ca_col(T); }

// Tasks of a super-tile: word tiles first, then the seven box pieces.
__host__ __device__ inline int ca_tasks(int wtiles) { return wtiles + 7; }

// Task -> (word column c, first row y0, rows) in super-tile coordinates; ME8:
// the margin rounded up to a multiple of 8.  y0 and rows are multiples of 8.
__device__ __forceinline__ void ca_task(int j, int wtiles, const uint32_t* tab, int T, int ME8, int& c, int& y0,
                                        int& rows) {
  if (j < wtiles) {
    const uint32_t e = tab[j];
    c = (int)(e & 0xffffu);
    y0 = (int)(e >> 16) * 32;
    rows = 32;
    return;
  }
  const int right = 2 * ME8 + 8;  // rows of the right box, [-ME8, ME8 + 8)
  switch (j - wtiles) {
    case 0: c = -1; y0 = 0; rows = ME8; return;                                  // left
    case 1: c = 0; y0 = -ME8; rows = ME8; return;                                // top
    case 2: c = T >> 5; y0 = -ME8; rows = min(right, 32); return;                // right, in pieces of 32
    case 3: c = T >> 5; y0 = -ME8 + 32; rows = min(max(right - 32, 0), 32); return;
    case 4: c = T >> 5; y0 = -ME8 + 64; rows = max(right - 64, 0); return;
    case 5: c = -1; y0 = T; rows = ME8; return;                                  // bottom, left word
    default: c = 0; y0 = T; rows = ME8; return;                                  // bottom, right word
  }
}

// 32 bytes of 0/1 cells -> 32 bits (bit i = cell i).
__device__ __forceinline__ uint32_t pack32(uint4 a, uint4 b) {
  return nz4(a.x) | nz4(a.y) << 4 | nz4(a.z) << 8 | nz4(a.w) << 12 | nz4(b.x) << 16 | nz4(b.y) << 20 |
         nz4(b.z) << 24 | nz4(b.w) << 28;
}

// Three-cell horizontal sum of a row word w with its left and right words,
// as two bit planes: bit i of (s, k) = cells i-1, i, i+1 summed (s the low
// bit, k the carry).
__device__ __forceinline__ void row_sum3(uint32_t l, uint32_t w, uint32_t r, uint32_t& s, uint32_t& k) {
  const uint32_t a = __funnelshift_l(l, w, 1), c = __funnelshift_r(w, r, 1);
  s = a ^ w ^ c;
  k = (a & w) | (c & (a ^ w));
}

// Next state of a word from the horizontal sums of the rows above (u), at
// (m) and below (d), the word itself and its member mask: the nine-cell sum
// modulo 4 (bit0, bit1), births masked to members (self is already a subset
// of the members).
__device__ __forceinline__ uint32_t life_rule_mod4(uint32_t us, uint32_t uk, uint32_t ms, uint32_t mk_, uint32_t ds,
                                                   uint32_t dk, uint32_t self, uint32_t mask) {
  const uint32_t bit0 = us ^ ms ^ ds;
  const uint32_t k0 = (us & ms) | (ds & (us ^ ms));
  const uint32_t bit1 = (uk ^ mk_ ^ dk ^ k0) & mask;
  return (bit0 & bit1) | (~bit0 & ~bit1 & self);
}

// TT: the super-tile side, a compile-time constant so that the column stride
// and the neighbour offsets of a word are immediates.
template <int MODE, int TT>
__global__ void __launch_bounds__(704, 2) ca_fused_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                       int nsteps, int M, Geo g,
                                                       unsigned long long* __restrict__ partials,
                                                       const uint32_t* __restrict__ pin, uint32_t* __restrict__ pout) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ unsigned long long red[32];
  int sx, sy;
  if (!cta_supertile<MODE>(g, sx, sy)) {
    if (partials && threadIdx.x == 0) partials[cta_id()] = 0ull;
    return;
  }
  const int n = g.n;
  constexpr int T = TT;
  constexpr int wlev = ilog2c(TT) - 5;                 // word-tile levels of the super-tile
  constexpr int wside = 1 << wlev;                     // word tiles per super-tile side
  int wtiles = 1, wlw = 1;                             // 3^wlev, 3^ceil(wlev/2)
  for (int i = 0; i < wlev; ++i) wtiles *= 3;
  for (int i = 0; i < (wlev + 1) / 2; ++i) wlw *= 3;
  constexpr int CW = ca_col(TT);                       // words per image column
  constexpr int img = ca_image_words(TT);
  const int ME8 = (M + 7) & ~7;
  uint32_t* tab = reinterpret_cast<uint32_t*>(sm);
  uint32_t* A = tab + tab_words(wtiles);
  uint32_t* B = A + img;
  const int ox = sx * T, oy = sy * T;
  int lwR = 1;  // 3^ceil(R/2)
  for (int i = 0; i < (g.R + 1) / 2; ++i) lwR *= 3;
  // first record of this super-tile, and the record of word tile (tx, ty)
  auto st_index = [&](int x, int y) -> int64_t {
    return MODE == kLambda ? lambda_inverse(x, y, g.R, lwR) : bb_rank(x, y, g.R);
  };
  const int64_t srec = (pin || pout) ? st_index(sx, sy) * wtiles : 0;
  auto tile_record = [&](int tx, int ty) -> int64_t {
    const int lx = tx & (wside - 1), ly = ty & (wside - 1);
    const int local = MODE == kLambda ? lambda_inverse(lx, ly, wlev, wlw) : bb_rank(lx, ly, wlev);
    return st_index(tx >> wlev, ty >> wlev) * wtiles + local;
  };

  // member word tiles of the super-tile
  if (MODE == kLambda) {
    for (int j = threadIdx.x; j < wtiles; j += blockDim.x) {
      int ux, uy;
      lambda_scalar((uint32_t)(j % wlw), (uint32_t)(j / wlw), wlev, ux, uy);
      tab[j] = (uint32_t)ux | ((uint32_t)uy << 16);
    }
  } else {
    for (int j = threadIdx.x; j < wside * wside; j += blockDim.x) {
      const int ux = j & (wside - 1), uy = j >> wlev;
      if ((ux & uy) == 0) {
        int rank = 0;
        for (int q = 0; q < j; ++q) rank += ((q & (wside - 1)) & (q >> wlev)) == 0;
        tab[rank] = (uint32_t)ux | ((uint32_t)uy << 16);
      }
    }
  }
  for (int i = threadIdx.x; i < 2 * img / 4; i += blockDim.x)
    reinterpret_cast<uint4*>(A)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  // this lane's four rows of its task: image offset of the first row, the
  // rows' member bits and words (the lane is their only writer)
  const int sub = threadIdx.x & (kCaLanes - 1), j = threadIdx.x / kCaLanes;
  const int ntasks = ca_tasks(wtiles);
  int off = -1, c = 0, y = 0;
  bool last = false;  // the task's last lane with rows: the row below comes from the image
  uint32_t mk[kCaRows], w[kCaRows];
#pragma unroll
  for (int r = 0; r < kCaRows; ++r) mk[r] = w[r] = 0u;
  if (j < ntasks) {
    int y0, rows;
    ca_task(j, wtiles, tab, T, ME8, c, y0, rows);
    if (kCaRows * sub < rows) {
      y = y0 + kCaRows * sub;
      last = kCaRows * (sub + 1) >= rows;
      const int gx0 = ox + 32 * c, gy = oy + y;
      off = (c + 2) * CW + y + kCaRow0;
      if ((unsigned)gx0 < (unsigned)n) {
#pragma unroll
        for (int r = 0; r < kCaRows; ++r) mk[r] = chunk_members<32>(gx0, gy + r, n);
      }
      if (mk[0] | mk[1] | mk[2] | mk[3]) {
        if (pin) {  // the four rows lie in one member word tile: 16 bytes of its record
          const int64_t rec = j < wtiles ? srec + j : tile_record(gx0 >> 5, gy >> 5);
          const uint4 v = __ldg(reinterpret_cast<const uint4*>(pin + rec * 32 + (gy & 31)));
          w[0] = v.x;
          w[1] = v.y;
          w[2] = v.z;
          w[3] = v.w;
        } else {
#pragma unroll
          for (int r = 0; r < kCaRows; ++r) {
            if (!mk[r]) continue;
            const uint4* q = reinterpret_cast<const uint4*>(in + (size_t)(gy + r) * n + gx0);
            w[r] = pack32(__ldg(q), __ldg(q + 1));
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kCaRows; ++r) w[r] &= mk[r];
      *reinterpret_cast<uint4*>(A + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  __syncthreads();

  // unrolled: the image pointers of both parities are fixed; every lane takes
  // part in the shuffles (lanes without rows carry zeros)
  const bool first = sub == 0;
#pragma unroll 2
  for (int t = 0; t < nsteps; ++t) {
    uint32_t s[kCaRows + 2], q[kCaRows + 2];  // horizontal sums of rows y-1 .. y+4
    const uint32_t* p = A + (off >= 0 ? off : kCaRow0);
    if (off >= 0) {
      const uint4 l = *reinterpret_cast<const uint4*>(p - CW), r = *reinterpret_cast<const uint4*>(p + CW);
      row_sum3(l.x, w[0], r.x, s[1], q[1]);
      row_sum3(l.y, w[1], r.y, s[2], q[2]);
      row_sum3(l.z, w[2], r.z, s[3], q[3]);
      row_sum3(l.w, w[3], r.w, s[4], q[4]);
    } else {
#pragma unroll
      for (int r = 1; r <= kCaRows; ++r) s[r] = q[r] = 0u;
    }
    // the row above is the previous lane's last, the row below the next lane's first
    s[0] = __shfl_up_sync(0xffffffffu, s[kCaRows], 1, kCaLanes);
    q[0] = __shfl_up_sync(0xffffffffu, q[kCaRows], 1, kCaLanes);
    s[kCaRows + 1] = __shfl_down_sync(0xffffffffu, s[1], 1, kCaLanes);
    q[kCaRows + 1] = __shfl_down_sync(0xffffffffu, q[1], 1, kCaLanes);
    if (off >= 0) {
      if (first) {  // row y - 1: the last word of the 16-byte groups above, in the three columns
        const uint32_t lu = reinterpret_cast<const uint4*>(p - CW)[-1].w, cu = reinterpret_cast<const uint4*>(p)[-1].w,
                       ru = reinterpret_cast<const uint4*>(p + CW)[-1].w;
        row_sum3(lu, cu, ru, s[0], q[0]);
      }
      if (last) {  // row y + 4: the first word of the 16-byte groups below
        const uint32_t ld = reinterpret_cast<const uint4*>(p - CW)[1].x, cd = reinterpret_cast<const uint4*>(p)[1].x,
                       rd = reinterpret_cast<const uint4*>(p + CW)[1].x;
        row_sum3(ld, cd, rd, s[kCaRows + 1], q[kCaRows + 1]);
      }
#pragma unroll
      for (int r = 0; r < kCaRows; ++r)
        w[r] = life_rule_mod4(s[r], q[r], s[r + 1], q[r + 1], s[r + 2], q[r + 2], w[r], mk[r]);
      *reinterpret_cast<uint4*>(B + off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    uint32_t* tmp = A;
    A = B;
    B = tmp;
  }

  // write back the word tiles (whole 32-byte row segments); count the alive
  unsigned alive = 0;
  if (off >= 0 && j < wtiles) {
#pragma unroll
    for (int r = 0; r < kCaRows; ++r) alive += __popc(w[r]);
    if (pout) {  // record of word tile j, rows y .. y + 3 mod 32
      *reinterpret_cast<uint4*>(pout + (srec + j) * 32 + (y & 31)) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
#pragma unroll
      for (int r = 0; r < kCaRows; ++r) {
        const uint32_t v = w[r];
        uint4 v0, v1;
        v0.x = spread4(v);
        v0.y = spread4(v >> 4);
        v0.z = spread4(v >> 8);
        v0.w = spread4(v >> 12);
        v1.x = spread4(v >> 16);
        v1.y = spread4(v >> 20);
        v1.z = spread4(v >> 24);
        v1.w = spread4(v >> 28);
        uint4* q = reinterpret_cast<uint4*>(out + (size_t)(oy + y + r) * n + ox + 32 * c);
        q[0] = v0;
        q[1] = v1;
      }
    }
  }
  if (partials) {  // alive members of the result, per CTA (uniform branch)
    const unsigned long long s = block_sum<unsigned long long>(alive, red);
    if (threadIdx.x == 0) partials[cta_id()] = s;
  }
}

template <int MODE>
cudaError_t go(const Launch& L, const uint8_t* in, uint8_t* out, int nsteps, int margin,
               unsigned long long* partials, const uint32_t* pin, uint32_t* pout, cudaStream_t s) {
  auto run = [&](auto* k) -> cudaError_t {
    cudaError_t e = allow_smem((const void*)k, L.smem);
    if (e != cudaSuccess) return e;
    k<<<L.grid, L.threads, L.smem, s>>>(in, out, nsteps, margin, L.geo, partials, pin, pout);
    return cudaGetLastError();
  };
  switch (L.geo.T) {
    case 32: return run(ca_fused_kernel<MODE, 32>);
    case 64: return run(ca_fused_kernel<MODE, 64>);
    case 128: return run(ca_fused_kernel<MODE, 128>);
    case 256: return run(ca_fused_kernel<MODE, 256>);
    case 512: return run(ca_fused_kernel<MODE, 512>);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int ca_fused_smem_bytes(const Geo& g, int margin) {
  (void)margin;  // the image covers the largest margin
  const int wlev = ilog2c(g.T) - 5;
  int wtiles = 1;
  for (int i = 0; i < wlev; ++i) wtiles *= 3;
  return tab_words(wtiles) * 4 + 2 * ca_image_words(g.T) * 4;
}

// Threads of a fused automaton launch: four lanes per task, in whole warps;
// 0 if the super-tile does not fit the kernel.
int ca_fused_threads(const Geo& g, int margin) {
  if (g.T < 32 || g.T > 512 || margin < 1 || margin > 31 || 2 * margin > g.T) return 0;
  int wtiles = 1;
  for (int i = 0; i < ilog2c(g.T) - 5; ++i) wtiles *= 3;
  return (kCaLanes * ca_tasks(wtiles) + 31) / 32 * 32;
}

cudaError_t launch_ca_fused(int mode, const Launch& L, const uint8_t* in, uint8_t* out, int nsteps, int margin,
                            cudaStream_t s, unsigned long long* partials, const uint32_t* pin, uint32_t* pout) {
  if (nsteps < 0 || nsteps > margin || ca_fused_threads(L.geo, margin) != L.threads || (!in && !pin) ||
      (!out && !pout))
    return cudaErrorInvalidValue;
  return mode == kLambda ? go<kLambda>(L, in, out, nsteps, margin, partials, pin, pout, s)
                         : go<kBB>(L, in, out, nsteps, margin, partials, pin, pout, s);
}

int64_t ca_records(int k) {
  int64_t r = 1;
  for (int i = 5; i < k; ++i) r *= 3;
  return k >= 5 ? r : 0;
}

}  // namespace fractal
