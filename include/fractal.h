/*
 * fractal.h -- C ABI of the GB300 (sm_103a) block-space-map library for the
 * embedded Sierpinski gasket.
 *
 * Method: "Efficient GPU Thread Mapping on Embedded 2D Fractals" (Navarro,
 * Quezada, Hitschfeld, Vega, Bustos).  A compact grid of 3^{r_b} blocks
 * (Lemma 2) is sent onto the member tiles of a gasket of level k embedded in
 * an n x n array (n = 2^k) by the block-space map lambda(omega) (Theorem 1,
 * Sec. 6.1); each tile of rho x rho cells is processed with the bounding
 * sub-box approach (Sec. 5.3).  The bounding-box (BB) launch, which maps
 * blocks by the identity and discards non-member ones (Sec. 1, Theorem 2), is
 * built beside it as the plain method.
 *
 * Geometry and layout (all entry points):
 *   - cell (x, y) is a gasket member iff 0 <= x, y < n and (x & y) == 0;
 *   - every data buffer is a caller-owned DEVICE array of n*n elements,
 *     row-major (element index y*n + x), 16-byte aligned;
 *   - kernels read only member cells: the contents of non-member cells of an
 *     input are ignored;
 *   - kernels that write a field write every cell of every member tile
 *     (value at members, 0 at the non-member cells of that tile) and leave
 *     all cells outside member tiles untouched;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All calls are asynchronous on that stream except
 *     fractal_reduce, which synchronises it.
 *
 * Status: every entry point returns FRACTAL_OK (0) or a negative code; the
 * caller's buffers are not touched when a call fails validation.  No call
 * aborts the process.
 */
#ifndef FRACTAL_H_
#define FRACTAL_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FRACTAL_OK 0
#define FRACTAL_EINVAL (-1)  /* bad argument: level, rho, mode, dtype, pointer, alignment */
#define FRACTAL_ENOMEM (-2)  /* host or device allocation failed */
#define FRACTAL_ECUDA (-3)   /* a CUDA runtime call or kernel launch failed */
#define FRACTAL_ETOOBIG (-4) /* fractal_reduce_noalloc: the launch needs more partials than its fixed array */

/* Launch modes. */
#define FRACTAL_LAMBDA 0     /* compact grid + lambda(omega) (Theorem 1) */
#define FRACTAL_BB 1         /* bounding-box grid, identity map, discard non-members */

/* Step-kernel schedules (fractal_plan_set_schedule). */
#define FRACTAL_SCHED_AUTO 0   /* TMA staging where it applies, else vector-load staging */
#define FRACTAL_SCHED_STAGED 1 /* vector loads into a shared-memory image of the super-tile */
#define FRACTAL_SCHED_TMA 2    /* one cp.async.bulk.tensor box per member tile (rows >= 16 B) */

/* Element types. */
#define FRACTAL_U8 0         /* uint8 automaton states (nonzero = alive) */
#define FRACTAL_F32 1        /* float32 field */
#define FRACTAL_DF 2         /* double-float field: (hi, lo) float pairs, 2 floats per cell (gradient path) */

#define FRACTAL_MAX_LEVEL 16

typedef struct fractal_plan_s* fractal_plan_t;

/* Read-only description of a plan (filled by fractal_plan_get_info). */
typedef struct fractal_plan_info {
  int32_t k;             /* gasket level; n = 2^k */
  int32_t rho;           /* tile side (block size of the map) */
  int32_t mode;          /* FRACTAL_LAMBDA or FRACTAL_BB */
  int32_t r_b;           /* block-space level k - log2(rho) (Theorem 1) */
  int64_t n;             /* embedding side */
  int64_t n_b;           /* blocks per side, 2^r_b */
  int32_t grid_w;        /* packed grid of the map at block level: 3^ceil(r_b/2) (Lemma 2) */
  int32_t grid_h;        /*                                      3^floor(r_b/2) */
  int64_t member_tiles;  /* 3^r_b */
  int64_t members;       /* 3^k cells */
  int32_t cta_levels[2]; /* per dtype: tile levels unrolled inside one CTA (Sec. 5.1) */
  int64_t ctas[2];       /* per dtype: CTAs one launch of this plan starts */
  int32_t threads[2];    /* per dtype: threads per CTA */
  int32_t smem_bytes[2]; /* per dtype: dynamic shared memory per CTA of a step kernel */
  int32_t tma[2];        /* per dtype: 1 if the step kernel stages tiles with TMA */
  int32_t sched;         /* FRACTAL_SCHED_* */
  int32_t steps_per_launch[2]; /* per dtype: steps one launch advances (temporal fusion) */
} fractal_plan_info;

/* Human-readable text of a status code (static storage). */
const char* fractal_strerror(int status);

/* Text of the last CUDA error seen by this thread inside the library ("" if none). */
const char* fractal_last_cuda_error(void);

/*
 * fractal_map -- build a plan for level k (0 <= k <= 16), tile side rho
 * (power of two, 1 <= rho <= min(32, 2^k)) and a launch mode.
 * Theorem 1: r_b = k - log2(rho); the lambda grid is the Lemma-2 orthotope of
 * 3^ceil(r_b/2) x 3^floor(r_b/2) blocks, the BB grid is n_b x n_b.
 * The plan belongs to the CUDA device current at this call, owns a small
 * device scratch area for fractal_reduce and a pinned host word; it is freed
 * by fractal_plan_destroy.  One plan may be used from one host thread at a
 * time.  Errors: FRACTAL_EINVAL (bad k, rho, mode or NULL out),
 * FRACTAL_ENOMEM, FRACTAL_ECUDA.
 */
int fractal_map(int k, int rho, int mode, fractal_plan_t* plan);

/* Free a plan (NULL is accepted).  Waits for nothing: the caller must make
 * sure no work using the plan is still queued. */
int fractal_plan_destroy(fractal_plan_t plan);

int fractal_plan_get_info(fractal_plan_t plan, fractal_plan_info* info);

/*
 * Tile levels unrolled inside one CTA for dtype (Sec. 5.1, "further
 * unrolling"): a CTA handles the 3^levels member tiles (lambda) or 4^levels
 * tile slots (BB) of one super-tile of side rho * 2^levels; the grid maps
 * super-tiles (level r_b - levels).  0 <= levels <= min(r_b, 5), and the
 * super-tile must fit in shared memory.  The single write runs rho-tile
 * kernels at these levels.  By default the float32 reduce runs its own kernel
 * (one 8 x 8 block of the gasket per thread, rho >= 4, k >= 3); once this is
 * called for FRACTAL_F32 it runs the rho-tile kernel at these levels too
 * (levels 0: one tile per CTA, the paper's block-per-tile setting).  Errors: FRACTAL_EINVAL, FRACTAL_ENOMEM
 * (reduce scratch could not grow).
 */
int fractal_plan_set_cta_levels(fractal_plan_t plan, int dtype, int levels);

/*
 * Choose how step kernels stage tiles: FRACTAL_SCHED_AUTO (default),
 * FRACTAL_SCHED_STAGED or FRACTAL_SCHED_TMA.  Results are identical; only
 * the data movement differs (TMA needs tile rows of at least 16 bytes: float32
 * rho >= 4, uint8 rho >= 16; other plans keep the staged kernels).  Errors:
 * FRACTAL_EINVAL (unknown value, or TMA requested where it never applies).
 */
int fractal_plan_set_schedule(fractal_plan_t plan, int sched);

/*
 * fractal_plan_autotune -- time the plan's step kernel for dtype under every
 * staging (TMA where it applies, vector loads), every valid number of tile
 * levels per CTA and 1 step per launch or temporal fusion (float32: 16, 25,
 * 50 or 100 steps per launch; uint8: 8, 16, 25 or 31), and keep the fastest
 * per step.  Each candidate runs `reps` timed units dev_in -> dev_scratch
 * (after two untimed ones) on `stream`, which is synchronised: one step, or
 * with fusion the launches of a 100-step call (200 for 100 per launch) as
 * the step driver runs them, records between.  dev_in is only read;
 * dev_scratch is overwritten.  Both are n*n arrays of dtype, 16-byte aligned.  *best_us
 * (nullable) receives the best mean step time in microseconds.  The tuned
 * choice applies to this plan only (results never depend on it).  Errors:
 * FRACTAL_EINVAL, FRACTAL_ENOMEM, FRACTAL_ECUDA.
 */
int fractal_plan_autotune(fractal_plan_t plan, int dtype, const void* dev_in, void* dev_scratch, int reps,
                          float* best_us, void* stream);

/*
 * fractal_plan_set_steps_per_launch -- temporal fusion: each launch advances
 * every member tile by up to `spl` steps, staging the tile once and the few
 * cells around the super-tile's three contacts with the rest of the gasket
 * (margin boxes of width >= spl).  Results equal those of single-step
 * launches (bit for bit for the automaton, up to FP32 rounding order for the
 * diffusion); the buffer holding the result after `steps` steps is unchanged
 * (dev_a for even, dev_b for odd).  spl = 1 turns fusion off.
 * FRACTAL_F32 (diffusion, one 8 x 8 block of the gasket per thread): spl <=
 * 128, rho >= 4, a super-tile side of at least 16 cells and twice the margin
 * (the smallest power of two >= max(spl, 8)); the kernel takes the largest
 * such super-tile it can hold, whatever fractal_plan_set_cta_levels chose.
 * FRACTAL_U8 (automaton, on a bit image of 32-cell words): spl <= 31, a
 * super-tile side of 32 to 512 cells and at least 2*spl (k >= 6).  The
 * super-tile may be smaller than the plan's step kernels use.
 * A call of more than one launch keeps the state between its launches in
 * compact records the plan allocates here, two buffers of 3^(k-3) records of
 * 112 bytes (float32: the 27 members of a member 8 x 8 block) or of 3^(k-5)
 * records of 128 bytes (uint8: the 32 words of a member 32 x 32 word tile),
 * freed with the plan: only the first launch reads dev_a and only the last
 * writes the result buffer; the other caller buffer is then not written.
 * Margin-box blocks farther than spl cells from the super-tile are not staged
 * (fractal_fused_box_blocks).
 * For float32 the call also writes, once, the setup of every thread of the
 * fused launch (its block, port owners and neighbours: 16 bytes a thread,
 * 34 MB at k = 16, rho = 8, spl = 50), which every fused launch then reads instead of
 * computing it; it waits for the device first (no call of this plan may be
 * in flight) and for that launch after.
 * Errors: FRACTAL_EINVAL (dtype, spl, or no fused kernel for this plan),
 * FRACTAL_ENOMEM, FRACTAL_ECUDA.
 */
int fractal_plan_set_steps_per_launch(fractal_plan_t plan, int dtype, int spl);

/*
 * fractal_fused_box_blocks -- margin-box blocks a float32 fused launch stages
 * per super-tile (host only; no device is touched).  A launch serving up to
 * `reach` steps (reach = spl) stages, besides the member 8 x 8 blocks of its
 * super-tile of side `supertile` cells, the member blocks of its margin boxes
 * (width `margin` = the smallest power of two >= max(spl, 8)) whose nearest
 * cell lies within `reach` cells (Manhattan distance, the reach of `reach`
 * 4-neighbour steps) of the super-tile: farther blocks cannot influence the
 * super-tile within the launch.  Returns the most such blocks any member
 * super-tile has (the launch gives each a thread slot), or FRACTAL_EINVAL
 * (supertile not a power of two in [16, 256], margin not 8 times a power of
 * two up to 128 or above supertile / 2, reach outside [1, margin]).
 */
int fractal_fused_box_blocks(int supertile, int margin, int reach);

/*
 * Device status word of the plan's TMA kernels: 0, or the first error a CTA
 * recorded (1: a tile copy did not complete within the wait limit; 2: the
 * drain after it also timed out).  The step kernels never trap or spin
 * forever; they record a code here and return.  Synchronous copy.
 */
int fractal_plan_device_status(fractal_plan_t plan, int* code);

/*
 * Record form.  Once steps per launch > 1 is set for a dtype, the plan's
 * fused launches keep the state between them in compact records, and a
 * caller may hold the state in that form too: float32, one 112-byte record
 * per member 8 x 8 block (its 27 members and a pad; 3^(k-3) records);
 * uint8, one 128-byte bit record per member 32 x 32 word tile (32 words of
 * 32 cells, 1 bit = alive; 3^(k-5) records).  The records are ordered by the
 * configuration's super-tiles (lambda or BB rank) and stored as the kernels
 * read them, so a record-form state belongs to the plan's configuration
 * (side, launch mode) for that dtype: change the configuration and convert
 * again.  Moving a state in record form (179 MB at k = 16 float32, 22.7 MB
 * uint8) replaces moving the embedded arrays (16 GiB, 4 GiB) and needs no
 * packing pass.  This library's compact form for the paper's closing remark
 * on storing only the fractal; no counterpart in the paper otherwise.
 *
 * fractal_plan_records_bytes -- bytes of one state in record form.  Errors:
 * FRACTAL_EINVAL (NULL, no fused configuration for dtype).
 *
 * fractal_records_from_array / fractal_records_to_array -- convert between
 * the embedded n*n array (16-byte aligned; read at members / written as the
 * step calls write it) and the record form (device memory, 16-byte
 * aligned); one launch of the fused kernel with no steps.  Asynchronous.
 * Errors: FRACTAL_EINVAL, FRACTAL_ECUDA.
 *
 * fractal_step_diffusion_records -- as fractal_step_diffusion_sums (sum
 * every `every` steps into dev_sums, nullable; steps >= 1 a multiple of
 * every) from records rec_in to records rec_out (distinct; rec_in is not
 * written), launches of up to steps-per-launch steps.
 * fractal_step_ca_records -- `steps` (>= 1) automaton steps from bit
 * records rec_in to rec_out, the alive count of the result into dev_count
 * (nullable).  Asynchronous.  Errors: FRACTAL_EINVAL, FRACTAL_ENOMEM (the
 * plan's records could not be allocated), FRACTAL_ECUDA.
 */
int fractal_plan_records_bytes(fractal_plan_t plan, int dtype, int64_t* bytes);
int fractal_records_from_array(fractal_plan_t plan, int dtype, const void* dev_embedded, void* dev_records,
                               void* stream);
int fractal_records_to_array(fractal_plan_t plan, int dtype, const void* dev_records, void* dev_embedded,
                             void* stream);
int fractal_step_diffusion_records(fractal_plan_t plan, const float* rec_in, float* rec_out, float a, int steps,
                                   int every, double* dev_sums, void* stream);
int fractal_step_ca_records(fractal_plan_t plan, const void* rec_in, void* rec_out, int steps, double* dev_count,
                            void* stream);

/*
 * Failure-path hooks for tests.  The paper has no counterpart: they exist so
 * that the library's error handling can be exercised without faulting a GPU.
 *
 * fractal_plan_selftest_wait -- launches one CTA that arms an mbarrier which
 * nothing completes (no copy is issued) and waits on it with the bounded wait
 * of the TMA step kernels, at most `spins` polls (1 .. 2^22); the wait runs
 * out, code 1 is recorded in the plan's device status word (first error
 * wins) and the kernel returns, leaving the context usable.  Synchronises
 * `stream`.  Errors: FRACTAL_EINVAL, FRACTAL_ECUDA.
 *
 * fractal_debug_fail_allocs -- process-wide: after `after` more successful
 * device allocations by the library, the next one fails as if the device
 * were out of memory (the call making it returns FRACTAL_ENOMEM, leaving the
 * caller's buffers untouched and an existing plan in its previous
 * configuration); then injection is off again.  after < 0: off.  Never
 * fails.
 */
int fractal_plan_selftest_wait(fractal_plan_t plan, unsigned spins, void* stream);
int fractal_debug_fail_allocs(int after);

/*
 * fractal_map_blocks -- export the block-space map of the plan (Theorem 1,
 * Sec. 6.1): for omega in row-major order of the grid_w x grid_h packed grid,
 * dev_xy[2*(wy*grid_w + wx) + {0,1}] = (block_x, block_y) in the
 * (x & y) == 0 orientation.  dev_xy: device array of 2*3^r_b int32, written
 * entirely.  Computed by the same warp-level lambda the step kernels use.
 * Errors: FRACTAL_EINVAL (NULL), FRACTAL_ECUDA.
 */
int fractal_map_blocks(fractal_plan_t plan, int32_t* dev_xy, void* stream);

/*
 * fractal_map_blocks_method -- the same table by one of three forms of
 * lambda: FRACTAL_MAP_BALLOT (one warp per omega, lane mu-1 computes level
 * mu, a ballot sums the Delta terms; what the step kernels use),
 * FRACTAL_MAP_SCALAR (one thread per omega), FRACTAL_MAP_MMA (the tensor-core
 * encoding of Sec. 6.3: 16 omegas per warp, their level bits as a 16 x 16
 * bf16 matrix times the powers of two, FP32 accumulate; exact, since the
 * entries are 0, 1 and powers of two and the sums stay below 2^24).  All
 * three write the same table; the method only changes the speed.  dev_xy
 * 8-byte aligned.  Errors: FRACTAL_EINVAL, FRACTAL_ECUDA.
 */
#define FRACTAL_MAP_BALLOT 0
#define FRACTAL_MAP_SCALAR 1
#define FRACTAL_MAP_MMA 2
int fractal_map_blocks_method(fractal_plan_t plan, int32_t* dev_xy, int method, void* stream);

/*
 * fractal_map_write -- the single-write test of Sec. 6.2 (SW): write `value`
 * (cast to dtype; uint8 takes (uint8_t)value) at every member cell of the
 * n x n device array dev_buf, 0 at the non-member cells of member tiles;
 * nothing is read.  Errors: FRACTAL_EINVAL (NULL, misaligned, dtype),
 * FRACTAL_ECUDA.
 */
int fractal_map_write(fractal_plan_t plan, void* dev_buf, int dtype, double value, void* stream);

/*
 * fractal_step_ca -- `steps` synchronous steps of the fractal Life-like
 * automaton of Sec. 6.2 (test CA), rule B3/S23 on the Moore neighbourhood,
 * counting only member neighbours; non-members are never born.  States are
 * uint8 (nonzero = alive; outputs are 0/1).  dev_a holds the start state;
 * the steps alternate dev_a -> dev_b -> dev_a ...: after the call the state
 * is in dev_a when `steps` is even and in dev_b when it is odd.  Both buffers
 * are n*n bytes, 16-byte aligned, distinct.  steps == 0 does nothing.
 * Only member tiles are written (their non-member cells as 0); with temporal
 * fusion on (fractal_plan_set_steps_per_launch), whole 32-cell row segments
 * of the member 32 x 32 blocks, non-member cells again as 0.
 * Errors: FRACTAL_EINVAL (NULL, equal or misaligned buffers, steps < 0),
 * FRACTAL_ECUDA.
 */
int fractal_step_ca(fractal_plan_t plan, uint8_t* dev_a, uint8_t* dev_b, int steps, void* stream);

/*
 * fractal_step_ca_count -- fractal_step_ca followed by the global measure of
 * Sec. 6.2 (RD) on the result: *dev_count (a device double) receives the
 * number of alive members after the steps.  With temporal fusion the count is
 * taken by the last launch from the words it writes (no second pass over the
 * array); otherwise a reduce follows.  steps == 0 counts dev_a.  Asynchronous.
 * Errors: as fractal_step_ca, FRACTAL_EINVAL for a NULL dev_count.
 */
int fractal_step_ca_count(fractal_plan_t plan, uint8_t* dev_a, uint8_t* dev_b, int steps, double* dev_count,
                          void* stream);

/*
 * fractal_step_diffusion -- `steps` explicit FDM heat-diffusion steps on the
 * gasket (the FDM time-step pattern of Sec. 1), FP32:
 *   u'_c = u_c + a * sum_{nb in N4(c), nb member} (u_nb - u_c),
 * zero flux towards non-members and the array edge.  a = alpha*dt; the
 * scheme is stable and positivity-preserving for 0 <= a < 1/3 (members have
 * at most three 4-neighbours).  Buffers and ping-pong as in fractal_step_ca
 * (n*n floats each).  Errors: FRACTAL_EINVAL (NULL, equal or misaligned
 * buffers, steps < 0, a not finite), FRACTAL_ECUDA.
 */
int fractal_step_diffusion(fractal_plan_t plan, float* dev_a, float* dev_b, float a, int steps,
                           void* stream);

/*
 * fractal_step_diffusion_sum -- fractal_step_diffusion followed by the global
 * sum of Sec. 6.2 (RD) on the result: *dev_sum (a device double) receives the
 * sum over the members after the steps (FP32 within an 8-cell row of a block,
 * FP64 above, fixed order).  With temporal fusion the sum is taken by the
 * last launch from the values it writes; otherwise a reduce follows.  steps
 * == 0 sums dev_a.  Asynchronous.  Errors: as fractal_step_diffusion,
 * FRACTAL_EINVAL for a NULL dev_sum.
 */
int fractal_step_diffusion_sum(fractal_plan_t plan, float* dev_a, float* dev_b, float a, int steps, double* dev_sum,
                               void* stream);

/*
 * fractal_step_diffusion_sums -- `steps` steps as fractal_step_diffusion (the
 * result in dev_a for even steps, dev_b for odd) with the global sum of the
 * state after every `every` steps: dev_sums[j] (device doubles, steps / every
 * of them) receives the member sum after (j + 1) * every steps, as
 * fractal_step_diffusion_sum computes it.  steps must be a multiple of every.
 * With temporal fusion the whole call is one sequence of fused launches: the
 * state stays in the plan's records across the sums (the launch that ends a
 * segment takes its sum), and only the last launch writes the result buffer;
 * the intermediate states are not written to dev_a / dev_b.  steps == 0
 * writes nothing.  Asynchronous.  Errors: as fractal_step_diffusion,
 * FRACTAL_EINVAL for a NULL dev_sums, every < 1 or steps not a multiple of
 * every.
 */
int fractal_step_diffusion_sums(fractal_plan_t plan, float* dev_a, float* dev_b, float a, int steps, int every,
                                double* dev_sums, void* stream);

/*
 * fractal_reduce -- the reduction test of Sec. 6.2 (RD): the sum over all
 * member cells of dev_buf (uint8: number of alive members, exact; float32:
 * per-thread FP32 partials of at most 16 cells, summed in FP64 in a fixed
 * order, so the result is deterministic).  Writes the result to *host_out
 * and synchronises `stream`.  Errors: FRACTAL_EINVAL (NULL, misaligned,
 * dtype), FRACTAL_ECUDA.
 */
int fractal_reduce(fractal_plan_t plan, const void* dev_buf, int dtype, double* host_out,
                   void* stream);

/*
 * fractal_reduce_async -- as fractal_reduce, but the result is written to the
 * device double *dev_out and nothing is synchronised (usable inside a step
 * loop or a CUDA graph).  Uses the plan's scratch: calls on one plan must be
 * ordered on one stream.  Errors: as fractal_reduce.
 */
int fractal_reduce_async(fractal_plan_t plan, const void* dev_buf, int dtype, double* dev_out,
                         void* stream);

/*
 * fractal_reduce_noalloc -- the sum over the members (as fractal_reduce_async)
 * for callers that cannot allocate: it takes no plan and calls no cudaMalloc,
 * cudaFree or other allocating routine.  It runs the kernels of a default
 * lambda plan, fractal_map(k, rho, FRACTAL_LAMBDA): float32 at rho >= 4 the
 * reduce over 8 x 8 blocks, otherwise the rho-tile reduce at the plan's
 * default tile levels per CTA (more levels only where those partials would
 * not fit the array), so its sum equals that plan's; uint8 counts are exact
 * in every case.  Such
 * callers are, for example, code that runs while another allocator (a
 * framework's caching allocator, a fixed memory pool) owns the device memory,
 * and latency-bound loops that must not pay for, or synchronise on, an
 * allocation.  There is no counterpart in the paper.
 *
 * Its scratch (one partial sum per CTA) is a fixed device array of
 * FRACTAL_NOALLOC_MAX_PARTIALS doubles (512 KiB) built into the library;
 * every GPU that loads the library holds it until the process exits.  Levels
 * whose launch would need more partials are rejected with FRACTAL_ETOOBIG
 * (k = 16 with rho = 1 is the only such case).  The array is shared by all
 * calls: calls whose work overlaps on the GPU (different streams without
 * ordering, or several host threads) race on it, so order them on one
 * stream.  The first call on a device looks up the array's device address
 * (once per device, with that device current) and keeps it for the life of
 * the process; make that first call before any stream capture.  A device
 * reset (cudaDeviceReset) releases the array with the context: do not call
 * this entry point on that device again in the same process.  k, rho and
 * dtype as in fractal_map / fractal_reduce; dev_buf: n*n array, 16-byte
 * aligned, and dev_out: a double receiving the sum, both addressable by the
 * current device (device memory of that device, managed, or mapped pinned
 * host memory).  Asynchronous on `stream`.  Errors: FRACTAL_EINVAL,
 * FRACTAL_ETOOBIG, FRACTAL_ECUDA.
 */
#define FRACTAL_NOALLOC_MAX_PARTIALS 65536
int fractal_reduce_noalloc(int k, int rho, const void* dev_buf, int dtype, double* dev_out, void* stream);

/*
 * fractal_pack / fractal_unpack -- compact storage through the block-space
 * map (the compact lambda / lambda^-1 storage the paper leaves for later
 * work): the member tiles of the n x n array dev_embedded, one after another
 * in lambda order -- packed tile j is the tile lambda(omega_j), omega_j =
 * (j mod grid_w, j div grid_w) (Theorem 1), rows of rho elements in order --
 * into dev_packed (member_tiles * rho^2 elements of dtype), and back.  Pack
 * reads only member tiles; unpack writes whole member tiles and nothing else.
 * The order is lambda's whatever the plan's launch mode.  Both buffers
 * 16-byte aligned and distinct; each is device memory of the plan's device
 * or pinned host memory mapped into its address space at the same address
 * (cudaHostAlloc / cudaHostRegister under unified addressing): with a host
 * packed buffer the kernel itself moves the packed field over the host link,
 * in place of a separate copy.  Pageable host memory is rejected (checked on
 * the host with cudaPointerGetAttributes, before any launch).  Asynchronous.
 * Not in the paper's measurements: the form in which a field crosses between
 * host and device.
 * Errors: FRACTAL_EINVAL, FRACTAL_ECUDA.
 */
int fractal_pack(fractal_plan_t plan, const void* dev_embedded, int dtype, void* dev_packed, void* stream);
int fractal_unpack(fractal_plan_t plan, const void* dev_packed, int dtype, void* dev_embedded, void* stream);

/*
 * fractal_set_l2_fetch_granularity -- set the L2 fetch granularity hint of
 * the CURRENT CUDA context (cudaLimitMaxL2FetchGranularity) to 32, 64 or 128
 * bytes.  Not part of the paper: a GB300 memory-system knob.  The tiles of a
 * gasket touch scattered 32-byte row segments (one sector: 32 uint8 cells or
 * 8 float32 cells); with a coarser fetch granularity every DRAM read brings
 * neighbouring sectors that hold no member tile.  32 makes reads exact.  The
 * setting is a hint, lasts until the context is destroyed or the limit is set
 * again, and applies to every kernel of the context (the caller's too), so the
 * library never changes it on its own.  Errors: FRACTAL_EINVAL (other sizes),
 * FRACTAL_ECUDA.
 */
int fractal_set_l2_fetch_granularity(int bytes);

/* Current value of that hint for the current context, in bytes. */
int fractal_get_l2_fetch_granularity(int* bytes);

/* ------------------------------------------------------------------------
 * Differentiation: diffusion with a per-cell conductivity and its adjoint.
 *
 * Not in the paper (which names the FDM time step, Sec. 1): the step of
 * fractal_step_diffusion with edge conductances g_{c,nb} = (kappa_c +
 * kappa_nb) / 2,
 *   u'_c = u_c + a * sum_{nb in N4(c), nb member} g_{c,nb} (u_nb - u_c),
 * i.e. u_{t+1} = A u_t with A symmetric (heat is conserved; stable for
 * a * 3 * max kappa < 1), and the reverse step that carries p_{t+1} =
 * dJ/du_{t+1} of a loss J back one step:
 *   p_t = A^T p_{t+1} = A p_{t+1},
 *   dJ/dkappa_c += (a / 2) sum_{nb} (u_t,nb - u_t,c) (p_{t+1},c - p_{t+1},nb).
 * Both use the plan's level k (k >= 3) and launch mode; they run one thread
 * per member 8 x 8 block (lambda map at the block level, Theorem 1), one step
 * per launch, and write whole member 8 x 8 blocks (0 at non-members).  All
 * arrays are n*n float32 device arrays, 16-byte aligned.
 * ------------------------------------------------------------------------ */

/*
 * fractal_step_diffusion_kappa -- `steps` steps with conductivity dev_kappa
 * (read only), ping-pong dev_a -> dev_b -> dev_a ... as fractal_step_diffusion
 * (result in dev_a for even `steps`, dev_b for odd).  Errors: FRACTAL_EINVAL
 * (NULL, equal or misaligned buffers, k < 3, steps < 0, a not finite),
 * FRACTAL_ECUDA.
 */
int fractal_step_diffusion_kappa(fractal_plan_t plan, float* dev_a, float* dev_b, const float* dev_kappa, float a,
                                 int steps, void* stream);

/*
 * fractal_step_diffusion_kappa_f64 -- the same with the state in doubles
 * (dev_a, dev_b: n*n double arrays; dev_kappa still float).  An FP32
 * trajectory rounds the state every step; through differences of neighbour
 * values those roundings alone move the gradients of a 200-step run by a few
 * 1e-4 of their scale, so gradient work that must stay within 1e-4 of an
 * FP64 reference keeps the state in doubles.  Errors as above.
 */
int fractal_step_diffusion_kappa_f64(fractal_plan_t plan, double* dev_a, double* dev_b, const float* dev_kappa,
                                     double a, int steps, void* stream);

/*
 * fractal_adjoint_diffusion_step -- one reverse step: dev_p_out = A dev_p_in
 * (A from dev_kappa and a) and dev_gkappa += the step's contribution to
 * dJ/dkappa, with dev_u the forward state u_t that entered the step and
 * dev_p_in = dJ/du_{t+1}.  dev_gkappa is an n*n array of DOUBLES (the sum
 * over steps cancels; each contribution, a product of differences of close
 * FP32 values, is formed exactly in FP64); its non-member cells in member
 * 8 x 8 blocks are set to 0.  All five arrays distinct.  Errors:
 * FRACTAL_EINVAL, FRACTAL_ECUDA.
 */
int fractal_adjoint_diffusion_step(fractal_plan_t plan, const float* dev_u, const float* dev_p_in, float* dev_p_out,
                                   const float* dev_kappa, double* dev_gkappa, float a, void* stream);

/* The reverse step with u and p in doubles (see fractal_step_diffusion_kappa_f64). */
int fractal_adjoint_diffusion_step_f64(fractal_plan_t plan, const double* dev_u, const double* dev_p_in,
                                       double* dev_p_out, const float* dev_kappa, double* dev_gkappa, double a,
                                       void* stream);

/*
 * fractal_step_diffusion_kappa_df / fractal_adjoint_diffusion_step_df -- the
 * same two operations with the state, p and dJ/dkappa in double-float: every
 * value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2, about
 * 48 significant bits), stored as consecutive (hi, lo) pairs, so each of
 * dev_a, dev_b, dev_u, dev_p_in, dev_p_out and dev_gkappa is an array of 2*n*n
 * floats (dev_kappa stays n*n floats).  Double-float arithmetic (Knuth's
 * TwoSum, Dekker's product with a fused multiply-add) runs on the FP32 pipes,
 * where this GPU has many times its FP64 rate; it keeps the gradients of a
 * 200-step run within 1e-4 of an FP64 reference like the double state does.
 * a is rounded to the nearest double-float.  For k >= 4 the steps of
 * fractal_step_diffusion_kappa_df run temporally fused (the launches below,
 * up to max_steps each, a and b alternating with the parity of `steps`).
 * Errors as above.
 */
int fractal_step_diffusion_kappa_df(fractal_plan_t plan, float* dev_a, float* dev_b, const float* dev_kappa,
                                    double a, int steps, void* stream);
int fractal_adjoint_diffusion_step_df(fractal_plan_t plan, const float* dev_u, const float* dev_p_in,
                                      float* dev_p_out, const float* dev_kappa, float* dev_gkappa, double a,
                                      void* stream);

/*
 * Fused gradient path (double-float, k >= 4).  The reverse step is the
 * forward operator A applied to p (A is symmetric), so one kernel carries u
 * forward and p back through a checkpoint segment, several steps per launch
 * (super-tiles of side min(128, n) with the member blocks of their margin
 * boxes, one 8 x 8 block per thread, ports in shared memory), recording the
 * states it passes in compact form; dJ/dkappa of the segment is then summed
 * from the two recorded trajectories in one pass.  Not in the paper.
 *
 * A trajectory holds states in record form: 3^(k-3) records of 56 floats
 * (the 27 members of a member 8 x 8 block as (hi, lo) pairs and a pad),
 * record_floats floats per state, state s at dev_traj + s * record_floats.
 *
 * fractal_kappa_fused_limits -- for level k and launch mode: the floats of
 * one recorded state and the most steps one launch takes.  Host only.
 * Errors: FRACTAL_EINVAL (k < 4 or > 16, bad mode, NULL).
 *
 * fractal_kappa_trajectory_df -- `steps` (1 .. max_steps) steps of the
 * double-float conductivity diffusion from dev_in (2*n*n floats): the state
 * before each step into the trajectory's states 0 .. steps - 1 (dev_traj,
 * nullable) and the result into dev_out (2*n*n floats, every cell of every
 * member 8 x 8 block written, 0 at non-members); with dev_out NULL the result
 * goes to trajectory state `steps` instead.  Asynchronous.  Errors:
 * FRACTAL_EINVAL (NULL dev_in or dev_kappa, both outputs NULL, aliasing,
 * alignment, steps out of range, a not finite, k < 4), FRACTAL_ECUDA.
 *
 * fractal_kappa_gradient_df -- dev_gkappa (2*n*n floats, double-float) +=
 * the dJ/dkappa contributions of `steps` steps t0 .. t0 + steps - 1 of a
 * segment: dev_utraj state s = u_(t0+s), dev_ptraj state s = p_(t0+steps-s)
 * (the trajectory the reverse launch records from p_(t0+steps)); per link and
 * step (a / 2) (u_nb - u_c) (p_c - p_nb) at both ends.  Writes every cell of
 * every member 8 x 8 block of dev_gkappa (0 at non-members).  Asynchronous.
 * Errors: FRACTAL_EINVAL, FRACTAL_ECUDA.
 */
int fractal_kappa_fused_limits(int k, int mode, int64_t* record_floats, int* max_steps);

/* Temporal fusion of fractal_step_diffusion_kappa_df on (on != 0, the
 * default) or off (one launch of the single-step kernel per step, for
 * comparison).  Errors: FRACTAL_EINVAL (NULL plan). */
int fractal_plan_set_kappa_fusion(fractal_plan_t plan, int on);
int fractal_kappa_trajectory_df(fractal_plan_t plan, const float* dev_in, float* dev_out, float* dev_traj,
                                const float* dev_kappa, double a, int steps, void* stream);

/*
 * fractal_kappa_trajectory_df_io -- fractal_kappa_trajectory_df with the
 * formats of its input and result chosen: in_format / out_format
 * FRACTAL_DF (n*n double-float pairs, as fractal_kappa_trajectory_df) or
 * FRACTAL_F32 (n*n floats: a float32 input x enters as the pair (x, 0); a
 * float32 result is hi + lo rounded to float).  The steps run in double-float
 * either way; this saves the caller the conversions before the first and
 * after the last launch.  A float32 result has every cell of every member
 * 8 x 8 block written (0 at non-members), no other cell.  Errors: as
 * fractal_kappa_trajectory_df, and FRACTAL_EINVAL for another format.
 */
int fractal_kappa_trajectory_df_io(fractal_plan_t plan, const void* dev_in, int in_format, void* dev_out,
                                   int out_format, float* dev_traj, const float* dev_kappa, double a, int steps,
                                   void* stream);
int fractal_kappa_gradient_df(fractal_plan_t plan, const float* dev_utraj, const float* dev_ptraj,
                              float* dev_gkappa, double a, int steps, void* stream);

/*
 * fractal_kappa_gradient_df_io -- fractal_kappa_gradient_df with the sum's
 * start and destination chosen: accumulate != 0 adds to dev_gkappa (as
 * fractal_kappa_gradient_df), accumulate == 0 starts from 0 (dev_gkappa is
 * then not read, so it need not be cleared); the result goes to dev_gkappa
 * (double-float), or, when dev_out_f32 is not NULL, to dev_out_f32 as float32
 * (n*n floats, hi + lo rounded once; dev_gkappa is then not written and may
 * be NULL without accumulate).  Either destination has every cell of every
 * member 8 x 8 block written (0 at non-members), no other cell.  With these a
 * segment loop needs no cleared accumulator and no final conversion.
 * Errors: as fractal_kappa_gradient_df, and FRACTAL_EINVAL for dev_gkappa
 * NULL where it is read or written, or aliasing buffers.
 */
int fractal_kappa_gradient_df_io(fractal_plan_t plan, const float* dev_utraj, const float* dev_ptraj,
                                 float* dev_gkappa, int accumulate, float* dev_out_f32, double a, int steps,
                                 void* stream);

/* ------------------------------------------------------------------------
 * Other fractals of the NBB family (Sec. 3.1, Table 1).
 *
 * An NBB fractal is given by its step: k cells (x, y) of an s x s grid
 * (s = 2..4, k = 1..s*s, distinct cells), listed in a host array cells_xy of
 * 2k int32 in the order that numbers the replicas (the hash H of Theorem 1;
 * the numbering is free).  A cell of the level-r fractal (side s^r) is a
 * member iff each of its r base-s digit pairs is a step cell.  For the
 * gasket of fractal_map, s = 2 and the cells (0,1), (0,0), (1,0) in this
 * order give the same map.  Not covered by plans: these entries allocate
 * nothing and keep no state.
 * ------------------------------------------------------------------------ */

/*
 * fractal_nbb_map_blocks -- lambda(omega) of Theorem 1 for every block of
 * the packed k^ceil(r/2) x k^floor(r/2) grid (Lemma 2) of the level-r
 * fractal: dev_xy[2 i], dev_xy[2 i + 1] = (x, y) of the member block that
 * omega = (i mod W, i div W) maps to (2 k^r int32, 8-byte aligned).
 * Asynchronous on `stream`.  Errors: FRACTAL_EINVAL (step, r < 0, k^r or s^r
 * above 2^31 - 1, NULL or misaligned dev_xy), FRACTAL_ECUDA.
 */
int fractal_nbb_map_blocks(int s, int k, const int32_t* cells_xy, int r, void* dev_xy, void* stream);

/*
 * fractal_nbb_write -- the single write of Sec. 6.2 on the level-(r_b + j)
 * fractal (side n = s^(r_b + j), dev_buf n*n floats, row-major) in tiles of
 * side t = s^j: `value` at every member cell, 0 at the other cells of member
 * tiles; no other cell is written.  cta_levels == 0: one CTA of t x t
 * threads per tile, one thread per cell (the paper's setting); mode
 * FRACTAL_LAMBDA launches the k^r_b member tiles through lambda (Theorem 1),
 * FRACTAL_BB all s^(2 r_b) tiles, the non-member ones returning at once.
 * cta_levels == m > 0: one CTA of 256 threads per super-tile of s^m x s^m
 * tiles (Sec. 5.1's further unrolling): lambda at level r_b - m for the
 * super-tiles and at level m for their k^m member tiles, or, BB, all
 * super-tiles and all their tiles with the non-members skipped (at most 4096
 * tiles per super-tile).  Asynchronous.  Errors: FRACTAL_EINVAL (step, r_b or
 * j < 0, cta_levels outside 0..r_b, t > 32, n > 2^20, a grid or super-tile
 * beyond the launch limits, NULL or misaligned dev_buf, mode), FRACTAL_ECUDA.
 */
int fractal_nbb_write(int s, int k, const int32_t* cells_xy, int r_b, int j, int cta_levels, int mode, float value,
                      float* dev_buf, void* stream);

/*
 * fractal_nbb_step_ca -- `steps` steps of the CA test of Sec. 6.2 (B3/S23 on
 * the Moore neighbourhood, only member neighbours counted, non-members never
 * born, cells outside the array dead) on the level-(r_b + j) fractal (side
 * n = s^(r_b + j); dev_a, dev_b: n*n bytes, nonzero = alive, distinct),
 * alternating dev_a -> dev_b -> dev_a ...: the state ends in dev_a for an even
 * `steps`, in dev_b for an odd one.  One CTA of t x t threads per tile of
 * side t = s^j (the paper's setting), the tile and its halo staged in shared
 * memory; mode FRACTAL_LAMBDA launches the member tiles through lambda
 * (Theorem 1), FRACTAL_BB all tiles.  Only member cells are read; member
 * tiles are written (0 at their non-member cells), no other cell.
 * Asynchronous.  Errors: FRACTAL_EINVAL (step, r_b or j < 0, t > 32,
 * n > 2^20, grid limits, NULL or equal buffers, steps < 0, mode),
 * FRACTAL_ECUDA.
 */
int fractal_nbb_step_ca(int s, int k, const int32_t* cells_xy, int r_b, int j, int mode, uint8_t* dev_a,
                        uint8_t* dev_b, int steps, void* stream);

/*
 * fractal_nbb_step_diffusion -- `steps` explicit heat-diffusion steps (float32,
 * u' = u + a * (sum over member 4-neighbours of u_nb - degree * u), zero flux
 * at non-members and at the array's edge, the FDM step of Sec. 1 read as for
 * the gasket) on the level-(r_b + j) fractal (dev_a, dev_b: n*n floats,
 * distinct, 4-byte aligned), alternating dev_a -> dev_b -> dev_a ... as
 * fractal_nbb_step_ca; one CTA of t x t threads per tile of side t = s^j,
 * the tile and its halo staged in shared memory, by the lambda or the BB
 * launch.  Only member cells are read; member tiles are written (0 at their
 * non-member cells), no other cell.  Asynchronous.  Errors: FRACTAL_EINVAL
 * (as fractal_nbb_step_ca, and a NaN), FRACTAL_ECUDA.
 */
int fractal_nbb_step_diffusion(int s, int k, const int32_t* cells_xy, int r_b, int j, int mode, float* dev_a,
                               float* dev_b, float a, int steps, void* stream);

/*
 * fractal_nbb_reduce -- the reduce test of Sec. 6.2 (RD): *dev_out = the sum
 * of dev_buf over the member cells of the level-(r_b + j) fractal (n*n
 * floats; non-member cells are not read), in FP64.  One CTA per tile of side
 * t = s^j (t * t threads rounded up to whole warps), each writing its FP64
 * partial into dev_partials (caller-owned: k^r_b doubles for
 * FRACTAL_LAMBDA, s^(2 r_b) for FRACTAL_BB, whose CTAs on non-member tiles
 * write 0); one CTA then adds the partials in a fixed order, so the result
 * does not vary from call to call.  Asynchronous; calls sharing dev_partials
 * must not overlap.  Errors: FRACTAL_EINVAL (step, sizes as
 * fractal_nbb_step_ca, NULL pointers, partials_len below the launch's CTA
 * count, mode), FRACTAL_ECUDA.
 */
int fractal_nbb_reduce(int s, int k, const int32_t* cells_xy, int r_b, int j, int mode, const float* dev_buf,
                       double* dev_partials, int64_t partials_len, double* dev_out, void* stream);

/* ------------------------------------------------------------------------
 * Batches: many independent gaskets of uneven levels in one launch.
 *
 * The diffusion step of fractal_step_diffusion applied to `count` separate
 * instances, instance i of level k_i in its own n_i x n_i arrays (n_i =
 * 2^k_i).  One persistent launch covers all of them: its CTAs walk the
 * instances' member super-tiles in order, an instance's super-tiles forming
 * the contiguous range [first_i, first_i + 3^R_i) of a per-instance offset
 * table (prefix sums); a CTA finds its instance by binary search on that
 * table and its super-tile by lambda(omega) at level R_i = k_i - log2(T)
 * (Theorem 1).  Each super-tile runs the temporally fused diffusion (several
 * steps per launch, one 8 x 8 block of the gasket per thread).  Results are
 * bit for bit those of fractal_step_diffusion on each instance with the same
 * steps per launch.  Not in the paper: the batching is this library's.
 * ------------------------------------------------------------------------ */
typedef struct fractal_batch_s* fractal_batch_t;

typedef struct fractal_batch_info {
  int32_t count;            /* instances */
  int32_t k_min, k_max;     /* smallest and largest level */
  int32_t supertile;        /* super-tile side T in cells (same for all instances) */
  int32_t steps_per_launch; /* temporal fusion: steps one launch advances */
  int32_t ctas;             /* persistent grid: CTAs per launch */
  int32_t threads;          /* threads per CTA */
  int32_t smem_bytes;       /* dynamic shared memory per CTA */
  int64_t supertiles;       /* member super-tiles over all instances: sum 3^R_i */
  int64_t members;          /* member cells over all instances: sum 3^k_i */
  int32_t bound;            /* 1 after fractal_batch_bind */
  int32_t graph_steps;      /* steps in the captured graph, 0 if none */
} fractal_batch_info;

/*
 * fractal_batch_create -- a batch of `count` (1 .. 65536) instances with the
 * levels ks[0..count-1] (host array; 4 <= k_i <= 16).  The batch owns a small
 * device table (the instances' pointers, sizes and super-tile offsets), a
 * non-blocking stream used only to capture graphs, and any captured graph.
 * Default: 8 steps per launch, the largest super-tile side <= 256 that every
 * instance holds.  Belongs to the device current at the call.  Errors:
 * FRACTAL_EINVAL, FRACTAL_ENOMEM, FRACTAL_ECUDA.
 */
int fractal_batch_create(int count, const int32_t* ks, fractal_batch_t* batch);

/* Free a batch and its graph (NULL accepted); waits for nothing. */
int fractal_batch_destroy(fractal_batch_t batch);

/*
 * fractal_batch_bind -- the instances' buffers: dev_a[i] and dev_b[i] (host
 * arrays of `count` device pointers) are distinct n_i*n_i float32 arrays,
 * 16-byte aligned.  Copies the table to the device (synchronous); may be
 * called again with other buffers, which a captured graph then uses too.
 * The first call also allocates the batch's block records (two buffers of
 * sum_i 3^(k_i-3) records of 112 bytes), where the state stays between the
 * launches of one step call.
 * Errors: FRACTAL_EINVAL (NULL, equal or misaligned pointers), FRACTAL_ENOMEM,
 * FRACTAL_ECUDA.
 */
int fractal_batch_bind(fractal_batch_t batch, float* const* dev_a, float* const* dev_b);

/*
 * fractal_batch_configure -- super-tile side T (a power of two, 16 <= T <=
 * 2^k_min, T >= 2 * margin, at most 288 block slots per super-tile, or 320
 * for T = 256 at margins of 64 cells) and steps per launch spl (1 .. 56;
 * margin = the smallest power of two >= max(spl, 8)).  T = 0 keeps
 * the current side.  Drops a captured graph.  Synchronous when bound (the
 * offset table is rewritten).  Errors: FRACTAL_EINVAL, FRACTAL_ECUDA.
 */
int fractal_batch_configure(fractal_batch_t batch, int supertile, int steps_per_launch);

/*
 * fractal_batch_step_diffusion -- `steps` diffusion steps (coefficient a, as
 * fractal_step_diffusion) on every instance, in ceil(steps / spl) persistent
 * launches (two for a single even-step launch), the state in the batch's
 * block records between them: after the call each instance's state is in
 * dev_a[i] when `steps` is even and in dev_b[i] when it is odd (the other
 * buffer is not written by a call of several launches).  Asynchronous on
 * `stream`.  Errors: FRACTAL_EINVAL (unbound,
 * steps < 0, a not finite), FRACTAL_ECUDA.
 */
int fractal_batch_step_diffusion(fractal_batch_t batch, float a, int steps, void* stream);

/*
 * fractal_batch_reduce -- per-instance sums over the member cells of dev_a[i]
 * (which = 0) or dev_b[i] (which = 1): dev_out[i] (device array of `count`
 * doubles).  Each super-tile's FP32 values are summed in FP64 in a fixed
 * order, then each instance's super-tiles in order: deterministic.
 * Asynchronous.  Errors: FRACTAL_EINVAL, FRACTAL_ENOMEM, FRACTAL_ECUDA.
 */
int fractal_batch_reduce(fractal_batch_t batch, int which, double* dev_out, void* stream);

/*
 * fractal_batch_autotune -- time every valid (super-tile side, steps per
 * launch in {8, 16, 32}) on the bound buffers (launches dev_a -> dev_b,
 * `reps` timed after two untimed; dev_a is only read, dev_b overwritten) and
 * keep the fastest per step.  Synchronises `stream`.  *best_us (nullable):
 * the best mean step time.  Errors: FRACTAL_EINVAL, FRACTAL_ENOMEM,
 * FRACTAL_ECUDA.
 */
int fractal_batch_autotune(fractal_batch_t batch, float a, int reps, float* best_us, void* stream);

/*
 * fractal_batch_graph_capture -- capture the launches of
 * fractal_batch_step_diffusion(batch, a, steps) into a CUDA graph owned by
 * the batch (replacing any earlier one) and instantiate it.  Captured on the
 * batch's own stream; nothing runs.  Errors: FRACTAL_EINVAL (unbound, steps
 * < 1), FRACTAL_ECUDA.
 */
int fractal_batch_graph_capture(fractal_batch_t batch, float a, int steps);

/* Launch the captured graph on `stream` (asynchronous).  Errors:
 * FRACTAL_EINVAL (no graph), FRACTAL_ECUDA. */
int fractal_batch_graph_launch(fractal_batch_t batch, void* stream);

/* Fill *info.  Errors: FRACTAL_EINVAL (NULL). */
int fractal_batch_get_info(fractal_batch_t batch, fractal_batch_info* info);

#ifdef __cplusplus
}
#endif

#endif /* FRACTAL_H_ */
