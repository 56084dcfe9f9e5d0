/*
 * d8.h -- C ABI of libd8, GB300 (sm_103a) D8 flow directions and up-slope area.
 *
 * Method: Barnes, Lehman, Mulla, "Distributed Parallel D8 Up-Slope Area
 * Calculation in Digital Elevation Models" (PDPTA 2011).
 *
 * Conventions shared by every call:
 *  - Grids are row-major: cell (i, j) of an H x W grid lives at i*ld + j,
 *    where ld >= W is the leading dimension in ELEMENTS.  Row i grows to the
 *    south.
 *  - Direction codes (uint8): 0..7 = N, NE, E, SE, S, SW, W, NW; 8 = OUTLET
 *    (a cell on the first/last row or column: it receives flow and passes none
 *    on); 9 = SINK (no strictly lower neighbour).
 *  - Every pointer passed to a compute call is a DEVICE pointer on the
 *    context's device unless the parameter says "host".  The caller owns all
 *    input and output buffers; the library never frees them.  Inputs and
 *    outputs must not overlap.
 *  - Compute calls are asynchronous on `stream` (a cudaStream_t, or NULL for
 *    the legacy default stream).  Their return value reports errors the host
 *    can see (bad arguments, allocation or launch failure).  Errors found on
 *    the device (non-finite elevation, invalid code, cycle, timeout) are
 *    OR-ed into the context's status word; d8_get_status() reads and clears it.
 *  - A context owns its workspace (device arrays for the per-tile perimeter
 *    summaries and the combine), grown lazily with cudaMalloc and reused.
 *    Calls on one context must not run concurrently on different streams.
 */
#ifndef D8_H_
#define D8_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  D8_OK = 0,
  D8_ERR_ARG = 1,       /* bad pointer, size, leading dimension, rule or code */
  D8_ERR_SHAPE = 2,     /* H*W too large for the output type */
  D8_ERR_NONFINITE = 3, /* device: an elevation is NaN or infinite */
  D8_ERR_CYCLE = 4,     /* device: the direction field contains a cycle */
  D8_ERR_NOMEM = 5,     /* workspace allocation failed */
  D8_ERR_CUDA = 6,      /* a CUDA runtime call failed */
  D8_ERR_TIMEOUT = 7,   /* an iteration bound was reached (d8_fill) */
  D8_ERR_CAPACITY = 8   /* grid larger than the fixed scratch of d8_flowdir_accumulate_noalloc */
} d8_status;

/* Direction rules ("The Algorithm": steepest slope, slope = drop divided by
 * the distance between cell centres, 1 or sqrt 2; "Introduction": lowest
 * neighbour).  Ties go to the first direction in N, NE, E, SE, S, SW, W, NW
 * order; only a strictly positive drop counts.  D8_RULE_NODATA may be added
 * to either rule: a cell with a non-finite elevation is then outside the
 * study area and gets OUTLET, and so does every cell next to one (the area's
 * edge drains off it, as the grid's edge does), with no error raised.  To
 * leave such cells out of weighted sums, give them weight 0 (and cell areas
 * as weights where cells differ in area: "Up-Slope Area"). */
typedef enum { D8_RULE_STEEPEST = 0, D8_RULE_LOWEST = 1, D8_RULE_NODATA = 2 } d8_rule;

typedef struct d8_ctx d8_ctx;
typedef struct d8_batch d8_batch;
typedef void* d8_stream; /* a cudaStream_t */

/* Create a context on CUDA device `device` (made current for the call).
 * *ctx receives the handle.  Errors: D8_ERR_ARG (ctx NULL), D8_ERR_CUDA. */
d8_status d8_create(d8_ctx** ctx, int device);

/* Synchronise the device, free the workspace and the handle.  NULL is a no-op. */
d8_status d8_destroy(d8_ctx* ctx);

/* Tile side used by later calls: 32, 64 or 128 (default 64).  One thread
 * block holds one T x T tile (the paper's "slave partition") in shared
 * memory.  D8_ERR_ARG for any other value. */
d8_status d8_set_tile(d8_ctx* ctx, int tile);

/* Frontier strategy used by later calls (and by batch plans made later): how
 * the chains of the flow forest are traversed.  0 = chain walks ("last input
 * continues", Algorithm 2's tail recursion) fed from a per-warp ring of
 * pending sources refilled by warp votes in the tiles, and the queue method
 * (Algorithm 6) with one walk per chain at the combine's top level
 * (default); 1 = the tiles' walks fed from per-thread source bit masks, idle
 * lanes served by lanes with sources to spare; 2 = ring walks in the tiles
 * and pointer jumping at the top level (every exit adds its partial sum to
 * its 2^r-th ancestor, then jumps, for ceil(log2(depth)) rounds), for DEMs
 * whose channels cross tile borders very many times.  Unit counts are
 * identical under every strategy; weighted sums may differ in the last bits
 * (their order of addition changes).  D8_ERR_ARG for any other value. */
d8_status d8_set_strategy(d8_ctx* ctx, int strategy);

/* D8 flow direction of every cell ("The Algorithm"; "Introduction").
 * z: H x W fp32 elevations (ld ldz); dir: H x W codes (ld lddir).
 * Non-finite z sets D8_ERR_NONFINITE in the status word and gives that cell
 * SINK, unless the rule carries D8_RULE_NODATA.  Errors: D8_ERR_ARG. */
d8_status d8_flowdir(d8_ctx* ctx, const float* z, int64_t H, int64_t W, int64_t ldz, uint8_t* dir,
                     int64_t lddir, d8_rule rule, d8_stream stream);

/* Unit up-slope area A(p) = 1 + sum of A over the cells draining into p
 * (Eq. 1, section "Up-Slope Area"), computed with the paper's partition
 * scheme: per-tile internal areas with unknown inflows (Algorithms 1-4), a
 * device solve of the tile-perimeter link graph (Algorithms 5-6) and a
 * finalising pass per tile (Algorithms 7-8).
 * dir: H x W codes (any field: a code 0..7 pointing off the grid, 8 and 9 end
 * a path; codes > 9 set D8_ERR_ARG in the status word; a cycle sets
 * D8_ERR_CYCLE).  A: H x W uint32 counts (ld ldA).
 * Errors: D8_ERR_ARG, D8_ERR_SHAPE (H*W > 2^32-1), D8_ERR_NOMEM, D8_ERR_CUDA. */
d8_status d8_accumulate(d8_ctx* ctx, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir, uint32_t* A,
                        int64_t ldA, d8_stream stream);

/* Directions and unit counts in one call: the direction stencil writes dir,
 * then the per-tile passes, the combine and the finalising pass of
 * d8_accumulate run on it (z is read once; dir is written once and read back
 * by the tile passes).  Same arguments and errors as d8_flowdir +
 * d8_accumulate. */
d8_status d8_flowdir_accumulate(d8_ctx* ctx, const float* z, int64_t H, int64_t W, int64_t ldz, d8_rule rule,
                                uint8_t* dir, int64_t lddir, uint32_t* A, int64_t ldA, d8_stream stream);

/* Directions of a horizontal strip of a taller grid (the paper's row-strip
 * partition, "The Algorithm": each partition owns consecutive rows and sees
 * one row of its neighbours).  As d8_flowdir on the H x W strip, except that
 * halo bit 0 says the row above the strip's first row is readable at
 * z - ldz and belongs to the grid (the first row is then not an edge and gets
 * a real direction, possibly towards that row), and bit 1 the same for the
 * row below the last row (at z + H*ldz).  Codes pointing out of the strip end
 * a path when the strip's directions are accumulated on their own: those
 * cells are the strip's exits.  Errors: D8_ERR_ARG. */
d8_status d8_flowdir_strip(d8_ctx* ctx, const float* z, int64_t H, int64_t W, int64_t ldz, int halo, d8_rule rule,
                           uint8_t* dir, int64_t lddir, d8_stream stream);

/* Unit up-slope counts of a direction field that also receives flow from
 * outside across its first and last rows (Algorithms 7-8 for a strip whose
 * neighbours' resolved exits drain into it): A(p) = 1 + sum of A over the
 * cells draining into p + in(p), where in(0, j) = top_in[j] and
 * in(H-1, j) = bottom_in[j] (device arrays of W uint32; either may be NULL
 * for none).  Otherwise as d8_accumulate. */
d8_status d8_accumulate_inflow(d8_ctx* ctx, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir,
                               const uint32_t* top_in, const uint32_t* bottom_in, uint32_t* A, int64_t ldA,
                               d8_stream stream);

/* Weighted up-slope area A(p) = w(p) + sum of A over the cells draining into
 * p (Eq. 1 with the paragraph after it: cells "may or may not be weighted
 * equally").  fp32 in and out.  Sums are float-float (TwoSum-compensated
 * fp32) inside tiles and across them; the inflow a tile receives is added
 * along its paths in exact per-tile fixed point (78 value bits, scaled to the
 * tile's summed inflow), so the result keeps fp32 accuracy across wide
 * ranges of weights.  w: H x W (ld ldw); A: H x W (ld ldA).  Errors as
 * d8_accumulate, plus D8_ERR_NONFINITE when a non-finite weight's area
 * reaches another tile. */
d8_status d8_accumulate_weighted(d8_ctx* ctx, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir,
                                 const float* w, int64_t ldw, float* A, int64_t ldA, d8_stream stream);

/* Adjoint of d8_accumulate_weighted: for a loss L with dL/dA = dA,
 * dw(q) = dL/dw(q) = dA(q) + dw(down-slope neighbour of q), i.e. the sum of
 * dA over q's flow path (the transpose of Eq. 1).  Per-tile path sums, a
 * pointer-jumping solve over the tile exits, then a finalising pass; the
 * tiles are 64 x 64, or 32 x 32 when d8_set_tile chose 32 (128 x 128 tiles
 * would not fit in shared memory).  Deterministic: the result does not depend
 * on the launch configuration.  fp32 in and out, compensated accumulation.
 * Errors as d8_accumulate. */
d8_status d8_accumulate_backward(d8_ctx* ctx, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir,
                                 const float* dA, int64_t lddA, float* dw, int64_t lddw, d8_stream stream);

/* Pit and flat removal by epsilon filling, the precondition of the method
 * ("The Algorithm", first paragraph: pits raised and flats resolved, so that
 * every interior cell has a strictly lower neighbour).  F is the unique
 * surface with F = z on the grid's edge and, for every interior cell c with
 * m = the lowest of its 8 neighbouring F values, F(c) = z(c) if z(c) > m,
 * else F(c) = max(fl32(m + eps), the next fp32 value above m); it is the
 * result of a priority flood from the edge that raises each cell reached
 * from a cell no lower than it to eps above that cell.
 * z: H x W fp32 elevations (ld ldz); F: H x W fp32 output (ld ldF), must
 * not overlap z; eps >= 0 (0 raises by one fp32 step).  rounds: optional
 * host pointer receiving the number of tile rounds the fill took (how far
 * the filled surface's dependencies wind across the 64 x 64 tiles).
 * Non-finite z sets D8_ERR_NONFINITE in the status word (F is then
 * unspecified).  The call synchronises `stream` (it checks for convergence
 * on the host every 16 rounds).
 * Errors: D8_ERR_ARG, D8_ERR_NOMEM, D8_ERR_CUDA, D8_ERR_TIMEOUT (not settled
 * after 2^20 rounds). */
d8_status d8_fill(d8_ctx* ctx, const float* z, int64_t H, int64_t W, int64_t ldz, float eps, float* F,
                  int64_t ldF, int64_t* rounds, d8_stream stream);

/* Plan a batch of n independent DEMs with the given shapes (host arrays of n
 * entries; DEM k is H[k] x W[k], dense, ld = W[k]).  The plan owns a tile
 * table, a workspace sized for the whole batch and (after the first run) a
 * CUDA graph of the pipeline.  Errors: D8_ERR_ARG, D8_ERR_SHAPE, D8_ERR_NOMEM. */
d8_status d8_batch_plan(d8_ctx* ctx, int n, const int64_t* H, const int64_t* W, d8_batch** plan);

/* Directions and unit counts for every DEM of the batch: one persistent
 * launch per pipeline stage over all tiles of all DEMs, fed by a device tile
 * work queue.  z, dir, A: host arrays of n device pointers.  The first call
 * captures the pipeline in a CUDA graph; later calls with the same pointers
 * and rule replay it.  Errors as d8_flowdir_accumulate. */
d8_status d8_batch_flowdir_accumulate(d8_batch* plan, const float* const* z, uint8_t* const* dir,
                                      uint32_t* const* A, d8_rule rule, d8_stream stream);

/* Free a plan (synchronises its stream first).  NULL is a no-op. */
d8_status d8_batch_destroy(d8_batch* plan);

/* Autotuner for batches: runs d8_batch_flowdir_accumulate on the given batch
 * (shapes and buffers exactly as for d8_batch_plan and
 * d8_batch_flowdir_accumulate) at every supported tile side (32, 64, 128)
 * with every frontier strategy (0, 1, 2; see d8_set_strategy): per point one
 * untimed run that captures the graph, then 5 graph replays timed one by
 * one, scored by their median.  The fastest point wins: *best_tile and
 * *best_strategy (may be NULL) receive it, and the context's tile side and
 * strategy are set to it, so a plan made next uses them.  ms: optional host
 * array of 9 floats receiving the medians in milliseconds, tile-major
 * (ms[3 * t + s] for tile index t = 0, 1, 2 and strategy s), -1 where a point
 * failed.  The paper has no counterpart: its partition size is an input of the
 * method, and here it is chosen by measurement on the target GPU.  dir and A
 * hold the results of the last run.  Synchronises `stream`.
 * Errors: D8_ERR_ARG, or the first error of the runs if every point failed. */
d8_status d8_batch_autotune(d8_ctx* ctx, int n, const int64_t* H, const int64_t* W, const float* const* z,
                            uint8_t* const* dir, uint32_t* const* A, d8_rule rule, d8_stream stream, int* best_tile,
                            int* best_strategy, float* ms);

/* Synchronise `stream`, read and clear the context's device status word.
 * Returns D8_OK or the first device-side error recorded (NONFINITE, ARG,
 * CYCLE, TIMEOUT, in that order of precedence). */
d8_status d8_get_status(d8_ctx* ctx, d8_stream stream);

/* Link-graph statistics of the combine of the last d8_accumulate,
 * d8_flowdir_accumulate or d8_accumulate_weighted call on this context
 * (Algorithms 5-6; the paper's winding of flow paths across partitions):
 * out[0] = group levels above the tiles, out[1] = units at the top level
 * (0 when the group levels covered the grid), out[2] = exits in the top
 * level's link graph, out[3] = pointer-jumping rounds that found work
 * (strategy 2; the graph's depth is below 2^out[3]) or -1 (queue walk).
 * out: host array of n >= 4 entries.  Synchronises `stream`.
 * Errors: D8_ERR_ARG, D8_ERR_CUDA. */
d8_status d8_combine_stats(d8_ctx* ctx, d8_stream stream, int64_t* out, int n);

/* Static text for a status code. */
const char* d8_status_string(d8_status s);

/* Per-stage device timing of the calls made while profiling is on.
 * d8_set_profiling(ctx, 1) records CUDA events around every stage launch of
 * the following calls.  d8_stage_times() synchronises on the last event and
 * writes, for each stage s < max, the summed milliseconds ms[s] and the
 * launch count launches[s] since the last reset (either may be NULL), then
 * resets them; it returns the number of stages through *n.  Stage names come
 * from d8_stage_name(s). */
d8_status d8_set_profiling(d8_ctx* ctx, int on);
d8_status d8_stage_times(d8_ctx* ctx, float* ms, int64_t* launches, int max, int* n);
const char* d8_stage_name(int stage);

/* Library version string. */
const char* d8_version(void);

/* Directions and unit counts exactly as d8_flowdir_accumulate computes them,
 * for callers that cannot allocate device memory when they call: processes
 * running under a fixed memory budget reserved at start-up, callers whose
 * pool or arena allocator owns all device memory, and callers that cannot
 * create a context (d8_create allocates its status word and, later, its
 * workspace).  This call needs no context and allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.  The paper has no counterpart;
 * this is an interface for such callers, not a step of the method.
 *
 * Its scratch is one fixed 64 MiB array inside the library, held by every GPU
 * that loads the library until the process exits.  It fits grids of up to
 * about 11,900 tiles of 64 x 64 cells (ceil(H/64) * ceil(W/64) tiles, e.g.
 * 6976 x 6976, ~48 M cells); larger grids return D8_ERR_CAPACITY before any
 * GPU work is queued.  Tile side 64, whatever d8_set_tile says elsewhere.
 *
 * z, dir, A: as d8_flowdir_accumulate (device pointers on the current device,
 * owned by the caller).  status: optional device pointer to one uint32 that
 * the call first clears and then ORs device-side errors into as
 * (1 << d8_status) bits (non-finite z, invalid code, cycle); with NULL the
 * errors go to a status word inside the shared scratch instead, which every
 * call clears and writes, so they cannot be read back reliably.
 * Asynchronous on `stream`.
 *
 * The first call on a device looks up the device address of the scratch
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before capturing any stream into a CUDA graph.  The address is kept for
 * the life of the process: after cudaDeviceReset on a device it is stale, so
 * do not call this entry point on that device again in the same process.
 * All calls share the one
 * scratch array and it keeps the previous call's contents (the call clears
 * what must start at zero itself); calls whose GPU work can overlap in time --
 * on different streams or from different threads without ordering between
 * them -- race on it and give wrong results.
 *
 * Errors: D8_ERR_ARG, D8_ERR_SHAPE (H*W > 2^32 - 1), D8_ERR_CAPACITY,
 * D8_ERR_CUDA. */
d8_status d8_flowdir_accumulate_noalloc(const float* z, int64_t H, int64_t W, int64_t ldz, d8_rule rule,
                                        uint8_t* dir, int64_t lddir, uint32_t* A, int64_t ldA, uint32_t* status,
                                        d8_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* D8_H_ */
