/*
 * gridder.h: C ABI of the GB300 convolutional gridder (Merry 2016, "Faster
 * GPU-based convolutional gridding via thread coarsening").
 *
 * Gridding (Sec. 2.2) treats every visibility as a Dirac delta. It convolves
 * the delta with an oversampled, separable gridding convolution function
 * (GCF, Sec. 2.2 and Sec. 4) and accumulates the result on a regular G x G
 * complex grid, one plane per polarization. The GPU kernels use Romein's
 * sliding-window work distribution (Sec. 2.2, Fig. 1) with thread coarsening
 * (Sec. 3, Fig. 2): each thread owns a Bu x Bv block of grid points and keeps
 * register accumulators, which it flushes with atomic adds only when the
 * visibility's bounding box moves off its block. Degridding is built as the
 * exact adjoint.
 *
 * Conventions (for every entry point):
 *  - uv: [n][2] float64 (u, v) in grid-pixel units relative to the grid
 *    centre. Cell G/2 holds u = 0.
 *  - Fine position: f = floor(u*O + 1/2), evaluated exactly on the float64
 *    input. Centre cell: C = floor((f + O/2)/O) + G/2. Table row:
 *    r = f - (C - G/2)*O + O/2, in [0, O).
 *  - Footprint: cells C-h .. C-h+S-1 per axis, with h = (S-1)/2. A
 *    visibility whose footprint is not wholly inside the grid, or whose
 *    coordinates are not finite, is skipped and counted.
 *  - Tap (i, j) of a visibility is table[r_u][i] * table[r_v][j].
 *  - Layouts:
 *    - vis: [n][npol] complex, interleaved (re, im). Stored as float32
 *      (GRID_PREC_F32), or as bf16 / fp16 pairs.
 *    - weights: [n] float32.
 *    - Values and weights are expected to be finite. A non-finite one is not
 *      confined to its footprint: the register blocks that take it also
 *      cover padding cells, and in the sorted schedule a thread's later
 *      blocks in the same chunk take it too.
 *    - kernel_table: [O][S] real, float32, or bf16 / fp16 to match the
 *      plan's precision.
 *    - grid: [npol][G][G] complex64, row index v, column index u.
 *  - Every data pointer is a caller-owned DEVICE pointer, except the *_host
 *    buffers of grid_degrid_host and grid_degrid_host_steps (pinned host
 *    memory). Pointers are borrowed until the work queued on `stream`
 *    completes. Calls are asynchronous on `stream`; a device fault surfaces
 *    at the caller's next synchronisation.
 *  - Threads: different plans (and batches) are independent. One plan must not
 *    be used by several host threads at once (its scratch, skipped counter,
 *    copy streams and events are shared by its calls). Error messages are
 *    per host thread.
 *  - Return value: GRID_OK (0) or a negative GRID_ERR_* code. The message of
 *    the last error on the calling thread is in grid_last_error(). Nothing
 *    aborts the process.
 */
#ifndef GB300_GRIDDER_H
#define GB300_GRIDDER_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grid_plan_s* grid_plan_t;

enum {
  GRID_OK = 0,
  GRID_ERR_INVALID = -1,     /* bad argument: size, null or misaligned pointer, range */
  GRID_ERR_UNSUPPORTED = -2, /* valid, but no kernel is built for it (for example a too large Bu*Bv*npol) */
  GRID_ERR_NOMEM = -3,       /* device allocation of plan scratch failed */
  GRID_ERR_CUDA = -4         /* a CUDA runtime call or kernel launch failed */
};

/* Storage precision of vis and kernel_table. Accumulation is always FP32. */
enum { GRID_PREC_F32 = 0, GRID_PREC_BF16 = 1, GRID_PREC_F16 = 2 };

/* Work distribution. */
enum {
  /* Sec. 4: fixed-size chunks of baseline-ordered visibilities, one team of
   * threads per chunk, in the input order. Flushes go straight to the grid in
   * global memory with atomic adds. */
  GRID_SCHED_CHUNKED = 0,
  /* The same chunks, first binned by the grid "patch" (a square region of
   * the grid) their footprints start in. A CTA accumulates one patch plus a
   * halo in shared memory. Register flushes that land there use shared
   * atomics, and flushes that land outside it go to global memory. The patch
   * reaches the grid once per work item, with coalesced vector atomics. */
  GRID_SCHED_PATCH = 1,
  /* Gridding as GRID_SCHED_CHUNKED. Degridding by tile gather: each warp
   * takes 32 consecutive visibilities, copies the bounding box of their
   * footprints (up to (S+13) x (S+13) cells per polarization) from the grid
   * into shared memory (tiled tensor copies through tensor maps over the
   * grid, one per plane), and each lane sums its own visibility's footprint
   * from there, with no reduction between threads (rows first, the separable
   * form of the Sec. 6 remark). A group whose box is larger reads the grid
   * directly. The same results as the chunked degridder up to FP32 rounding.
   * Odd S <= 15 have unrolled kernels; every other S runs a kernel that
   * reads S at run time (taps from shared memory), while one warp's tile
   * (at most 8*P*(S+13)*(S+24) bytes) and the [O][S] table fit in shared
   * memory (GRID_ERR_UNSUPPORTED otherwise). threads must be a multiple of
   * 32; the CTA is cut to the warps whose tiles fit. tile_group picks 32 or 8
   * visibilities per warp group. */
  GRID_SCHED_TILE = 2,
  /* Gridding with the Sec. 4 chunks and a wider bin than Sec. 3 needs
   * (bin_u x bin_v cells, multiples of Bu and Bv, at most 32 threads per
   * team). A thread still owns the blocks congruent to its position modulo
   * the bin (Sec. 3), but the team's box around the footprint moves only
   * when the footprint leaves it, and then by the fewest blocks. Paths that
   * turn back inside the slack flush nothing; the cost is padding (more
   * zero taps per visibility). With the paper's bin this is the paper's box
   * rule. Built for (Bu, Bv) = (2,1) (2,2) (4,1) (4,2) (2,4) (8,1) at npol 4;
   * (2,2) (4,2) (2,4) (4,4) (8,2) (2,8) at npol 2; those and (8,4) (4,8) (8,8)
   * at npol 1. Threads a multiple of 32.
   * Degridding with such a plan uses the chunked degridder on the paper's
   * bin for the same (Bu, Bv), or for 2 x 2 blocks where no chunked kernel
   * is built for (Bu, Bv). */
  GRID_SCHED_LAZY = 3,
  /* The chunked schedule with each staged batch of 32 visibilities processed
   * in the order of its footprints' first block (v, then u) instead of the
   * input order, so that visibilities sharing a box are neighbours (fewer
   * flushes where tracks step back and forth across block edges); the grid
   * is the same up to FP32 summation order. Tap tables are rotated per
   * (fine row, cell phase), O * bin^2 entries per axis, so that a thread
   * reads its taps at a fixed offset. Teams of at most 64 threads whose CTA
   * fits in shared memory (GRID_ERR_UNSUPPORTED otherwise). Degridding with
   * such a plan uses the chunked degridder. */
  GRID_SCHED_SORTED = 4
};

typedef struct {
  int G;            /* grid side, even, 2 .. 65536 */
  int S;            /* GCF support (taps per axis), 1 .. 64, S <= G */
  int oversample;   /* O, a power of two, 1 .. 256 */
  int npol;         /* polarizations P: 1, 2 or 4 */
  int Bu, Bv;       /* coarsening (block) factors per axis, 1 .. 8; (1, 1) is Romein's plain algorithm */
  int vis_per_chunk;/* visibilities per team chunk (Sec. 4 uses 1024); 0 = default */
  int threads;      /* threads per CTA target; 0 = default (256) */
  int precision;    /* GRID_PREC_* */
  int schedule;     /* GRID_SCHED_* */
  int patch;        /* GRID_SCHED_PATCH: patch side in cells; 0 = default */
  int bin_u, bin_v; /* GRID_SCHED_LAZY: bin sides in cells (multiples of Bu, Bv, at least
                       roundup(S + B - 1, B)); 0 = the paper's bin, one block wider along each
                       axis where it leaves a footprint less than a block of room (u first), as
                       long as the team stays within 32 threads */
  int tile_group;   /* GRID_SCHED_TILE: visibilities per warp group, 32 or 8; 0 = 32. With 8,
                       four lanes share a visibility (each sums every fourth footprint row, the
                       partial sums are added by shuffles) and the tile is 8 cells wider: for
                       tracks that move several cells per visibility, whose groups of 32 do
                       not fit a tile */
} grid_plan_desc;

/* Fill `desc` with the defaults for the given problem and coarsening B (Bu = Bv = B). */
void grid_plan_desc_init(grid_plan_desc* desc, int G, int S, int oversample, int npol, int B);

/*
 * Create a plan (host call). It validates the problem, derives the bin
 * geometry (bin width per axis N_b = roundup(S + B - 1, B), Sec. 3), picks the
 * team shape and allocates the plan's device scratch on the current device.
 * The plan is bound to that device.
 * On success *out holds a plan the caller owns and destroys with
 * grid_plan_destroy().
 */
int grid_plan_create(grid_plan_t* out, int G, int S, int oversample, int npol, int B);
int grid_plan_create_ex(grid_plan_t* out, const grid_plan_desc* desc);

/* Destroy a plan and free its device scratch. NULL is allowed. The caller
 * must make sure no queued work still uses it. */
void grid_plan_destroy(grid_plan_t plan);

/* Copy the plan's resolved parameters (bin widths, team size, ...) into desc. */
int grid_plan_describe(grid_plan_t plan, grid_plan_desc* desc, int* bin_u, int* bin_v, int* team_size);

/*
 * Gridding (Sec. 2.2; kernels: Sec. 3 and Sec. 4):
 *   grid[p][C_v-h+j][C_u-h+i] += w_n * vis[n][p] * table[r_u][i] * table[r_v][j]
 * for every valid visibility n, polarization p and tap (i, j). ACCUMULATES
 * into grid, which the caller zeroes when a fresh grid is wanted.
 * weights may be NULL (unit weights). n_vis may be 0. Visibilities should be
 * ordered by baseline and time (Sec. 4); any order gives the same sums, only
 * more slowly.
 */
int grid(grid_plan_t plan, int64_t n_vis, const double* uv, const void* vis, const float* weights,
         const void* kernel_table, void* grid, cudaStream_t stream);

/*
 * Degridding, the adjoint of gridding with unit weights:
 *   vis[n][p] = sum_{i,j} table[r_u][i] * table[r_v][j] * grid[p][C_v-h+j][C_u-h+i]
 * The paper proposes it as future work (Sec. 6). OVERWRITES vis (always
 * complex64, [n][npol]). A skipped visibility gets 0.
 */
int degrid(grid_plan_t plan, int64_t n_vis, const double* uv, const void* grid, const void* kernel_table,
           void* vis, cudaStream_t stream);

/*
 * Weighted degridding, the exact adjoint of grid() with weights w:
 *   vis[n][p] = w_n * sum_{i,j} table[r_u][i] * table[r_v][j] * grid[p][C_v-h+j][C_u-h+i]
 * This is the backward pass of grid() with respect to the visibilities
 * (Sec. 2.2 defines the forward map). weights may be NULL, which gives
 * degrid(). The other arguments and the overwrite semantics are those of
 * degrid().
 */
int degrid_weighted(grid_plan_t plan, int64_t n_vis, const double* uv, const void* grid, const void* kernel_table,
                    const float* weights, void* vis, cudaStream_t stream);

/*
 * Oversampled Kaiser-Bessel table (Sec. 2.2: precomputed and oversampled).
 * Writes [O][S] values to the DEVICE buffer table_out, in the plan precision
 * `precision`:
 *   table[r][i] = I0(beta*sqrt(1 - (2d/S)^2)) / I0(beta),  d = i - h - (r - O/2)/O,
 * and 0 where |2d/S| > 1. The values are computed in FP64 on the device and
 * rounded once.
 */
int grid_make_kernel_table(int S, int oversample, double beta, int precision, void* table_out, cudaStream_t stream);

/*
 * The per-visibility indices the kernels use, for bit-exact checking (a test
 * hook). The passage they follow is Sec. 2.2's: a visibility is snapped to
 * the nearest point of the oversampled grid, which fixes its cell and the GCF
 * row; the exact rounding rule is the one in the conventions above.
 *   cell[n][2] = (C_u, C_v) and sub[n][2] = (r_u, r_v), or (-1, -1) for both
 *   when the visibility is skipped.
 * Device pointers, int32, caller-owned, n_vis entries each; the call is
 * asynchronous on `stream`. GRID_ERR_INVALID for a null or misaligned
 * pointer.
 */
int grid_compute_indices(grid_plan_t plan, int64_t n_vis, const double* uv, int32_t* cell, int32_t* sub,
                         cudaStream_t stream);

/*
 * Number of visibilities skipped (invalid or off the grid) by the plan's calls
 * since it was created or last reset. A bookkeeping call with no passage of
 * its own: it reports the edge rule of the conventions above (the paper is
 * silent on footprints that leave the grid). This synchronises with the
 * plan's device counter. reset != 0 zeroes the counter afterwards.
 */
int grid_plan_skipped(grid_plan_t plan, int64_t* n_skipped, int reset);

/*
 * Status flags of the plan's calls since it was created or last reset (host
 * call; synchronises with the device word). No passage of the paper defines
 * it: it reports the bounded waits of the kernels that copy with the TMA
 * unit (the lazy-box gridder and the tile degridder).
 *   bit 0 (GRID_STATUS_COPY_TIMEOUT): a bulk copy into shared memory did not
 *   complete within the kernel's poll limit. The lazy gridder's team then
 *   skipped the rest of its chunk (the grid is incomplete); the tile
 *   degridder's warp wrote wrong values for that group and read the grid
 *   directly afterwards.
 * reset != 0 zeroes the flags afterwards. flags must not be NULL.
 */
enum { GRID_STATUS_COPY_TIMEOUT = 1 };
int grid_plan_status(grid_plan_t plan, unsigned* flags, int reset);

/*
 * Name of the kernel grid() launches for this plan (host call, no device
 * work): "chunked", "patch", "lazy", "sorted" (GRID_SCHED_SORTED, teams of at
 * most 32 threads) or "sorted-wide" (33..64 threads). The string is static;
 * NULL plan gives "".
 */
const char* grid_plan_gridder(grid_plan_t plan);

/*
 * Compression (Sec. 2.2, last paragraph, after Muscat): adjacent visibilities
 * that fall on the same point of the oversampled grid meet the same GCF
 * samples, so their weighted values can be added and gridded as one
 * visibility. The grid is unchanged up to FP32 rounding.
 *  - A run is a maximal sequence of consecutive visibilities (in the given
 *    order) whose fine positions floor(u*O + 1/2), floor(v*O + 1/2) are equal
 *    on both axes: the same cell and the same GCF sample row. A visibility
 *    whose coordinate is not finite or has |u*O| >= 2^26 (far off any
 *    supported grid) is a run of its own.
 *  - Run m gets uv_out[m] = uv of its first member and vis_out[m][p] = the sum
 *    over its members, in input order, of w_k * vis[k][p] (FP32). Grid the
 *    output with weights = NULL and an FP32 plan of the same G, S, O and
 *    npol: vis_out is complex64 whatever the plan's precision.
 *  - run_of[k] (optional, may be NULL) = the run holding visibility k.
 *  - *n_out = the number of runs, written on the stream (n_out is a DEVICE
 *    pointer to one int64; read it after the stream work completes).
 * Inputs as for grid(): uv [n][2] f64, vis [n][npol] in the plan precision,
 * weights [n] f32 or NULL. Outputs are caller-allocated device buffers with
 * room for n_vis runs: uv_out [n][2] f64 (16-byte aligned), vis_out [n][npol]
 * complex64, run_of [n] int64. The plan keeps a scratch buffer of about
 * n_vis/8 bytes, allocated on the first call that needs more (synchronous
 * cudaMalloc). Returns GRID_OK, GRID_ERR_INVALID, GRID_ERR_NOMEM or
 * GRID_ERR_CUDA.
 */
int grid_compress(grid_plan_t plan, int64_t n_vis, const double* uv, const void* vis, const float* weights,
                  double* uv_out, void* vis_out, int64_t* run_of, int64_t* n_out, cudaStream_t stream);

/*
 * One gridding and degridding pass from HOST buffers, with the transfers
 * overlapped with the kernels (a pipeline over chunks of `chunk`
 * visibilities; 0 = 1,048,576):
 *   - the grid is zeroed, chunk c of uv, values and weights is uploaded on a
 *     copy stream while chunk c-1 is gridded on `stream`;
 *   - the grid is copied down (if grid_host is not NULL) while the
 *     visibilities are degridded, and each degridded chunk is copied down
 *     while the next one is degridded.
 * gplan grids and dplan degrids; they must agree in G, S, oversample, npol
 * and precision (they may be the same plan).
 * HOST buffers (pinned, for the copies to overlap): uv_host [n][2] f64,
 * vis_host [n][npol] in the plan precision, weights_host [n] f32 or NULL,
 * vis_out_host [n][npol] complex64 (the degridded values, unweighted),
 * grid_host [npol][G][G] complex64 or NULL.
 * DEVICE buffers (caller-owned, room for n visibilities, aligned as for
 * grid()): uv_dev, vis_dev, weights_dev (needed when weights_host is given),
 * vis_out_dev, kernel_table, grid_dev (overwritten: zeroed, then gridded).
 * The work is ordered after earlier work on `stream`, and later work on
 * `stream` sees every output; the host outputs are complete once `stream`
 * reaches that point. The plan keeps a copy stream and events (created on
 * first use). Returns GRID_OK or a negative error code.
 */
int grid_degrid_host(grid_plan_t gplan, grid_plan_t dplan, int64_t n_vis, const double* uv_host, const void* vis_host,
                     const float* weights_host, double* uv_dev, void* vis_dev, float* weights_dev, void* vis_out_dev,
                     const void* kernel_table, void* grid_dev, void* vis_out_host, void* grid_host, int64_t chunk,
                     cudaStream_t stream);

/* One step of grid_degrid_host_steps: its pinned host inputs and outputs. */
typedef struct {
  const double* uv_host;    /* [n][2] f64 */
  const void* vis_host;     /* [n][npol], plan precision */
  const float* weights_host; /* [n] f32, or NULL (all steps alike) */
  void* vis_out_host;       /* [n][npol] complex64: degridded values (unweighted) */
  void* grid_host;          /* [npol][G][G] complex64, or NULL */
} grid_host_step;

/*
 * A sequence of n_steps passes of grid_degrid_host() (each: zero the grid,
 * grid the step's visibilities, degrid them), pipelined ACROSS steps: the
 * uploads of step s+1 run while step s degrids and downloads. Two device work
 * sets alternate between steps: uv_dev[2], vis_dev[2], weights_dev[2] (NULL
 * array when unweighted) and vis_out_dev[2], each with room for n
 * visibilities. Uploads go on one copy stream and downloads on another,
 * ordered by events; the grid is shared and rezeroed per step once the
 * previous step's grid went down. Every step has n visibilities. chunk as in
 * grid_degrid_host(), 0 = 4,194,304 here. n_steps in 0..64, at most 64
 * chunks per step. Ordering with `stream` as for grid_degrid_host(). Returns
 * GRID_OK or a negative error code.
 */
int grid_degrid_host_steps(grid_plan_t gplan, grid_plan_t dplan, int n_steps, const grid_host_step* steps,
                           int64_t n_vis, double* const* uv_dev, void* const* vis_dev, float* const* weights_dev,
                           void* const* vis_out_dev, const void* kernel_table, void* grid_dev, int64_t chunk,
                           cudaStream_t stream);

/*
 * Expansion after degridding compressed records: every member of a run has
 * the run's fine position, so its degridded value is the run's.
 *   vis_out[k][p] = w_k * vis_compressed[run_of[k]][p]   (w_k = 1 if weights is NULL)
 * run_of [n] int64 comes from grid_compress() on the same n visibilities;
 * vis_compressed is complex64 [n_compressed][npol] (for example from degrid()
 * on the compressed uv). A run index outside [0, n_compressed) gives 0.
 * OVERWRITES vis_out (complex64 [n][npol]). Device pointers; with even npol,
 * vis_compressed and vis_out must be 16-byte aligned.
 */
int degrid_expand(grid_plan_t plan, int64_t n_vis, const int64_t* run_of, int64_t n_compressed,
                  const void* vis_compressed, const float* weights, void* vis_out, cudaStream_t stream);

/*
 * Batched gridding: many grids of the same side
 * G, oversampling O and polarization count, for example every
 * (channel, w-plane) of an observation (Sec. 5 grids each w-slice with its
 * own kernel instance). Each item has its own visibilities, GCF support S
 * (<= max_S), kernel table and grid. One persistent kernel launch grids all
 * of them. Work units (runs of chunks of one item) are ordered by cost on
 * the host, and CTAs take them from an atomic counter. Every item uses the
 * gridding semantics of grid(), including accumulation into its grid.
 *
 * grid_batch_create(): a plan for the common parameters and the block shape
 *   (Bu, Bv). vis_per_chunk and threads may be 0 (defaults 256 and 256).
 * grid_batch_set(): uploads the item descriptors and the unit list
 *   (synchronous). `items` is a host array. The pointers inside it are device
 *   pointers, borrowed until the last execute using them has completed.
 * grid_batch_execute(): enqueues a counter reset and ONE kernel launch on
 *   `stream`. It allocates nothing and does not synchronise, so it can be
 *   captured in a CUDA graph and replayed.
 */
typedef struct grid_batch_s* grid_batch_t;

typedef struct {
  int64_t n_vis;
  const double* uv;          /* [n_vis][2] */
  const void* vis;           /* [n_vis][npol] complex, in the batch precision */
  const float* weights;      /* [n_vis] or NULL */
  const void* kernel_table;  /* [O][S] */
  void* grid;                /* [npol][G][G] complex64 */
  int S;
} grid_batch_item;

int grid_batch_create(grid_batch_t* out, int G, int oversample, int npol, int Bu, int Bv, int max_S, int precision,
                      int vis_per_chunk, int threads);

/*
 * As grid_batch_create(), with two block shapes: items with S >= S_split use
 * (Bu2, Bv2), the others (Bu, Bv). Larger supports favour larger blocks
 * (Sec. 5: the best coarsening depends on the bin size). Each shape has its
 * own persistent launch (back to back on the stream), compiled for that shape
 * alone, so either may be any built one-shape kernel: npol 1 with (1,1),
 * (2,1), (1,2), (2,2), (3,3), (4,2), (2,4), (4,4); npol 4 with (1,1), (2,1),
 * (2,2), (4,2). (Bu2, Bv2) equal to (Bu, Bv) gives one launch. S_split in
 * 0..64 (0: one shape).
 */
int grid_batch_create_ex(grid_batch_t* out, int G, int oversample, int npol, int Bu, int Bv, int Bu2, int Bv2,
                         int S_split, int max_S, int precision, int vis_per_chunk, int threads);
int grid_batch_set(grid_batch_t batch, int n_items, const grid_batch_item* items);
int grid_batch_execute(grid_batch_t batch, cudaStream_t stream);
int grid_batch_skipped(grid_batch_t batch, int64_t* n_skipped, int reset);
int grid_batch_describe(grid_batch_t batch, int* threads, int* n_units, int* ctas);
void grid_batch_destroy(grid_batch_t batch);
const char* grid_batch_last_error(void);

/*
 * Gridding without device allocation. The paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc:
 *  - a real-time pipeline that reserves all of its device memory at start-up
 *    and may not allocate while observing (an allocation can stall or fail
 *    part way through);
 *  - a host framework that owns the device heap through its own allocator,
 *    whose accounting a library allocating behind its back would break.
 * Such callers cannot create a plan, because grid_plan_create and the patch
 * schedule allocate scratch.
 *
 * grid_patch_static() takes the plan parameters directly and grids exactly
 * as grid() does with GRID_SCHED_PATCH and 64-visibility chunks. The other
 * arguments and the accumulate semantics are those of grid(), except that
 * skipped (invalid or off-grid) visibilities are not reported: there is no
 * plan to read a count from. Its binning scratch lives in one file-scope
 * device array of about 1.9 MB, which every GPU that loads the library holds
 * until the process exits.
 *  - Limits: at most 8,388,608 visibilities per call and at most 16,384 grid
 *    patches (patches are 32 cells at npol 4, 48 at npol 2, 96 at npol 1).
 *    A larger call returns GRID_ERR_INVALID with a message and queues
 *    nothing.
 *  - Allocation: it calls no cudaMalloc, no cudaFree and no allocating
 *    library routine; it only enqueues memsets and kernels on `stream`.
 *  - First call: the first call on each device looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current and keeps it for
 *    the life of the process. Make that first call before any stream capture.
 *    Do not use the entry point across cudaDeviceReset (the kept address
 *    would be stale).
 *  - Concurrency: all calls share the one array. Calls whose work overlaps
 *    on the GPU (other streams, other host threads) race and give wrong
 *    results; serialise them.
 * The message of the last error on the calling thread is in
 * grid_patch_static_last_error().
 */
int grid_patch_static(int G, int S, int oversample, int npol, int Bu, int Bv, int precision, int64_t n_vis,
                      const double* uv, const void* vis, const float* weights, const void* kernel_table, void* grid,
                      cudaStream_t stream);
const char* grid_patch_static_last_error(void);

/* Message of the last error on the calling thread ("" if none). */
const char* grid_last_error(void);

/* How the kernels for a Bu x Bv block and npol polarizations form the
 * products t_u[i] t_v[j] V_p of one visibility (the Sec. 6 remark on the
 * separable GCF), chosen at compile time per kernel as the form with the
 * fewest multiplications:
 *   GRID_TAPS_PRODUCT  (0): w_ij = t_u[i] t_v[j] first, then w_ij V_p;
 *   GRID_TAPS_FACTOR_V (1): Y_jp = t_v[j] V_p first, then t_u[i] Y_jp;
 *   GRID_TAPS_FACTOR_U (2): X_ip = t_u[i] V_p first, then t_v[j] X_ip.
 * *form receives the form and *multiplies the multiplications per visibility
 * per block, counted as in Sec. 6 (a real-by-complex product counts as one):
 * Bu*Bv + Bu*Bv*npol, Bv*npol + Bu*Bv*npol or Bu*npol + Bu*Bv*npol. Either
 * output may be null, not both. Host only (no device is touched). Returns
 * GRID_OK, GRID_ERR_INVALID (bad sizes, both outputs null) or
 * GRID_ERR_UNSUPPORTED (no kernel is built for the shape). */
enum { GRID_TAPS_PRODUCT = 0, GRID_TAPS_FACTOR_V = 1, GRID_TAPS_FACTOR_U = 2 };
int grid_tap_form(int Bu, int Bv, int npol, int* form, int* multiplies);

/* Peak FP32 FMA lanes per SM per clock (128 on sm_103) and the SM count of the current device. */
int grid_device_info(int* sm_count, int* fma_lanes_per_sm, int* max_clock_khz);

/*
 * Measured FP32 FMA throughput of the current device, the denominator of the
 * "% of FP32 FMA peak" figures (Sec. 5 quotes efficiency against the GPU's
 * FP32 peak; here the peak is measured rather than derived). Runs a kernel of
 * independent packed FMA chains (iters iterations of 8 FFMA2 per thread, 64
 * warps per SM) once to warm up and once timed with CUDA events on `stream`,
 * then synchronises. *tflops = 4 flop x FFMA2 lanes x instructions / time
 * (2 FMAs per FFMA2, 2 flop per FMA). iters 1 .. 2^24; a few thousand make a
 * launch of some milliseconds. Host call; allocates nothing on the device.
 */
int grid_measure_fma_peak(int iters, double* tflops, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_GRIDDER_H */
