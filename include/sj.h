/*
 * sj.h -- C ABI of the GB300 (sm_103a) spatial-join filter step.
 *
 * The library computes the filter step of the partitioning-based spatial
 * join (PBSM) studied in "Parallel In-Memory Evaluation of Spatial Joins"
 * (Tsitsigkos, Bouros, Mamoulis, Terrovitis): given two collections R and S
 * of axis-aligned rectangles (MBRs), it returns every pair (r, s) whose
 * rectangles have at least one common point (Sec. 1), each pair exactly once.
 *
 * Method (all steps run as CUDA kernels on the device):
 *   1. uniform nx x ny grid; each rectangle is assigned to every tile it
 *      overlaps (multi-assignment, Sec. 2.2), with the count -> prefix-sum ->
 *      write scheme of Sec. 3.4 steps 2-4;
 *   2. per tile, both sides are sorted by the lower x endpoint x_l
 *      (Algorithm 1, "sort"; Sec. 3.4 step 5);
 *   3. per tile, a forward-scan plane sweep (Algorithm 1) with a y-overlap
 *      test; a pair is reported only by the tile that holds the reference
 *      point (max x_l, max y_l) of the intersection (Eq. 1, Sec. 3.2).
 *
 * Conventions for every entry point:
 *  - Rectangle and pair pointers marked d_ are DEVICE pointers on the
 *    context's device; the caller owns them and keeps them alive until the
 *    context's stream has passed the call.  h_ pointers are host memory.
 *  - Rectangles are sj_rect (16 bytes, float32 xl, yl, xu, yu); d_R / d_S
 *    must be 16-byte aligned.  Valid input: every coordinate finite,
 *    xl <= xu, yl <= yu.  0 <= n <= SJ_MAX_N.
 *  - Intersection is closed: touching edges and corners count.  Comparisons
 *    are exact float32 compares (no arithmetic on coordinates other than the
 *    cell function), so the result does not depend on the grid.
 *  - Pair ids are 0-based indices into R and S.  Pair order is unspecified
 *    unless sj_opts.sort_output is set (then ascending by (r, s)).
 *  - All work is enqueued on the context's stream.  Calls that return a
 *    count to the host synchronise that stream once at the end (and the
 *    two-pass join once more, after counting, to size its output).
 *  - Status codes are returned; nothing aborts and no exception crosses the
 *    ABI.  sj_last_error() gives a message for the last failure.
 *  - A context is not thread-safe; use one context per host thread/stream.
 */
#ifndef SJ_H
#define SJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define SJ_OK         0
#define SJ_EINVAL     1   /* bad argument, NaN/Inf coordinate, xl > xu, size limit */
#define SJ_ENOMEM     2   /* an allocation failed                                 */
#define SJ_EOVERFLOW  3   /* caller-owned output too small (see sj_join_into)     */
#define SJ_ETIMEOUT   4   /* a bounded device-side wait gave up                   */
#define SJ_ECUDA      5   /* a CUDA runtime call failed                           */
#define SJ_EINTERNAL  6   /* an internal consistency check failed (in the debug
                             build also a failed bounds check; sj_last_error names
                             its source file and line)                           */

#define SJ_MAX_N      ((int64_t)1 << 30)   /* ids carry two flag bits above bit 29 */
#define SJ_MAX_TILES  ((int64_t)1 << 26)   /* nx * ny                               */

/* ---- plain data types ------------------------------------------------- */
typedef struct { float xl, yl, xu, yu; } sj_rect;       /* an MBR, Sec. 1        */
typedef struct { int32_t r, s; } sj_pair;               /* one result of J       */
typedef struct { float x, y; } sj_point;                /* a point (distance join) */

/* Uniform grid over [x0, x1] x [y0, y1] with nx columns and ny rows (Sec. 2.2;
 * ny = 1 gives vertical stripes, Sec. 3.1).  Tile (col, row) has index
 * row * nx + col.  A coordinate v falls in column
 *   clamp(floor((v - x0) * gx), 0, nx - 1),  gx = (float)nx / (x1 - x0),
 * with the subtraction and the product each rounded to float32; rows alike.
 * Rectangles outside the grid's extent land in the border tiles, so the
 * extent only shapes the partitioning, never the result. */
typedef struct { int32_t nx, ny; float x0, y0, x1, y1; } sj_grid;

/* Join modes. */
#define SJ_TWO_PASS      0   /* count pairs, allocate exactly, sweep again and write   */
#define SJ_ONE_PASS      1   /* sweep once into a buffer sized by the learned
                                per-tile predictor; exact two-pass rerun of the
                                chunks that do not fit.  A join that found more
                                pairs than its plan held scales the capacities of
                                later joins on the context by the shortfall (+10 %,
                                at most 8x; reset by sj_set_model)                     */
#define SJ_ONE_PASS_HEUR 2   /* as SJ_ONE_PASS, sized by the Eq. 2 histogram estimate  */
#define SJ_AUTO          3   /* SJ_ONE_PASS when a model is loaded, else SJ_TWO_PASS   */

/* Option flags (sj_opts.flags). */
#define SJ_SWEEP_ADAPTIVE 1  /* choose the sweep axis of every tile from the Eq. 2
                                histograms of Sec. 3.3: the axis with the smaller
                                estimate of intersecting projections (k = 8 buckets
                                per tile axis, built from all of the tile's
                                entries); without it every tile is swept along x
                                (Algorithm 1).  Two-level path (single joins and
                                batches); the single-level path (tiles beyond
                                shared memory) sweeps along x.  The pairs are
                                the same either way.  See sj_tile_axes.          */
#define SJ_DEDUP_GBDA     2  /* grouping-based duplicate avoidance instead of the
                                reference-point test of Eq. 1: the entries of a
                                tile are grouped in four classes by where their
                                projections begin (A: in the tile on x and y,
                                B: on x only, C: on y only, D: neither), and
                                only the 9 class pairs that can report a pair
                                in this tile are joined (A with any, any with A,
                                B with C, C with B), with no test per pair.  The
                                pairs are the same.  Two-level path (single
                                joins and batches); the single-level path uses
                                Eq. 1.  Not combinable with SJ_SWEEP_ADAPTIVE.  */

typedef struct {
    int32_t mode;         /* one of the modes above                          */
    int32_t sort_output;  /* nonzero: pairs ascending by (r, s)              */
    float   margin;       /* one-pass capacity = predicted * (1 + margin) + slack */
    int32_t flags;        /* SJ_SWEEP_ADAPTIVE, SJ_DEDUP_GBDA or 0           */
} sj_opts;

typedef struct sj_ctx sj_ctx;     /* device, stream, allocator, workspace    */
typedef struct sj_part sj_part;   /* a partitioned (R, S, grid)              */

/* Optional allocator for every device buffer the library obtains (workspace
 * and result buffers).  alloc returns a device pointer aligned to 256 bytes
 * or NULL; free releases one.  Default: cudaMallocAsync / cudaFreeAsync on
 * the context's stream. */
typedef void *(*sj_alloc_fn)(size_t bytes, void *user);
typedef void (*sj_free_fn)(void *ptr, void *user);

/* ---- context ---------------------------------------------------------- */
/* Create a context on `device` issuing all work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Returns SJ_EINVAL for a bad device, SJ_ECUDA / SJ_ENOMEM.
 * Environment variables read here, for measurements only (the results are
 * the same either way): SJ_L1_WRITE=private (per-CTA L1 write ranges),
 * SJ_BLOCK_TARGET=n (entries per block of the two-level plan),
 * SJ_STRIPES=0 (1D grids take the general path), SJ_BATCH_GRAPHS=0 (batches
 * launch directly), SJ_BATCH_COUNT=global (batch count by global atomics). */
int sj_create(sj_ctx **out, int device, void *cuda_stream);

/* Release the context and its workspace (synchronises its stream). */
int sj_destroy(sj_ctx *ctx);

/* Install (alloc, free, user) as the context's allocator; both NULL restores
 * the default.  Frees the current workspace. */
int sj_set_allocator(sj_ctx *ctx, sj_alloc_fn alloc, sj_free_fn free_fn, void *user);

/* Free a buffer the library returned (a pair buffer of sj_join). */
void sj_free(sj_ctx *ctx, void *d_ptr);

/* Message of the last failure on this context ("" if none); static text for
 * a status code. */
const char *sj_last_error(sj_ctx *ctx);
const char *sj_strerror(int status);

/* ---- partitioning (Sec. 3.4 steps 2-4) -------------------------------- */
/* Partition R and S on grid *g: per-tile counts, exclusive prefix sums and
 * the replicated entries of every tile, contiguous per tile.  *out receives
 * a handle that owns that device state; reuse it with sj_part_join and
 * release it with sj_part_free.  Synchronises once (to size the entries).
 * Errors: SJ_EINVAL (arguments or invalid rectangles), SJ_ENOMEM. */
int sj_partition(sj_ctx *ctx, const sj_rect *d_R, int64_t nR,
                 const sj_rect *d_S, int64_t nS, const sj_grid *g, sj_part **out);

/* Per-tile state of a partition, for inspection (all device pointers owned
 * by the partition, valid until sj_part_free):
 *   off    : uint32[2 * (T + 1)], (R offset, S offset) per tile, exclusive
 *            prefix sums of the per-tile counts; off[2T], off[2T+1] = E_R, E_S
 *   ent_r  : float4[E_R] the replicated R rectangles, grouped by tile
 *   id_r   : uint32[E_R] original index | 1<<30 if the tile is the first
 *            column the rectangle covers | 1<<31 if it is the first row
 *   ent_s, id_s : the same for S
 * Order inside a tile's segment is unspecified.  T = nx * ny. */
typedef struct {
    int64_t n_tiles, e_r, e_s;
    const void *off, *ent_r, *id_r, *ent_s, *id_s;
} sj_part_view;
int sj_part_view_get(const sj_part *p, sj_part_view *out);

/* Join a partition (steps 5-6 and Eq. 1).  Same output contract as sj_join. */
int sj_part_join(sj_ctx *ctx, sj_part *p, const sj_opts *o,
                 sj_pair **d_pairs, int64_t *npairs);

void sj_part_free(sj_part *p);

/* ---- joins -------------------------------------------------------------- */
/* Exact number of result pairs of R join S on grid *g, without writing
 * pairs (partition + sort + sweep in count mode).  *out_npairs on host. */
int sj_count(sj_ctx *ctx, const sj_rect *d_R, int64_t nR,
             const sj_rect *d_S, int64_t nS, const sj_grid *g, int64_t *out_npairs);

/* Full filter step.  On SJ_OK, *d_pairs receives a device buffer holding
 * *npairs sj_pair (allocated with the context's allocator; release it with
 * sj_free, or through the installed allocator's owner), or NULL when
 * *npairs == 0.  o may be NULL (two-pass, unsorted). */
int sj_join(sj_ctx *ctx, const sj_rect *d_R, int64_t nR,
            const sj_rect *d_S, int64_t nS, const sj_grid *g, const sj_opts *o,
            sj_pair **d_pairs, int64_t *npairs);

/* As sj_join but writing into a caller-owned device buffer of `cap` pairs.
 * If the result does not fit, nothing beyond cap is written, *npairs gets
 * the required count and SJ_EOVERFLOW is returned. */
int sj_join_into(sj_ctx *ctx, const sj_rect *d_R, int64_t nR,
                 const sj_rect *d_S, int64_t nS, const sj_grid *g, const sj_opts *o,
                 sj_pair *d_buf, int64_t cap, int64_t *npairs);

/* Per-tile statistics of a join on grid *g (device outputs, caller-owned,
 * each nx*ny long; any may be NULL): replicated entries per side and the
 * exact number of pairs each tile reports.  Used to train and evaluate the
 * per-tile result-count predictor.  Synchronises once. */
int sj_tile_stats(sj_ctx *ctx, const sj_rect *d_R, int64_t nR,
                  const sj_rect *d_S, int64_t nS, const sj_grid *g,
                  uint32_t *d_cnt_r, uint32_t *d_cnt_s, uint32_t *d_pairs_per_tile);

/* ---- one band of tile rows (several GPUs on one join) ------------------- */
/* The pairs of R join S on grid *g whose reference point (Eq. 1) lies in
 * tile rows [row0, row1) (0 <= row0 <= row1 <= ny).  The tiles are
 * independent tasks and every pair is reported by exactly one tile (Sec. 1,
 * Sec. 3.2), so bands that cover the rows once give disjoint pair sets whose
 * union is the join: one GPU per band joins one input without exchanging
 * pairs.  Only the rectangles that overlap the band's rows take part (the
 * call selects them); a caller that stages only those rectangles on a GPU
 * gets the same pairs in the indices of what it passed.  Ids are indices
 * into d_R / d_S as given.  Output contract as sj_join / sj_join_into (pair
 * order unspecified unless sort_output; SJ_EOVERFLOW with the required count
 * for a too small buffer).  Synchronises twice (band sizes, pair count).
 * SJ_EINVAL for a band outside the grid. */
int sj_join_rows(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                 const sj_grid *g, int32_t row0, int32_t row1, const sj_opts *o,
                 sj_pair **d_pairs, int64_t *npairs);
int sj_join_rows_into(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                      const sj_grid *g, int32_t row0, int32_t row1, const sj_opts *o,
                      sj_pair *d_buf, int64_t cap, int64_t *npairs);

/* The sweep axis SJ_SWEEP_ADAPTIVE gives every tile of a join on grid *g
 * (Sec. 3.3, Eq. 2 with k = 8 divisions per tile axis): d_axis is a
 * caller-owned device uint8[nx * ny], row-major; 1 = swept along y, 0 = x
 * (also for tiles holding no entry of one side).  Runs the partition and the
 * count pass of the two-level path.  SJ_EINVAL when the grid or the data need
 * the single-level path (which sweeps every tile along x).  Synchronises
 * once. */
int sj_tile_axes(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                 const sj_grid *g, uint8_t *d_axis);

/* ---- host buffers ------------------------------------------------------ */
/* sj_join for HOST arrays: copies R and S to the device (into the context's
 * workspace), joins them, and copies the pairs back into h_out (cap pairs).
 * If the result has more than cap pairs, *npairs gets the required count
 * and SJ_EOVERFLOW is returned (h_out untouched).  Page-locked host memory
 * makes the copies asynchronous.  Synchronises the context's stream. */
int sj_join_host(sj_ctx *ctx, const sj_rect *h_R, int64_t nR, const sj_rect *h_S, int64_t nS,
                 const sj_grid *g, const sj_opts *o, sj_pair *h_out, int64_t cap,
                 int64_t *npairs);

/* A sequence of n independent joins from HOST buffers (the serving case: a
 * stream of host-resident requests).  Join i is R_i join S_i on grid g[i]
 * with options o, exactly as sj_join_host; the difference is the schedule:
 * the host -> device copy of join i+1's inputs runs on a second (copy)
 * stream, into the other of two device staging buffers, while join i runs,
 * so each join costs about max(copy, join) instead of copy + join.
 *   h_R[i], h_S[i], nR[i], nS[i] : host rectangles (page-locked memory makes
 *       the copies asynchronous; pageable memory works but does not overlap)
 *   g : n grids;  o : options for every join (may be NULL)
 *   h_out[i], cap[i] : host output of join i, cap[i] pairs
 *   npairs : host, n values: the pairs of each join (also on SJ_EOVERFLOW)
 * Every argument is checked before any work.  If a join has more pairs than
 * its cap, its output is left untouched, the other joins complete, and
 * SJ_EOVERFLOW is returned.  The staging buffers (16 bytes per rectangle,
 * twice) and the copy stream belong to the context until sj_destroy.
 * Synchronises the context's stream (inside each join, as sj_join_host)
 * and both streams at the end. */
int sj_join_host_many(sj_ctx *ctx, int n, const sj_rect *const *h_R, const int64_t *nR,
                      const sj_rect *const *h_S, const int64_t *nS, const sj_grid *g, const sj_opts *o,
                      sj_pair *const *h_out, const int64_t *cap, int64_t *npairs);

/* ---- tuning ------------------------------------------------------------------ */
/* Sums of the widths and heights of R and S (device inputs; host out[4] =
 * sum w_R, sum h_R, sum w_S, sum h_S, float64): the statistics behind the
 * grid rule of Sec. 4.3 (tile extent about ten times the average extent). */
int sj_extent_stats(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                    double *out);
/* Entries per block of the two-level partition (default 1536, >= 64): the
 * knob the autotuner sets next to the grid. */
int sj_set_tuning(sj_ctx *ctx, int block_target);
/* Order in which the one-pass join's persistent block-join CTAs take the
 * blocks: heaviest predicted cost first (entries + predicted pairs, 32 log2
 * classes; the default, 1) or block order (0).  The pairs are the same; only
 * the balance of the CTAs changes. */
int sj_set_schedule(sj_ctx *ctx, int heaviest_first);

/* ---- batches of independent joins ---------------------------------------- */
/* nj independent joins (R_j join S_j on grid g[j]) in one pass of the
 * two-level kernels: one count, one scan, one write and one persistent
 * block-join launch over the blocks of all joins (each join keeps its own
 * grid and blocks), captured into CUDA graphs that are replayed while the
 * arguments do not change (work runs on an internal stream ordered after the
 * context's stream; the context's stream waits for the result).
 *   d_R[j], d_S[j], nR[j], nS[j] : device inputs as for sj_join (1 <= nj <= 4096)
 *   g : nj grids, or NULL = per join, tiles about ten times the average
 *       rectangle extent (the rule of Sec. 4.3) over the unit square
 *   d_out, cap : caller-owned device buffer of cap pairs; the pairs of join j
 *       are d_out[h_offsets[j] .. h_offsets[j+1]) (ids local to the join)
 *   h_offsets : host, nj + 1 values (also filled on SJ_EOVERFLOW, which is
 *       returned when cap < h_offsets[nj]; nothing is written then)
 * Modes (o->mode): SJ_TWO_PASS (default) is the exact two-pass join in
 * graphs and synchronises once after counting.  SJ_ONE_PASS (with a model
 * set by sj_set_model), SJ_ONE_PASS_HEUR and SJ_AUTO size the whole batch in
 * one pass: the Eq. 2 sample of every join's blocks, the predicted pairs per
 * block, one capacity for all blocks (heaviest first, see sj_set_schedule),
 * one reserve-and-write block-join launch into the context's workspace, an
 * exact re-run of the blocks that did not fit, and a regroup of every block's
 * pairs into its join's range; direct launches, two synchronisations (the
 * capacity, the offsets).  The pairs are the same in every mode.
 * With o->sort_output every join's range is sorted by (r, s) after the join
 * (one device sort of the whole buffer with every join's r shifted past the
 * joins before it; the R inputs must total fewer than 2^32 rectangles, else
 * SJ_EINVAL); o->flags (adaptive axis, GBDA) apply to every join of the batch.
 * Joins whose tiles exceed shared memory fall back to sj_join_into each
 * (exact two-pass). */
int sj_join_batch(sj_ctx *ctx, int nj, const sj_rect *const *d_R, const int64_t *nR,
                  const sj_rect *const *d_S, const int64_t *nS, const sj_grid *g, const sj_opts *o,
                  sj_pair *d_out, int64_t cap, int64_t *h_offsets);

/* ---- learned per-block result-count predictor ---------------------------- */
/* The one-pass join (SJ_ONE_PASS) sizes its output from predicted result
 * counts.  The unit of prediction is a block of the two-level partition
 * (G x G tiles, about 1.5k entries; sj_last_stats().block_side).  Its 32
 * features are the Eq. 2 histograms of Sec. 3.3 with k = 8 buckets: for R
 * and S, the x and y projections of a sample (one rectangle of every 16 of
 * each side, cf. the sampling of Sec. 3.3) counted per bucket of the block's
 * extent, scaled to the block's exact entry count, then log1p.  Layout of a
 * feature row: [R x (8) | R y (8) | S x (8) | S y (8)].
 * The model: 32 -> 64 ReLU -> 64 ReLU -> 1 (predicted log1p of the block's
 * pairs), bf16 weights, fp32 accumulation.  Parameter vector (fp32,
 * SJ_MLP_PARAMS): W1[64][32], b1[64], W2[64][64], b2[64], W3[64], b3. */
#define SJ_MLP_FEATURES 32
#define SJ_MLP_PARAMS   6337
typedef struct sj_mlp sj_mlp;

/* Create a model on the context's device (parameters zero; set them with
 * sj_mlp_set_params).  Release with sj_mlp_free (before its context). */
int  sj_mlp_create(sj_ctx *ctx, sj_mlp **out);
void sj_mlp_free(sj_mlp *m);
/* Host fp32 parameter vector -> model (resets the Adam state). */
int  sj_mlp_set_params(sj_ctx *ctx, sj_mlp *m, const float *h_params);
/* Model -> host: fp32 master parameters, and (if h_inference != NULL) the
 * values inference uses (weights rounded to bf16, as fp32).  Synchronises. */
int  sj_mlp_get_params(sj_ctx *ctx, const sj_mlp *m, float *h_params, float *h_inference);
/* d_y[i] = model(d_X[i]) for n rows of SJ_MLP_FEATURES floats (device; d_X
 * 16-byte aligned, else SJ_EINVAL).  Sums in fp32 in a fixed order: the same
 * bits as the forward pass of sj_mlp_grad. */
int  sj_mlp_forward(sj_ctx *ctx, const sj_mlp *m, const float *d_X, int64_t n, float *d_y);
/* Gradient of the mean squared error of the n rows (device d_X, d_Y) with
 * respect to the parameters as inference uses them: d_grad (SJ_MLP_PARAMS
 * floats, overwritten) and the loss in d_loss[0] (overwritten). */
int  sj_mlp_grad(sj_ctx *ctx, const sj_mlp *m, const float *d_X, const float *d_Y, int64_t n,
                 float *d_grad, float *d_loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on a batch;
 * the batch loss goes to d_loss[0] when d_loss != NULL. */
int  sj_mlp_train_step(sj_ctx *ctx, sj_mlp *m, const float *d_X, const float *d_Y, int64_t n,
                       float lr, float *d_loss);
/* Features and exact labels (log1p of the pairs each block reports) of every
 * block that holds both R and S entries, for a join on grid *g: d_feat
 * (cap x SJ_MLP_FEATURES floats), d_label (cap floats) and, if not NULL,
 * d_block (cap int32: block index by * blocks_x + bx), all caller-owned
 * device buffers, rows in an unspecified order.  *n_items receives the
 * number of blocks (also on SJ_EOVERFLOW when cap is too small).  SJ_EINVAL
 * if the grid or the data do not suit the two-level path. */
int  sj_block_features(sj_ctx *ctx, const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                       const sj_grid *g, float *d_feat, float *d_label, int32_t *d_block, int64_t cap,
                       int64_t *n_items);
/* Use model m (kept by pointer; NULL = none) for SJ_ONE_PASS / SJ_AUTO. */
int  sj_set_model(sj_ctx *ctx, const sj_mlp *m);

/* ---- statistics of the last join ------------------------------------------ */
/* Counters of the last join / count on this context (host copy; valid after
 * the call returned SJ_OK).  path: 1 = two-level (blocked) partitioning,
 * 0 = single-level, 2 = stripes (a 1D grid joined stripe by stripe in
 * shared memory, swept along the stripe; blocks = stripes).  For the two-level path, l1_entries_* are the entries
 * written to the coarse blocks (a rectangle is copied into every block it
 * overlaps) and blocks / block_side describe the coarse grid; the per-tile
 * segments of the method then exist only in shared memory.  For the
 * single-level path, entries_* are the replicated per-tile entries. */
typedef struct {
    int32_t path;
    int32_t block_side;          /* tiles per block side (two-level)        */
    int64_t blocks;              /* blocks of the coarse grid               */
    int64_t work_items;          /* blocks holding both R and S entries     */
    int64_t l1_entries_r, l1_entries_s;
    int64_t entries_r, entries_s;
    int64_t npairs;
    int32_t one_pass;            /* 1 if the last join ran one-pass          */
    int32_t dedup;               /* 1 if the two-level join used GBDA, 0: Eq. 1 */
    int64_t capacity;            /* one-pass: pairs the output was sized for */
    int64_t refit_items;         /* one-pass: blocks re-run because they did not fit */
    int64_t y_sweep_tiles;       /* SJ_SWEEP_ADAPTIVE: tiles swept along y    */
} sj_stats;
int sj_last_stats(sj_ctx *ctx, sj_stats *out);

/* ---- device-side timing ------------------------------------------------- */
/* When enabled, every phase of every join is bracketed by CUDA events on the
 * context's stream; sj_timing_read synchronises the stream and returns the
 * summed device time of each phase since the last enable/read, with the
 * number of kernel launches.  Phase names: sj_timing_phase_name(i). */
#define SJ_NPHASE 13
typedef struct {
    int64_t launches;        /* kernels of this library launched (all phases)  */
    int64_t n[SJ_NPHASE];    /* timed occurrences of each phase                 */
    double ms[SJ_NPHASE];    /* summed device milliseconds of each phase        */
} sj_timing;
int sj_timing_enable(sj_ctx *ctx, int on);
int sj_timing_read(sj_ctx *ctx, sj_timing *out);
const char *sj_timing_phase_name(int phase);

/* ---- eps-distance join on point sets (Sec. 1) ------------------------------- */
/* All pairs (i, j) with Euclidean distance |P[i] - Q[j]| <= eps.  The paper
 * (Sec. 1) answers this query with the intersection join: every point is
 * replaced by a square of side eps centred on it, the squares are joined,
 * and every intersecting pair is refined by its distance.  Here:
 *   - the squares are built on the device with half-width eps * (1/2 +
 *     2^-21) rounded up and corners rounded outward, so each holds the exact
 *     square of side eps and no pair can be lost to rounding;
 *   - the squares are joined on grid *g in mode o (as sj_join: the two-level
 *     or single-level path, two-pass or one-pass), giving the candidates;
 *   - the distance test runs in IEEE binary64 in a fixed order: dx = x_p -
 *     x_q, dy = y_p - y_q, d2 = dx*dx + dy*dy, each operation rounded once
 *     (no fused multiply-add), accepted when d2 <= (double)eps * (double)eps.
 *     The decision is therefore a fixed function of the float32 inputs.
 *   d_P, d_Q : device sj_point arrays (8 bytes each, 8-byte aligned), caller-
 *       owned; 0 <= n < SJ_MAX_N.  Coordinates must be finite, and the
 *       square corners must stay finite (else SJ_EINVAL from the join).
 *   eps : 0 <= eps <= 1e18 (eps = 0 keeps coincident points only).
 *   g, o : the grid of the squares and the join options, as for sj_join.
 *   d_pairs / npairs : as for sj_join (exact-size buffer from the context's
 *       allocator, release with sj_free; NULL when there is no pair).
 *   ncand : if not NULL, receives the number of intersecting square pairs
 *       (the candidates the distance test examined).
 * Workspace: 16 bytes per point for the squares, 8 bytes per candidate, and
 * a bit per candidate.  Synchronises the stream after the candidate join
 * (as sj_join) and once more to size the output.  Pair order: ascending
 * candidate order of the filter (unspecified unless o->sort_output). */
int sj_distance_join(sj_ctx *ctx, const sj_point *d_P, int64_t nP, const sj_point *d_Q, int64_t nQ,
                     float eps, const sj_grid *g, const sj_opts *o, sj_pair **d_pairs, int64_t *npairs,
                     int64_t *ncand);

/* As sj_distance_join, writing into a caller-owned device buffer of cap
 * pairs; SJ_EOVERFLOW (with *npairs = the required count, nothing written)
 * when it is too small. */
int sj_distance_join_into(sj_ctx *ctx, const sj_point *d_P, int64_t nP, const sj_point *d_Q, int64_t nQ,
                          float eps, const sj_grid *g, const sj_opts *o, sj_pair *d_buf, int64_t cap,
                          int64_t *npairs, int64_t *ncand);

/* ---- a join that allocates nothing --------------------------------------- */
/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: plug-ins whose host process owns every
 * device allocation (a fixed budget or a custom pool that nothing may
 * bypass), and callers on a latency-critical path that cannot afford an
 * allocation's latency or the device-wide synchronisation of cudaFree.
 *
 * Same result as sj_join_into (two-pass, exact), but every scratch buffer is
 * carved from one fixed device array of 20 MiB inside this library.  Every
 * GPU on which the library is used holds that array until the process
 * exits.  No cudaMalloc, cudaFree or allocating library call is made.
 *   d_R, d_S  : device rectangles as for sj_join (16-byte aligned)
 *   g         : the grid; nx * ny <= 65536
 *   d_out/cap : caller-owned device buffer of cap pairs
 *   npairs    : host; receives the number of pairs (also on SJ_EOVERFLOW)
 *   cuda_stream : the stream to use (cudaStream_t, NULL = legacy default)
 * Limits: nR, nS <= 65536 and at most 131072 replicated entries per side;
 * beyond them SJ_EINVAL (sizes are checked first, the entry count on the
 * device, in which case nothing is written).  If cap is too small, *npairs
 * gets the required count and SJ_EOVERFLOW is returned.  SJ_ETIMEOUT if a
 * bounded device-side wait gave up, SJ_EINTERNAL for an internal table
 * overflow, SJ_ECUDA for a failed runtime call.
 * Uses the current device.  The first call on a device resolves the array's
 * address (cudaGetSymbolAddress) and the launch parameters: make that first
 * call before any stream capture.  Calls share the array: two calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race and corrupt each other; serialise them.  Each call clears the
 * counters it needs, so stale contents of an earlier call do no harm.
 * The call waits for the stream once, after the count pass (it reads the
 * pair count back into host memory); the pairs are written asynchronously
 * afterwards.  Status codes only (no sj_last_error). */
int sj_join_noalloc(const sj_rect *d_R, int64_t nR, const sj_rect *d_S, int64_t nS,
                    const sj_grid *g, sj_pair *d_out, int64_t cap, int64_t *npairs,
                    void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SJ_H */
