/*
 * spid.h -- C ABI of the GB300 (sm_103a) sketched column interpolative
 * decomposition library (libspid.so).
 *
 * The method (arXiv 2103.01380, Pacella, Dunton, Doostan, Iaccarino):
 *   a data matrix A (m x n; rows = grid points x QoIs, columns = time
 *   snapshots, Section 2) is compressed per spatial subdomain as
 *   A ~ A(:,J) C.  A Gaussian sketch Y = Omega A (Omega l x m i.i.d. N(0,1),
 *   l = k_max + p; Section 2, random projection) is accumulated as snapshot
 *   columns arrive; a column-pivoted QR of Y picks the k skeleton columns J
 *   (Section 2, A Z = Q R, Algorithm 1 step 3; adaptive rank per Remark 2.1)
 *   and C = [I_k | R11^-1 R12] Z^T (Section 2, Eq. for C; Algorithms 1-2).
 *   Subdomains are independent (Section 3.2) and are processed as one batch.
 *
 * Conventions shared by every entry point:
 *   - Window layout ("blocks"): subdomain s is an m[s] x n[s] column-major
 *     matrix (column j = snapshot j, contiguous rows) that starts at element
 *     off[s] of one device buffer and has leading dimension ld[s] elements.
 *     This covers both subdomain-major ([s][j][r]) and snapshot-major
 *     ([j][s][r]) windows.  Elements are double for SPID_PREC_FP64 and float
 *     otherwise.  off[s] and ld[s] must be multiples of 16 bytes / element
 *     size, and the window base must be 16-byte aligned (checked).
 *   - Window layout ("boxes", spid_box_layout): the window is the solver's
 *     own global field, [t][q][Z][Y][X] (snapshot t of QoI q at grid point
 *     (x, y, z)), and each subdomain is a box of it (Algorithm 6 saves the
 *     data of each block of the domain; Section 3.2 blocks the domain into
 *     sub-domains), either with all QoIs stacked or one QoI per subdomain
 *     (Section 5.3: each QoI of each sub-domain compressed on its own).
 *   - Omega(i, r), i < l, r < m, is never stored.  It is the Box-Muller
 *     transform of Philox4x32-10 (Salmon et al., SC'11) with key =
 *     (seed & 0xffffffff, seed >> 32) and counter = (r, i / 4, 0, 0); words
 *     (x0, x1) give rows 4g, 4g+1 and (x2, x3) rows 4g+2, 4g+3 of group
 *     g = i / 4, with u = (x + 0.5) 2^-32, g0 = sqrt(-2 ln ua) cos(2 pi ub),
 *     g1 = sqrt(-2 ln ua) sin(2 pi ub).  The same Omega serves every
 *     subdomain (subdomain s uses its first m[s] columns).
 *   - Pointers named *_host are host memory; *_dev and window/out are device
 *     memory.  The caller owns the window and every output buffer; the plan
 *     owns its workspace (sketch Y, partial sums, factors, status word).
 *   - Every call that takes a stream is asynchronous on that stream unless
 *     stated otherwise.  A plan must be used from one stream at a time.
 *   - Argument errors are returned synchronously and launch nothing.  Errors
 *     found on the device (non-finite sketch, a bounded wait that timed out)
 *     set a sticky status word read by spid_device_status().  No call ever
 *     traps or aborts the process.
 */
#ifndef SPID_H
#define SPID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st* spid_stream_t;

typedef struct spid_plan_s* spid_plan_t;

typedef enum {
  SPID_OK = 0,
  SPID_ERR_INVALID_ARG = 1,  /* a size, pointer, alignment or mode is invalid */
  SPID_ERR_CUDA = 2,         /* a CUDA runtime call failed (spid_last_error() says which) */
  SPID_ERR_OOM = 3,          /* device allocation failed in spid_plan_create */
  SPID_ERR_STATE = 4,        /* call out of order (e.g. factors before finalize) */
  SPID_ERR_TIMEOUT = 5,      /* a bounded device wait gave up (device status) */
  SPID_ERR_NONFINITE = 6,    /* NaN/Inf reached the sketch of some subdomain (device status) */
  SPID_ERR_UNSUPPORTED = 7,  /* valid request this library does not implement */
  SPID_ERR_RANK = 8          /* informational, from spid_device_status only: the rank guard
                                stopped some subdomain's factorization before its target (k_max
                                pivots, or the tolerance); its factors are valid, with the
                                smaller k that spid_get_factors reports */
} spid_status;

/* Every FP32-window mode factors the sketch with FP32 Householder reflectors,
 * pivot norms held as FP32 pairs (hi + lo, ~48-bit significand, exact
 * argmax) and a pair-precision back-substitution: FP64-class accuracy without
 * GB300's 1:64-rate FP64 pipe.  The unit roundoff u of each mode sets its rank
 * guard |R_jj| > 2 u |R_00|. */
typedef enum {
  SPID_PREC_FP64 = 0,   /* FP64 window; sketch, QR, solve and error in FP64 (SIMT); u = 2^-53 */
  SPID_PREC_FP32 = 1,   /* FP32 window; FP32 SIMT sketch; u = 2^-24 */
  SPID_PREC_TF32 = 2,   /* FP32 window; tcgen05 TF32 sketch (FP32 accumulate in TMEM, tiles
                           staged by TMA); u = 2^-11 */
  SPID_PREC_BF16 = 3,   /* FP32 window; tcgen05 BF16 sketch (A and Omega rounded to BF16,
                           FP32 accumulate); u = 2^-9 */
  SPID_PREC_BF16X3 = 4  /* FP32 window; tcgen05 3xBF16 sketch (two-term BF16 splits of A and
                           Omega, three products, FP32 accumulate); u = 2^-16 */
} spid_precision;

/* Plain (unbatched) form: one kernel launch per subdomain per stage. */
#define SPID_FLAG_PER_SUBDOMAIN 1u
/* Error pass / reconstruction with the rank-k product on the tensor cores
 * (TF32, BF16 and 3xBF16 plans, batched, k_max <= 32; ignored otherwise). */
#define SPID_FLAG_TC_ERROR 2u

/* Boxes of the solver's global field as subdomains.  The window pointer is
 * element (t, q, z, y, x) = (0, 0, 0, 0, 0) of [t][q][Z][Y][X]: snapshot t of
 * QoI q at grid point (x, y, z) is element t snap_stride + ((q Z + z) Y + y) X
 * + x.  Box b covers the points org + [0, ext).  Its data matrix (Section 2:
 * rows = grid points x QoIs, columns = snapshots) has rows
 * r = ((q ez + z) ey + y) ex + x, QoI slowest, so m = nq ex ey ez (split_qoi
 * = 0), or, with split_qoi = 1, QoI q of box b is subdomain b nq + q with rows
 * r = (z ey + y) ex + x and m = ex ey ez.  The tensor-core sketches read each
 * box by TMA as 5-D tiles and need ex to be a multiple of 32
 * (SPID_ERR_UNSUPPORTED otherwise); the CUDA-core kernels take any ex that is
 * a multiple of 4 elements (16 bytes; 2 for FP64).  Boxes may overlap; they
 * do not wrap around the field's edges. */
typedef struct {
  int32_t nq;              /* QoIs per grid point, >= 1 */
  int64_t X, Y, Z;         /* global grid extents, each >= 1; X a multiple of 16 bytes / element
                              size */
  int64_t snap_stride;     /* elements from one snapshot to the next, >= nq X Y Z, a multiple of
                              16 bytes / element size */
  int32_t num_box;         /* B >= 1 */
  const int32_t* org3;     /* host [3 B]: (x, y, z) of box b's first point; x a multiple of 16
                              bytes / element size */
  const int32_t* ext3;     /* host [3 B]: (ex, ey, ez) >= 1, ex a multiple of 16 bytes / element
                              size; org + ext <= (X, Y, Z) */
  int32_t split_qoi;       /* 0 or 1, as above */
} spid_box_layout;

typedef struct {
  int32_t num_sub;        /* number of subdomains S >= 1 (boxes: B, or B nq with split_qoi) */
  const int32_t* m;       /* host [S]: rows m_s >= 1 (ignored with boxes; may be NULL) */
  const int32_t* n;       /* host [S]: window length n_s >= 1 (columns) */
  const int64_t* off;     /* host [S]: element offset of A_s(0,0) in the window (ignored with
                             boxes; may be NULL) */
  const int64_t* ld;      /* host [S]: leading dimension (elements), >= m_s (ignored with
                             boxes; may be NULL) */
  int32_t k_max;          /* maximum rank, 1 <= k_max; k_s <= min(k_max, n_s) */
  int32_t p;              /* oversampling, p >= 0; l = k_max + p <= 64 */
  double tol;             /* 0: fixed rank k_max.  > 0: smallest k with
                             ||R22||_F <= tol ||Y||_F (Remark 2.1 reading) */
  int32_t precision;      /* spid_precision */
  uint32_t flags;         /* SPID_FLAG_* */
  uint64_t seed;          /* Omega key */
  const int32_t* qoi;     /* host [S] or NULL: the QoI that subdomain s holds, 0 <= qoi[s] <
                             num_qoi, for per-QoI error totals (Section 5.1 reports each QoI's
                             error); with boxes and split_qoi = 1, NULL means qoi[s] = s % nq */
  int32_t num_qoi;        /* 0 (no per-QoI totals) .. 64; with boxes and split_qoi = 1 and
                             qoi == NULL, 0 means nq */
  const spid_box_layout* boxes;   /* NULL: the blocks layout (m, off, ld); else the boxes
                                     layout (copied at creation) */
} spid_plan_desc;

/* Create a plan: validates the descriptor and allocates ALL device
 * workspace (later calls allocate nothing).  Rows m_s up to 2^31-1, columns
 * up to 2^20 per subdomain.  Returns SPID_ERR_OOM if device memory runs out.
 * The plan is bound to the current CUDA device.  The workspace is cleared and
 * the descriptor tables uploaded on `stream`, which is then synchronized (the
 * plan is ready for any stream on return). */
spid_status spid_plan_create(const spid_plan_desc* desc, spid_stream_t stream,
                             spid_plan_t* plan_out);

/* Release every resource of the plan.  Synchronizes the device first. */
spid_status spid_plan_destroy(spid_plan_t plan);

/* l = k_max + p, l_pad (row stride of the stored sketch, a multiple of 16),
 * and the plan's device workspace in bytes.  Any pointer may be NULL. */
spid_status spid_plan_info(spid_plan_t plan, int32_t* l, int32_t* l_pad,
                           int64_t* workspace_bytes);

/* Sketch accumulation (Section 2, Y = Omega A), step a2 of the hot path:
 * for every subdomain s, Y_s(:, j) = Omega(:, 0:m_s) A_s(:, j) for the
 * window columns j in [col0, min(col0 + ncols, n_s)).  Columns are
 * independent, so a window may be sketched in any number of calls (one per
 * snapshot or per micro-batch, as the snapshots arrive: Algorithm 6 saves
 * each time step's data); columns never sketched stay zero after
 * spid_plan_create / spid_reset.  window: device, layout as above.  The
 * tensor-core sketches read columns in TMA tiles of the slice width (64
 * columns, or 32 / 16 when tuned so): a range that ends inside a tile still
 * reads the whole tile from memory (past n_s the tile is zero-filled and costs
 * nothing), so micro-batches that are multiples of the slice width read every
 * column once. */
spid_status spid_sketch_accumulate(spid_plan_t plan, const void* window, int32_t col0,
                                   int32_t ncols, spid_stream_t stream);

/* Zero the stored sketch (start a new window).  Asynchronous. */
spid_status spid_reset(spid_plan_t plan, spid_stream_t stream);

/* Finalize (steps a3-a5): batched Householder QR with column pivoting of
 * every Y_s (pivot norms with FP64-class accuracy -- double-float pairs in
 * FP32 modes, FP64 in FP64 mode -- ties to the lowest column index), the rank
 * decision (fixed k_max or adaptive tol, then the guard |R_jj| > 2 u |R_00|
 * with u the unit roundoff of the sketch arithmetic; a guard stop before the
 * target sets the informational SPID_ERR_RANK status), the back-substitution
 * T = R11^-1 R12 with FP64-class accuracy and C with C(:, J) = I exactly. */
spid_status spid_finalize(spid_plan_t plan, spid_stream_t stream);

/* Relative Frobenius error (Section 5.1; step a6): for every subdomain,
 * err_dev[2 s] = ||A_s - A_s(:,J_s) C_s||_F^2 and err_dev[2 s + 1] =
 * ||A_s||_F^2 (FP64 reduction in a fixed order), and total_dev[0..3] =
 * {sum e2, sum a2, sum m_s n_s, sum k_s (m_s + n_s)}, so the global relative
 * error is sqrt(total[0] / total[1]) and the compression factor (Section 2,
 * Eq. for CF, aggregated over subdomains) is total[2] / total[3].  A plan with
 * num_qoi = G > 0 also writes the per-QoI sums total_dev[4 + 2 g] = sum e2 and
 * total_dev[5 + 2 g] = sum a2 over the subdomains holding QoI g (in subdomain
 * order), so total_dev must then hold 4 + 2 G doubles; QoI g's relative
 * error over the domain is sqrt(total[4 + 2 g] / total[5 + 2 g]).
 * A_hat is formed in FP32 on the CUDA cores (FP64 for FP64 plans), or, with
 * SPID_FLAG_TC_ERROR on a batched TF32/BF16/3xBF16 plan with k_max <= 32, on
 * the tensor cores as a three-term TF32 split product (about 2^-21 of
 * |A(:,J)| |C| per entry).
 * err_dev may be NULL.  Requires spid_finalize. */
spid_status spid_error(spid_plan_t plan, const void* window, double* err_dev, double* total_dev,
                       spid_stream_t stream);

/* Reconstruction A_hat_s = A_s(:, J_s) C_s written to out (same layout,
 * offsets and leading dimensions as the window; rows between m_s and ld_s
 * are not touched).  Requires spid_finalize. */
spid_status spid_reconstruct(spid_plan_t plan, const void* window, void* out,
                             spid_stream_t stream);

/* Copy the factors to the host (synchronizes the stream): k_host[S],
 * J_host[S * k_max] (pivot order, -1 past k_s), and C_host packed per
 * subdomain as k_max x n_s row-major blocks, block s at element
 * k_max * sum_{s' < s} n_{s'} (rows >= k_s are zero); element type as the
 * window.  Any pointer may be NULL. */
spid_status spid_get_factors(spid_plan_t plan, int32_t* k_host, int32_t* J_host, void* C_host,
                             spid_stream_t stream);

/* Copy the stored sketch to the host (synchronizes): Y_s as n_s x l_pad
 * (row j = column j of Y_s, entries i >= l are zero), block s at element
 * l_pad * sum_{s' < s} n_{s'}; element type as the window. */
spid_status spid_get_sketch(spid_plan_t plan, void* Y_host, spid_stream_t stream);

/* Synchronize the stream and return the sticky device status, then clear
 * it: SPID_ERR_TIMEOUT, else SPID_ERR_NONFINITE, else SPID_ERR_RANK (the
 * informational rank-guard cut, reading of the paper's silence on a
 * rank-revealing stop), else SPID_OK. */
spid_status spid_device_status(spid_plan_t plan, spid_stream_t stream);

/* Omega(i, r0 + c) for i < l, c < nrows into out_dev as nrows x l row-major
 * (row c holds Omega(:, r0 + c)); FP64 (precision SPID_PREC_FP64) or FP32
 * (the value every FP32 sketch uses).  Step a1, exposed for checking. */
spid_status spid_omega(uint64_t seed, int64_t r0, int32_t nrows, int32_t l, int32_t precision,
                       void* out_dev, spid_stream_t stream);

/* Philox4x32-10 of count counters (ctr_dev: count x 4 words) under the key
 * {key0, key1}; out_dev: count x 4 words.  Exposed for checking. */
spid_status spid_philox(const uint32_t* ctr_dev, uint32_t key0, uint32_t key1, uint32_t* out_dev,
                        int64_t count, spid_stream_t stream);

/* Aggregate compression factor (Section 2, Eq. for CF; Section 3.2):
 * sum m_s n_s / sum k_s (m_s + n_s) over host arrays (step a7).  Host-only
 * arithmetic; returns +inf when every k_s is 0. */
double spid_compression_factor(int32_t num_sub, const int32_t* m, const int32_t* n,
                               const int32_t* k);

/* ---- Tuning ------------------------------------------------------------
 * Tile shapes and schedules of a plan's kernels.  The defaults are fixed;
 * spid_plan_autotune measures the candidates below on the caller's own window
 * (CUDA events on the plan's stream, median of 5 timed runs after one warm-up)
 * and keeps the fastest; a candidate replaces the best one so far only when it
 * is at least 2% faster, so the defaults stay unless a shape clearly wins.  No paper passage corresponds: the paper's
 * subdomains run as independent Legion tasks (Section 3.2) with no kernel of
 * their own.  Results depend on the tuning only through the order of FP32
 * partial sums (sketch slots, error-pass units); each tuning is deterministic. */
typedef struct {
  int32_t sketch_pack_slices;  /* tensor-core and batched CUDA-core sketches: 64-column slices of
                                  equal-shape subdomains sharing one generated Omega chunk: 1, 2,
                                  4 or 8 (default 8, and 2 for the CUDA-core sketch, whose register
                                  tile grows with it; its FP64 form uses at most 4);
                                  spid_plan_autotune also tries both sketch_slice_major orders
                                  (tensor-core sketches) */
  int32_t sketch_stages;       /* tensor-core sketch pipeline depth: 0 = as many as fit in
                                  shared memory (default), else 2..8 (capped by what fits) */
  int32_t sketch_ctas_per_sm;  /* CUDA-core (FP32/FP64) sketch: persistent CTAs per SM, 1..4;
                                  0 = by the register budget of the kernel variant the call's
                                  widest column group selects (default).  One launch per
                                  subdomain (SPID_FLAG_PER_SUBDOMAIN) uses at most 2 */
  int32_t error_path;          /* 0 = CUDA-core error pass (default); 1 = tensor-core pass
                                  (batched TF32/BF16/3xBF16 plans with k_max <= 32 only) */
  int32_t error_rows;          /* CUDA-core error pass: rows per work unit, 256, 512 (default)
                                  or 1024 */
  int32_t error_cols;          /* CUDA-core error pass: columns per work unit, 64, 128 or 256
                                  (default) */
  int32_t sketch_slice_major;  /* tensor-core sketch: 0 = a pack holds consecutive slices of one
                                  subdomain (default), 1 = slice j of consecutive subdomains
                                  (same columns) */
  int32_t sketch_slice_cols;   /* TF32 sketch: window columns per slice (one TMA box), 64
                                  (default; 0 means 64), 32 or 16; packs still hold up to
                                  sketch_pack_slices x 64 columns.  Narrower slices cover fewer
                                  snapshots per chunk, which helps windows whose snapshots lie far
                                  apart (a global field).  Other precisions: 64 only. */
  float sketch_ms;             /* spid_plan_autotune: measured time of the chosen shape to
                                  sketch the whole window in the tuner's calls (0 if the
                                  tuning was set, not measured) */
  float error_ms;              /* spid_plan_autotune: measured error-pass time */
} spid_tuning;

/* Current tuning of the plan.  Host-only. */
spid_status spid_plan_get_tuning(spid_plan_t plan, spid_tuning* out);

/* Apply a tuning (for example one saved from an earlier spid_plan_autotune of
 * a plan with the same spid_plan_tuning_key).  Synchronizes the device and
 * rebuilds the cached sketch schedules; may allocate (schedule tables, the
 * tensor-core error schedule on first use), so call it outside stream capture.
 * SPID_ERR_INVALID_ARG for a value outside the lists above,
 * SPID_ERR_UNSUPPORTED for error_path 1 on a plan that cannot use it,
 * SPID_ERR_STATE while graphs captured from the plan exist.  sketch_ms and
 * error_ms are ignored. */
spid_status spid_plan_set_tuning(spid_plan_t plan, const spid_tuning* tuning);

/* Measure every candidate shape on `window` (device, the plan's layout) and
 * apply the fastest: the sketch candidates on the whole window, then, after a
 * finalize, the error-pass candidates.  Leaves the plan as after
 * spid_sketch_accumulate(whole window) + spid_finalize with the chosen tuning.
 * Synchronizes; may allocate (as spid_plan_set_tuning); best (may be NULL)
 * receives the chosen tuning and its times.  SPID_ERR_STATE while graphs
 * captured from the plan exist. */
spid_status spid_plan_autotune(spid_plan_t plan, const void* window, spid_stream_t stream,
                               spid_tuning* best);

/* spid_plan_autotune for the way the caller sketches: each sketch candidate is
 * timed on the whole window sketched in calls of `microbatch` columns (columns
 * [0, b), [b, 2b), ... up to the longest window; 0 = one whole-window call,
 * which is spid_plan_autotune), since the best shape of a 64-column call
 * differs from that of a 512-column one.  sketch_ms is the time of all those
 * calls.  SPID_ERR_INVALID_ARG for microbatch < 0; otherwise as
 * spid_plan_autotune. */
spid_status spid_plan_autotune_calls(spid_plan_t plan, const void* window, int32_t microbatch,
                                     spid_stream_t stream, spid_tuning* best);

/* A text key for caching tunings across runs: the device (compute capability,
 * SM count), precision, flags, l_pad, k_max and log2 buckets of the subdomain
 * count and of the mean m and n.  Writes at most len bytes including the
 * terminating NUL; SPID_ERR_INVALID_ARG if it does not fit. */
spid_status spid_plan_tuning_key(spid_plan_t plan, char* buf, int32_t len);

/* ---- CUDA graphs -------------------------------------------------------
 * One step of the hot path captured once and replayed with one launch:
 * the sketch of window columns [col0, col0 + ncols) (in calls of `microbatch`
 * columns each, 0 = one call), the finalize and the error pass, or any subset
 * (`what`, an OR of the SPID_GRAPH_* bits, kept in that order).  The graph
 * owns its own tensor maps of `window`, so other calls on the plan with other
 * windows do not disturb it; it uses the plan's workspace (sketch, partial
 * sums, factors, counters), so a graph launch and any other call on the same
 * plan must not overlap on the GPU.  err_dev / total_dev as spid_error (used
 * with SPID_GRAPH_ERROR; both may be NULL).  Creation synchronizes and may
 * allocate (schedules of new column ranges, the graph's tensor maps); launches
 * allocate nothing.  Graphs must be destroyed before their plan (the plan's
 * destroy and set_tuning return SPID_ERR_STATE while any exists). */
typedef struct spid_graph_s* spid_graph_t;
#define SPID_GRAPH_SKETCH 1u
#define SPID_GRAPH_FINALIZE 2u
#define SPID_GRAPH_ERROR 4u
spid_status spid_graph_create(spid_plan_t plan, const void* window, int32_t col0, int32_t ncols,
                              int32_t microbatch, uint32_t what, double* err_dev,
                              double* total_dev, spid_graph_t* graph_out);

/* Replay the captured step on `stream` (asynchronous). */
spid_status spid_graph_launch(spid_graph_t graph, spid_stream_t stream);

/* One end-to-end step from host memory.  Enqueues, in this order: on
 * copy_stream, once the previous launch of this graph has finished with its
 * window, the copy of the window -- the plan's extent, the last element any
 * subdomain reads plus one (blocks: max_s off_s + ld_s (n_s - 1) + m_s) --
 * from window_host to the device window the graph was created on; on
 * `stream`, once that copy has landed, the graph; then, on `stream`, the
 * copies of the step's results to host memory: the error sums (total_dev, 4 +
 * 2 num_qoi doubles) to total_host and the compressed representation
 * (Algorithms 2-3 output: the ranks, skeleton indices and coefficients, laid
 * out as spid_get_factors gives them) to k_host [S], J_host [S k_max] and
 * C_host (k_max sum n_s elements of the window's type).  Any of the four host
 * pointers may be NULL.  All asynchronous: synchronize `stream` before reading
 * them.  window_host and the result buffers should be page-locked for the
 * copies to run at the link's rate; copy_stream may be the same stream (no
 * overlap).  Two graphs on two device windows, launched alternately, overlap
 * one step's copy with the other's compute (the plan's workspace is shared:
 * launch both on the same `stream`, and read a step's factors before the next
 * step's copies overwrite them).  SPID_ERR_INVALID_ARG for a NULL graph or
 * window_host, a graph without a window, or total_host without the graph's
 * total_dev. */
spid_status spid_graph_launch_host(spid_graph_t graph, const void* window_host,
                                   double* total_host, int32_t* k_host, int32_t* J_host,
                                   void* C_host, spid_stream_t copy_stream,
                                   spid_stream_t stream);

/* Release the graph (synchronizes the device first). */
spid_status spid_graph_destroy(spid_graph_t graph);

/* ---- Allocation-free sketch -------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they need a sketch: an in-situ
 * simulation that reserves nearly all GPU memory for its own fields through
 * its own pool at start-up, or whose time loop must not call cudaMalloc /
 * cudaFree (they may synchronize the whole device).  Such a caller cannot
 * create a plan mid-run, because spid_plan_create allocates its workspace.
 *
 * spid_sketch_fp32_noalloc computes the FP32 sketch of ONE subdomain,
 * Y(:, j) = Omega(:, 0:m) A(:, j) for j < n (Omega as defined above, same
 * values as the FP32 entry points), with A an m x n column-major FP32 matrix
 * at device pointer A (16-byte aligned, leading dimension ld >= m, a multiple
 * of 4), and writes Y(i, j) to device memory Y[j * ldy + i] for i < l
 * (ldy >= l); 1 <= l <= 64.  It allocates nothing and calls no allocating
 * routine: its split-K partial sums live in one file-scope device array of
 * SPID_NOALLOC_SCRATCH_FLOATS floats (8 MiB) that every GPU loading this
 * library holds until the process exits.  Limit: ceil(n / 512) * 512 * l_pad
 * <= SPID_NOALLOC_SCRATCH_FLOATS (l_pad = l rounded up to 16), i.e. n <= 65536
 * for l <= 32; larger requests return SPID_ERR_INVALID_ARG with nothing
 * launched.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for
 * the life of the process; make that first call before any stream capture,
 * and do not call cudaDeviceReset on that device afterwards (the kept address
 * would then be stale).  Devices with ordinals of 64 or more get
 * SPID_ERR_UNSUPPORTED.  Every call shares the array and leaves its
 * contents behind (each call overwrites every slot it reads, so nothing needs
 * clearing); calls that overlap on the GPU -- on different streams, or from
 * host threads without ordering -- race on the array and must be serialized
 * by the caller.  Asynchronous on `stream`. */
#define SPID_NOALLOC_SCRATCH_FLOATS (1u << 21)
spid_status spid_sketch_fp32_noalloc(const float* A, int32_t m, int32_t n, int64_t ld, int32_t l,
                                     uint64_t seed, float* Y, int32_t ldy, spid_stream_t stream);

/* ---- In-situ producer ---------------------------------------------------
 * A snapshot producer for measuring compression next to a running solver
 * (Section 5.2 and Algorithms 4-6: the solver updates the state every time
 * step and the compression consumes its snapshots).  A stand-in for the
 * paper's compressible Navier-Stokes solver, not part of the decomposition:
 * one forward-Euler step of f_t + (u . grad) f = nu lap f for every QoI f,
 * velocity u = QoIs 1..3, periodic grid^3 grid of spacing 2 pi / grid,
 * first-order upwind advection and the 7-point Laplacian (stable for
 * dt (3 max|u| / h + 6 nu / h^2) <= 1).  state_in / state_out: device, one
 * snapshot each, boxes of edge^3 points with box index (bz nb + by) nb + bx,
 * nb = grid / edge; box b's [q][z][y][x] block (nq edge^3 floats) starts at
 * element b * box_stride -- nq edge^3 for a snapshot-major window, nq edge^3 n
 * for a subdomain-major one (pointer at the snapshot's column).  Distinct
 * buffers.  SPID_ERR_INVALID_ARG unless grid % edge == 0, nq >= 4, dt > 0,
 * nu >= 0 and both strides >= nq edge^3.  Asynchronous on `stream`. */
spid_status spid_producer_step(const float* state_in, int64_t in_box_stride, float* state_out,
                               int64_t out_box_stride, int32_t grid, int32_t edge, int32_t nq,
                               float dt, float nu, spid_stream_t stream);

/* Human-readable name of a status code (static storage). */
const char* spid_status_string(spid_status status);

/* Detail of the last error raised on the calling thread ("" if none). */
const char* spid_last_error(void);

/* ==========================================================================
 * Subsampled ID and single-pass ID on a coarse grid (Section 2, SubID and SPID
 * paragraphs; Algorithms 2 and 3; Section 5.2 subsampling study).
 *
 * The sketch is deterministic: B = A(J,:) keeps the rows of a coarse grid of
 * each subdomain box (interval s along each axis: indices 0, s, 2s, ... and
 * the last point of the axis, which is appended when it is not a multiple of
 * s).  A pivoted modified Gram-Schmidt QR of B (the paper's mgsqr: residual
 * norms from the updated columns at every step, ties to the lowest column,
 * adaptive stop as Remark 2.1 when tol > 0, rank guard |R_jj| > 2^-23 |R_00|)
 * gives I_B and C_B = [I | R11^-1 R12] Z^T.  Two reconstructions:
 *   SubID  A ~ A(:, I_B) C_B                (needs the window again)
 *   SPID   A ~ M B(:, I_B) C_B              (M = trilinear interpolation from
 *                                            the coarse grid; needs only the
 *                                            stored coarse skeleton)
 * FP32 windows only.  Subdomain s is a box of nq x ez x ey x ex (QoIs x
 * points), stored as an m_s x n_s column-major block of the window
 * (m_s = nq ez ey ex; rows r = ((q ez + z) ey + y) ex + x; off/ld as for
 * spid_plan_desc).  The coarse matrix B_s is m_c(s) x n_s with rows in
 * (q, cz, cy, cx) order.
 * ========================================================================== */
typedef struct spid_sub_plan_s* spid_sub_plan_t;

/* Reconstruction forms of spid_sub_error / spid_sub_reconstruct. */
#define SPID_FORM_SPID 0
#define SPID_FORM_SUBID 1

typedef struct {
  int32_t num_sub;        /* S >= 1 */
  const int32_t* box;     /* host [4 S]: (nq, ez, ey, ex) of subdomain s, all >= 1 */
  const int32_t* n;       /* host [S]: window length n_s, 1 <= n_s <= 1024 */
  const int64_t* off;     /* host [S]: element offset of A_s(0,0) (multiple of 4) */
  const int64_t* ld;      /* host [S]: leading dimension >= m_s (multiple of 4) */
  int32_t stride[3];      /* coarse interval along z, y, x; each >= 1 */
  int32_t k_max;          /* 1 <= k_max <= 64; k_s <= min(k_max, n_s, m_c(s)) */
  double tol;             /* 0: fixed rank k_max; > 0: smallest k with
                             ||R22||_F <= tol ||B||_F (Remark 2.1 reading) */
  uint32_t flags;         /* 0 */
} spid_sub_desc;

/* Point-set form (unstructured grids; Section 2 allows the rows of A in any
 * order, and Section 5.1 compresses a randomly generated point set): the
 * caller gives, per subdomain, the rows of A_s kept in B_s and the
 * interpolation operator M as a fixed-width stencil -- fine row r of
 * subdomain s is sum_q w(r, q) B_s(idx(r, q), :) -- instead of a box and an
 * interval.  Every spid_sub_* call accepts the plan; SPID reconstruction
 * without the window forms M B(:, I_B) C_B directly.  The compression-factor
 * sums count k (m_c + n) (M is not counted, as for boxes). */
typedef struct {
  int32_t num_sub;            /* S, 1..65535 */
  const int32_t* m;           /* host [S]: rows m_s >= 1 */
  const int32_t* n;           /* host [S]: window length, 1 <= n_s <= 1024 */
  const int64_t* off;         /* host [S]: element offset of A_s(0,0) (multiple of 4) */
  const int64_t* ld;          /* host [S]: leading dimension >= m_s (multiple of 4) */
  const int32_t* mc;          /* host [S]: coarse rows, 1 <= m_c(s) <= min(m_s, 40960) */
  const int32_t* coarse_rows; /* host [sum m_c]: subdomain s's rows of A_s (each in
                                 [0, m_s)) at offset sum_{s'<s} m_c(s'); B_s row i is A_s
                                 row coarse_rows[...+ i] */
  int32_t stencil;            /* t, 1..16: coarse rows per fine row */
  const int32_t* interp_idx;  /* host [t sum m]: fine row r of subdomain s at
                                 t (sum_{s'<s} m_s' + r) .. + t - 1: coarse rows in [0, m_c(s)) */
  const float* interp_w;      /* host, same layout: finite weights */
  int32_t k_max;              /* 1..64 */
  double tol;                 /* as spid_sub_desc */
  uint32_t flags;             /* 0 */
} spid_sub_points_desc;

/* Create a point-set plan (the host tables are copied; later calls allocate
 * nothing).  SPID_ERR_INVALID_ARG for a size, index or weight out of range.
 * Like spid_sub_plan_create, it sets the current context's L2 fetch
 * granularity (cudaLimitMaxL2FetchGranularity) to 32 bytes. */
spid_status spid_sub_plan_create_points(const spid_sub_points_desc* desc, spid_sub_plan_t* plan);

/* Create a plan: validates, allocates all workspace (later calls allocate
 * nothing).  m_c(s) <= 40960 coarse rows (the QR keeps one column of B in
 * shared memory); SPID_ERR_UNSUPPORTED beyond.  Side effect: sets the current
 * context's L2 fetch granularity (cudaLimitMaxL2FetchGranularity) to 32 bytes
 * -- the gathers read scattered sectors, which whole-line fills from DRAM
 * would double; the limit is a hint that belongs to the context (it ends with
 * the process) and moved the streaming kernels' rates by < 1%. */
spid_status spid_sub_plan_create(const spid_sub_desc* desc, spid_sub_plan_t* plan);
spid_status spid_sub_plan_destroy(spid_sub_plan_t plan);

/* mc_host (may be NULL): [S] coarse rows m_c(s).  workspace (may be NULL):
 * device bytes owned by the plan. */
spid_status spid_sub_plan_info(spid_sub_plan_t plan, int64_t* mc_host, int64_t* workspace);

/* Gather B_s(:, col0 .. col0 + ncols) = A_s(J, cols) for every subdomain with
 * n_s > col0 (columns past n_s are skipped).  Single pass: the window columns
 * may be overwritten once the call's stream has passed it. */
spid_status spid_sub_sample(spid_sub_plan_t plan, const float* window, int32_t col0,
                            int32_t ncols, spid_stream_t stream);

/* Pivoted MGS QR of every B_s, rank decision, C_B and the coarse skeleton
 * B_s(:, I_B).  A subdomain whose B holds a non-finite value gets k = 0 and
 * sets SPID_ERR_NONFINITE in the sticky status. */
spid_status spid_sub_finalize(spid_sub_plan_t plan, spid_stream_t stream);

/* Errors of the chosen form, as spid_error: err_dev[2 s] = ||A_s - A_hat_s||^2,
 * err_dev[2 s + 1] = ||A_s||^2 (may be NULL), total_dev[0..3] = {sum e2,
 * sum a2, sum m_s n_s, sum k_s (r_s + n_s)} with r_s = m_c(s) for SPID (the
 * coarse skeleton is what is stored) and r_s = m_s for SubID. */
spid_status spid_sub_error(spid_sub_plan_t plan, const float* window, int32_t form,
                           double* err_dev, double* total_dev, spid_stream_t stream);

/* A_hat written to out (window layout).  SPID needs no window (NULL allowed). */
spid_status spid_sub_reconstruct(spid_sub_plan_t plan, const float* window, int32_t form,
                                 float* out, spid_stream_t stream);

/* Copy factors to the host (synchronizes): k_host[S], J_host[S k_max] (-1 past
 * k_s), C_host k_max x n_s row-major per subdomain at k_max sum_{s'<s} n_s',
 * Bskel_host m_c(s) x k_max column-major per subdomain at
 * k_max sum_{s'<s} m_c(s') (columns past k_s zero).  Any pointer may be NULL. */
spid_status spid_sub_get_factors(spid_sub_plan_t plan, int32_t* k_host, int32_t* J_host,
                                 float* C_host, float* Bskel_host, spid_stream_t stream);

/* Copy the gathered coarse matrices to the host (synchronizes): B_s as
 * m_c(s) x n_s column-major at sum_{s'<s} m_c(s') n_s'. */
spid_status spid_sub_get_coarse(spid_sub_plan_t plan, float* B_host, spid_stream_t stream);

/* Sticky device status of the plan (as spid_device_status), then cleared. */
spid_status spid_sub_device_status(spid_sub_plan_t plan, spid_stream_t stream);

/* ==========================================================================
 * Modified (two-stage) SPID (Section 3.3.2, Algorithm 6).
 *
 * Stage 1: the window of every subdomain is cut into N time blocks of n_s / N
 * snapshots and each block gets its own sketched column ID with target rank k
 * (A_b ~ A_b(:, I_b) C_b), computed block by block as the snapshots arrive.
 * Stage 2: the skeleton columns of all blocks, A0' = [A_0(:, I_0) .. A_{N-1}(:,
 * I_{N-1})] (m_s x N k), get a sketched column ID with a tolerance,
 * A0' ~ A1' C1, and the final factors are A1' = A(:, J) with J the union
 * indices I_U picked by stage 2, and C1' = C1 C0' (C0' = blockdiag(C_b)),
 * so A ~ A(:, J) C1'.  C1'(:, J) = I exactly.
 * ========================================================================== */
typedef struct spid_ts_plan_s* spid_ts_plan_t;

typedef struct {
  spid_plan_desc base;   /* the S subdomains over the whole window: m, n (each n_s a
                            multiple of blocks), off, ld; k_max = the stage-1 target
                            rank k; p, precision, seed as spid_plan_desc (both stages);
                            base.tol and base.flags must be 0 */
  int32_t blocks;        /* N >= 1 */
  int32_t k2_max;        /* stage-2 rank cap, 1 <= k2_max <= N k_max, k2_max + p <= 64 */
  double tol2;           /* stage-2 tolerance (> 0; Remark 2.1 reading as spid_plan_desc) */
} spid_ts_desc;

/* Create: allocates every workspace (N stage-1 plans, the stage-2 plan over
 * the N k skeleton slots per subdomain and the final factors).  Later calls
 * allocate nothing.  k_max + p and k2_max + p must both be <= 64. */
spid_status spid_ts_plan_create(const spid_ts_desc* desc, spid_ts_plan_t* plan);
spid_status spid_ts_plan_destroy(spid_ts_plan_t plan);

/* Stage 1 for time block b (0 <= b < N): sketch of columns b n_s / N ..
 * (b + 1) n_s / N - 1 of every subdomain, QR, rank k, C_b.  Blocks may be run
 * in any order, each once per window. */
spid_status spid_ts_block(spid_ts_plan_t plan, const void* window, int32_t block,
                          spid_stream_t stream);

/* Stage 2 (after every block): the sketched ID of A0' with tol2 and the
 * composition C1' = C1 C0', J = I_U(J2).  Both stages draw the same rows of
 * Omega, so the sketch of A0' is the blocks' sketch columns at their
 * skeleton indices (the block plans sketch k2_max + p rows for it): stage 2
 * gathers them and reads no window data.  window must be the block window
 * (16-byte aligned); it is checked, not read. */
spid_status spid_ts_finalize(spid_ts_plan_t plan, const void* window, spid_stream_t stream);

/* Error / reconstruction of the final factors, as spid_error / spid_reconstruct. */
spid_status spid_ts_error(spid_ts_plan_t plan, const void* window, double* err_dev,
                          double* total_dev, spid_stream_t stream);
spid_status spid_ts_reconstruct(spid_ts_plan_t plan, const void* window, void* out,
                                spid_stream_t stream);

/* Final factors as spid_get_factors (synchronizes): k_host[S],
 * J_host[S k2_max] (window column indices, -1 past k_s), C_host k2_max x n_s
 * row-major per subdomain at k2_max sum_{s'<s} n_s'. */
spid_status spid_ts_get_factors(spid_ts_plan_t plan, int32_t* k_host, int32_t* J_host,
                                void* C_host, spid_stream_t stream);

/* Stage-1 factors of block b, as spid_get_factors of a plan over the block
 * (J local to the block, C k_max x n_s / N per subdomain). */
spid_status spid_ts_get_block_factors(spid_ts_plan_t plan, int32_t block, int32_t* k_host,
                                      int32_t* J_host, void* C_host, spid_stream_t stream);

/* Sticky status of every plan the two-stage plan owns, then cleared. */
spid_status spid_ts_device_status(spid_ts_plan_t plan, spid_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPID_H */
