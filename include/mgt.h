/*
 * mgt -- transposition of multigraphs and high-cardinality sparse matrices
 * (XCSR) on one GB300 GPU.
 *
 * The operation (paper, Sec. 2 "Problem Specification"): a matrix M whose
 * cell (i, j) holds a list of values of its own length is transposed,
 * M^T_ij = M_ji; every edge {i, j, e} becomes {j, i, e}.  The storage format
 * is the paper's XCSR (Sec. 2): CSR plus a per-cell count of values, the
 * values serialised into one array.  Here the per-row and per-cell counts
 * are passed as prefix arrays:
 *
 *   row_ptr[n_rows + 1]   cells of row i are [row_ptr[i], row_ptr[i+1])
 *   col_idx[n_cells]      column of each cell (int32)
 *   cell_ptr[n_cells + 1] values of cell k are [cell_ptr[k], cell_ptr[k+1])
 *   values[n_values]      payload_stride bytes each, opaque (never interpreted)
 *
 * row_ptr and cell_ptr are offset_bytes wide (4: int32, 8: int64).
 *
 * The result is the XCSR of M^T: n_cols rows, the same cells and values.
 * Inside each output row the cells follow ascending source-cell order (for
 * inputs whose rows hold distinct columns: ascending source row), which is
 * the "row-column ordering" of the view-swap step (Sec. 3); the values of a
 * cell keep their order.  The paper's R ranks holding row blocks (Sec. 2,
 * Sec. 3) are P virtual partitions: rows [part_off[d], part_off[d+1]) form
 * block d of the input and, because vertex information stays local
 * (Sec. 2), block d of the output.  The P x P counts of cells and of values
 * sent from source block s to destination block d are the metadata-count
 * and value-count matrices that the two view-swap exchanges transpose
 * (Sec. 3, Figs. 5-6); on one GPU the exchange itself collapses into the
 * on-device scatter.
 *
 * Conventions for every call:
 *   - Pointers named "device" must be GPU global memory of the current
 *     device; "host" pointers are read during the call only.
 *   - The caller owns every buffer: inputs, outputs (same sizes as the
 *     input except that the output row_ptr has n_cols + 1 entries) and the
 *     workspace.  A plan owns only host metadata.
 *   - Transposes are out of place (the paper's in-place reference swap of
 *     Sec. 2 becomes: the caller swaps its pointers afterwards).
 *   - Calls that take a stream enqueue work on it and return; nothing is
 *     synchronised unless the call says so.
 *   - Return values: MGT_OK or a negative MGT_E* code (Sec. 2: every MPI
 *     call of the paper returns an int status).  Device-detected problems
 *     (malformed input, internal limits) are recorded in a status word in
 *     the workspace and returned by mgt_read_status.
 */
#ifndef MGT_H
#define MGT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGT_OK 0
#define MGT_EINVAL (-1)     /* bad descriptor or argument */
#define MGT_ENOMEM (-2)     /* host allocation failed, or workspace too small */
#define MGT_EBADINPUT (-3)  /* device found malformed input (column out of
                               range, decreasing pointers, wrong totals) */
#define MGT_ETIMEOUT (-4)   /* a bounded device wait expired */
#define MGT_EAGAIN (-5)     /* admission refused: no slot or memory now */
#define MGT_ECUDA (-6)      /* a CUDA runtime call failed */
#define MGT_EOVERFLOW (-7)  /* an internal per-tile limit was exceeded */
#define MGT_ENOTFOUND (-8)  /* unknown ticket */

/* A cudaStream_t, passed as an opaque pointer (NULL = legacy stream). */
typedef void *mgt_stream_t;

typedef struct mgt_plan_s mgt_plan_t;

/* Problem descriptor (Sec. 2: the row count, the XCSR arrays' sizes, the
 * datatype serialised as bytes -- the MPI_BYTE variant of Sec. 2 -- and the
 * ranks' row blocks). */
typedef struct {
    int64_t n_rows;          /* R >= 0, R <= 2^31 - 1 (rows become int32 columns) */
    int64_t n_cols;          /* N >= 0, N <= 2^31 - 1 */
    int64_t n_cells;         /* C >= 0 (C < 2^31 when offset_bytes == 4) */
    int64_t n_values;        /* V >= 0 (V < 2^31 when offset_bytes == 4) */
    int32_t offset_bytes;    /* 4 or 8: width of row_ptr and cell_ptr */
    int32_t payload_stride;  /* bytes per value: > 0 and a multiple of 4 */
    int32_t n_parts;         /* P >= 1; P > 1 requires n_rows == n_cols (Sec. 2: M is square) */
    int32_t flags;           /* 0, or MGT_FLAG_VAR_WIDTH (then payload_stride must be 1) */
    const int64_t *part_off; /* host, P + 1 entries, 0 = off[0] <= ... <= off[P] = n_rows;
                                NULL = P equal blocks, off[d] = floor(d R / P) */
} mgt_desc;

/* desc.flags: the values have individual byte widths (see mgt_transpose_var). */
#define MGT_FLAG_VAR_WIDTH 1

/* Input matrix: all device pointers, layout as described at the top. */
typedef struct {
    const void *row_ptr;
    const int32_t *col_idx;
    const void *cell_ptr;
    const void *values;
} mgt_xcsr_in;

/* Writable buffers for one matrix's four arrays (mgt_transpose_host: the
 * device copies of the input). */
typedef struct {
    void *row_ptr;
    int32_t *col_idx;
    void *cell_ptr;
    void *values;
} mgt_xcsr_buf;

/* Output matrix: all device pointers.  part_cells / part_values are
 * optional (NULL skips them): P x P int64, row-major [source][destination]. */
typedef struct {
    void *row_ptr;
    int32_t *col_idx;
    void *cell_ptr;
    void *values;
    int64_t *part_cells;
    int64_t *part_values;
} mgt_xcsr_out;

/* Tile shapes of the kernels (picked by mgt_plan's heuristic, or set by an
 * autotuner through mgt_plan_tuned).  Zero fields take the default. */
typedef struct {
    int32_t bucket_shift; /* log2 of the columns per bucket, 0..16 */
    int32_t scatter_tile; /* cells per bucket-scatter tile (multiple of 512, <= 262144) */
    int32_t cluster;      /* CTAs per sort cluster: 1, 2, 4 or 8 */
    int32_t chunk_cap;    /* records per sort CTA (multiple of 512, <= 8192) */
    int32_t copy_unroll;  /* 16-byte loads in flight per thread in the value copy: 1, 2 or 4 */
    int32_t reserved[3];
} mgt_tile_cfg;

/* Builds a plan for one descriptor.  Validates the descriptor (MGT_EINVAL),
 * copies part_off, picks tile shapes, and returns in *workspace_bytes the
 * device workspace mgt_transpose needs.  Host-only; no CUDA calls other
 * than a device-attribute query. */
int mgt_plan(const mgt_desc *desc, mgt_plan_t **plan, size_t *workspace_bytes);

/* Same with explicit tile shapes (fields outside their ranges: MGT_EINVAL). */
int mgt_plan_tuned(const mgt_desc *desc, const mgt_tile_cfg *cfg, mgt_plan_t **plan,
                   size_t *workspace_bytes);

/* The tile shapes a plan uses. */
int mgt_plan_config(const mgt_plan_t *plan, mgt_tile_cfg *cfg);

void mgt_plan_destroy(mgt_plan_t *plan);

/* Re-transposes only the values of a matrix whose structure did not change
 * (the value part of Sec. 3's view swap: each run moves to its cell's new
 * place, internal order kept):
 * after an mgt_transpose with this plan and workspace, the workspace holds
 * every output cell's run offset in the input and out->cell_ptr the output
 * run offsets; this call copies in->values into out->values along them (one
 * kernel: the value-copy phase).  The caller guarantees that row_ptr,
 * col_idx and cell_ptr are those of that transpose and that the workspace
 * was not used for another matrix since.  in->values may hold new payloads.
 * Same argument checks as mgt_transpose for the arrays it touches.  The
 * paper repeats full transposes (its 12-transpose chains); this is the
 * cheaper repetition when only payloads change. */
int mgt_transpose_values(mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                         void *workspace, size_t workspace_bytes, mgt_stream_t stream);

/* Transposes a matrix whose values have individual byte widths -- the
 * paper's second variation of the exchange (Sec. 2: heterogeneous datatypes
 * across edges, one MPI datatype per edge through MPI_Alltoallw).  The plan
 * comes from mgt_plan with desc.flags = MGT_FLAG_VAR_WIDTH and
 * desc.payload_stride = 1 (n_values still counts values).  Value v of the
 * input occupies bytes [in_val_off[v], in_val_off[v + 1]) of in->values.
 * The cells move exactly as in mgt_transpose (same row_ptr', col_idx',
 * cell_ptr' and P x P counts); every value keeps its bytes and its place in
 * its cell's list, so out->values holds the same values in the output's cell
 * order and out_val_off[0 .. n_values] their byte offsets there.
 *   in_val_off, out_val_off: device int64, n_values + 1 entries each
 *   (in_val_off[0] = 0, non-decreasing, in_val_off[n_values] = n_bytes).
 *   in->values, out->values: device, n_bytes bytes each (may be NULL when
 *   n_bytes == 0).  Any byte width is allowed, zero included; widths and
 *   offsets that are multiples of 16, 8 or 4 take wider copies.
 *   events: NULL, or caller-created CUDA events as for mgt_transpose_profiled
 *   (n_events >= phases + 1; the "copy" phase covers the byte copy).
 * Device-detected errors (mgt_read_status): MGT_EBADINPUT also for value
 * offsets that decrease, do not start at 0 or do not end at n_bytes; no
 * byte outside [0, n_bytes) is read or written.  Other errors as for
 * mgt_transpose; MGT_EINVAL for a plan without MGT_FLAG_VAR_WIDTH.  Plans
 * with MGT_FLAG_VAR_WIDTH are refused by every other transpose call. */
int mgt_transpose_var(mgt_plan_t *plan, const mgt_xcsr_in *in, const int64_t *in_val_off,
                      mgt_xcsr_out *out, int64_t *out_val_off, int64_t n_bytes, void *workspace,
                      size_t workspace_bytes, mgt_stream_t stream, void *const *events,
                      int n_events);

/* Transposes one matrix (Sec. 3: Transpose = LocalTranspose o ViewSwap,
 * computed here as a bucketed counting sort).  workspace: device, at least
 * the plan's workspace_bytes, 256-byte aligned, not shared with a transpose
 * in flight.  Input and output must not overlap.  Enqueues on stream. */
int mgt_transpose(mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out, void *workspace,
                  size_t workspace_bytes, mgt_stream_t stream);

/* The transpose of a matrix held in HOST memory (the operation of Sec. 3, as
 * mgt_transpose), host copies included:
 * host_in -> dev_in (host to device), mgt_transpose(dev_in, dev_out), then
 * dev_out -> host_out (device to host).  host_in / host_out: host arrays of
 * the input and output sizes (pinned memory for asynchronous copies; pageable
 * memory works, with copies that block the calling thread).  dev_in /
 * dev_out: device buffers of the same sizes; dev_out's P x P arrays (device)
 * are filled when given and copied into host_out's P x P arrays (host) when
 * both are non-NULL.  workspace: as for mgt_transpose.
 * With copy_stream non-NULL (a second stream of the caller) the copies that
 * do not feed the next kernel overlap the kernels: the values are uploaded on
 * copy_stream while the structure phases run on stream (only the value copy
 * reads them), and the output structure (row_ptr', col_idx', cell_ptr', P x P)
 * is downloaded on copy_stream while the value copy runs.  Everything the call
 * enqueues is complete when stream reaches its end; copy_stream carries work
 * of this call only between those points.  NULL: all on stream, in order.
 * Callers that alternate two sets of device buffers (and streams) between
 * calls overlap one call's downloads with the next call's uploads.
 * Errors: as mgt_transpose, plus MGT_EINVAL for NULL host arrays that the
 * sizes require, or host P x P arrays without device ones; MGT_ECUDA when a
 * copy or event call fails (mgt_last_error names it). */
int mgt_transpose_host(mgt_plan_t *plan, const mgt_xcsr_in *host_in, mgt_xcsr_out *host_out,
                       const mgt_xcsr_buf *dev_in, mgt_xcsr_out *dev_out, void *workspace,
                       size_t workspace_bytes, mgt_stream_t stream, mgt_stream_t copy_stream);

/* As mgt_transpose, and also records caller-created CUDA events (cudaEvent_t
 * passed as void *) on the stream around the pipeline's phases: events[0]
 * before the first phase, events[i + 1] after phase i.  n_events must be at
 * least mgt_plan_phases(plan, NULL, 0) + 1.  For timing individual kernels;
 * the work enqueued is identical to mgt_transpose's. */
int mgt_transpose_profiled(mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                           void *workspace, size_t workspace_bytes, mgt_stream_t stream,
                           void *const *events, int n_events);

/* Number of pipeline phases; fills names[0 .. min(max_names, phases)) with
 * static strings ("setup", "hist", "scan_tiles", "scan_buckets", "scatter",
 * "scatter2", "build_work", "chunk_hist", "chunk_scan", "place", "place_chunks",
 * "place_fallback", "part_counts", "copy"). */
int mgt_plan_phases(const mgt_plan_t *plan, const char **names, int max_names);

/* Number of kernel launches one mgt_transpose of this plan makes. */
int mgt_plan_kernel_launches(const mgt_plan_t *plan);

/* Synchronises stream and returns the status word the last transpose wrote
 * into workspace: MGT_OK, MGT_EBADINPUT, MGT_EOVERFLOW or MGT_ETIMEOUT. */
int mgt_read_status(const void *workspace, mgt_stream_t stream);

/* ---------------------------------------------------------- autotuner
 * Tile shapes only change how the work is cut (bucket width, sort cluster
 * size, value-copy width); every shape computes the same transpose.  The
 * autotuner searches around mgt_plan's default: bucket_shift -1/0/+1 x
 * cluster 1/2/4/8 at the default copy width, then the other copy widths
 * for the fastest of those. */

/* Fills cands[0 .. min(n, max)) with the shapes the search may try and
 * returns n (or a negative status for a bad descriptor). */
int mgt_autotune_candidates(const mgt_desc *desc, mgt_tile_cfg *cands, int max);

/* Largest workspace any candidate needs. */
int mgt_autotune_workspace(const mgt_desc *desc, size_t *bytes);

/* Times every candidate on the caller's buffers (one warm-up, then `reps`
 * runs between two events on `stream`; synchronizes), skipping candidates
 * whose workspace exceeds workspace_bytes, and returns in *best the full
 * shape of the fastest (to pass to mgt_plan_tuned) and in *best_ms its mean
 * time.  `out` holds a correct transpose afterwards.  MGT_ENOMEM when no
 * candidate fits; a device status other than MGT_OK stops the search. */
int mgt_autotune(const mgt_desc *desc, const mgt_xcsr_in *in, mgt_xcsr_out *out, void *workspace,
                 size_t workspace_bytes, mgt_stream_t stream, int reps, mgt_tile_cfg *best,
                 float *best_ms);

/* ------------------------------------------------------------ batches
 * Many independent transposes at once (the paper transposes one matrix per
 * call; batching is this library's addition for many small and uneven
 * matrices).  Every pipeline phase is ONE kernel launch over all members:
 * the grid's blocks are dealt to the members through a device table, in
 * proportion to their work, so small matrices share the GPU instead of
 * each paying a launch sequence of its own.  Members whose plans need the
 * same kernel instantiations (offset width, record format, cluster size,
 * copy width) share launches; others get launches of their own.  Each
 * member's result is exactly what mgt_transpose gives for it. */

/* Workspace for a batch of n members: a table region followed by every
 * member's own workspace (mgt_plan's size, 256-byte aligned). */
int mgt_batched_workspace(int n, mgt_plan_t *const *plans, size_t *workspace_bytes);

/* Transposes n independent matrices, one launch per phase for the whole
 * batch.  plans[m], in[m], out[m] describe member m; workspace: device,
 * 256-byte aligned, >= mgt_batched_workspace bytes.  Copies the batch's
 * launch tables from pageable host memory into the workspace on `stream`
 * (the call returns once they are staged).  MGT_EINVAL / MGT_ENOMEM as for
 * mgt_transpose; per-member device status: mgt_batch_status or
 * mgt_read_status on the member's workspace. */
int mgt_transpose_batched(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in,
                          mgt_xcsr_out *out, void *workspace, size_t workspace_bytes,
                          mgt_stream_t stream);

/* mgt_transpose_batched with events (cudaEvent_t passed as void *) around
 * its steps: events[0] first, events[1] after zeroing the members' counters,
 * events[i + 2] after phase i (mgt_plan_phases order).  n_events >=
 * phases + 2.  For timing the batched kernels. */
int mgt_transpose_batched_profiled(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in,
                                   mgt_xcsr_out *out, void *workspace, size_t workspace_bytes,
                                   mgt_stream_t stream, void *const *events, int n_events);

typedef struct mgt_batch_s mgt_batch_t;

/* A reusable batch: writes the launch tables into `workspace` (synchronous
 * copy) and captures the whole launch sequence once into a CUDA graph.  The
 * buffers in in[] / out[] and the workspace are bound to the batch: they
 * must stay allocated, and each mgt_batch_launch recomputes the transposes
 * of whatever the inputs then hold (same sizes as the plans).  Launches of
 * one batch must not overlap each other (they share the workspace). */
int mgt_batch_create(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                     void *workspace, size_t workspace_bytes, mgt_batch_t **batch);

/* Replays the batch's graph on `stream` (one graph launch). */
int mgt_batch_launch(mgt_batch_t *batch, mgt_stream_t stream);

/* Kernel launches one replay contains. */
int mgt_batch_kernel_launches(const mgt_batch_t *batch);

/* Synchronizes `stream`, then reads every member's device status word into
 * status[m] (MGT_OK, MGT_EBADINPUT, MGT_EOVERFLOW or MGT_ETIMEOUT, in call
 * order); returns the first non-OK status, or MGT_OK. */
int mgt_batch_status(const mgt_batch_t *batch, mgt_stream_t stream, int *status);

void mgt_batch_destroy(mgt_batch_t *batch);

/* ------------------------------------------------------------ serving
 * A request loop for many concurrent transposes (this library's addition;
 * the paper has none).  A request is (plan, input, output) on caller-owned
 * device buffers that stay valid until the request is done.  The server
 * owns a scheduler thread, n_streams CUDA streams and a memory pool for the
 * workspaces.  A request's footprint is its workspace plus its input and
 * output bytes (mgt_minimal_bytes); requests are admitted in arrival order
 * while the in-flight footprint stays within hbm_budget_bytes and fewer
 * than max_slots are in flight, so new requests start as soon as slots and
 * memory free up while others run (continuous batching).  Runs of queued
 * requests with at most fuse_max_cells cells, at most 64 row blocks and the
 * same kernel formats are fused (up to batch_max) into one batched launch.
 * Results are bit-identical to mgt_transpose of the same request alone.
 * Latency = completion (stamped on the stream by a host function) minus
 * submission. */
typedef struct {
    size_t hbm_budget_bytes; /* admission budget, bytes (e.g. 180e9) */
    int32_t max_slots;       /* requests in flight at once, 1..4096 */
    int32_t n_streams;       /* streams the launches spread over, 1..64 */
    int32_t max_queue;       /* waiting requests before mgt_submit says MGT_EAGAIN */
    int32_t batch_max;       /* most requests fused into one launch (1: no fusion), <= 256 */
    int64_t fuse_max_cells;  /* requests up to this many cells may be fused */
    int32_t batch_window_us; /* a fusable request at the head of the queue waits up to this
                                long for batch_max - 1 compatible ones (0: never waits),
                                <= 1e6 */
} mgt_server_cfg;

typedef struct {
    uint64_t submitted, completed, failed, rejected;
    uint64_t launches;               /* single or fused launches started */
    uint64_t fused_requests;         /* requests that ran inside fused launches */
    uint64_t bytes;                  /* minimal bytes of the completed requests */
    uint64_t peak_inflight_bytes;    /* largest admitted footprint at once (<= budget) */
    uint64_t peak_inflight_requests;
    uint64_t inflight_bytes, queued; /* now */
    double p50_ms, p99_ms, mean_ms;  /* latency of the completed requests */
    double span_s;                   /* first submission -> last completion */
} mgt_server_stats;

typedef struct mgt_server_s mgt_server_t;

/* Creates the server on the current device.  MGT_EINVAL for fields out of
 * range. */
int mgt_server_create(const mgt_server_cfg *cfg, mgt_server_t **server);

/* Queues a request; *ticket identifies it.  MGT_EAGAIN when max_queue
 * requests are waiting, MGT_ENOMEM when its footprint alone exceeds the
 * budget, MGT_EINVAL for missing buffers.  Thread-safe. */
int mgt_submit(mgt_server_t *server, mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out,
               uint64_t *ticket);

/* *done = 1 once the request finished; then *status (MGT_OK or the device
 * status) and *latency_ms are set and the ticket is released (a second poll
 * gives MGT_ENOTFOUND).  Non-blocking, thread-safe. */
int mgt_poll(mgt_server_t *server, uint64_t ticket, int *done, int *status, double *latency_ms);

/* Blocks until nothing is queued or in flight. */
int mgt_server_drain(mgt_server_t *server);

int mgt_server_get_stats(mgt_server_t *server, mgt_server_stats *stats);
int mgt_server_reset_stats(mgt_server_t *server);

/* Finishes queued and in-flight requests, then frees the server. */
void mgt_server_destroy(mgt_server_t *server);

/* Transpose without any allocation, for callers that cannot allocate device
 * memory themselves (for example a plug-in whose host framework owns every
 * device allocation, or a loop that cannot afford the implicit device-wide
 * synchronisation of cudaMalloc / cudaFree).  The paper has no counterpart:
 * this is an interface convenience of this library.
 *
 * Same result as mgt_plan + mgt_transpose with the default plan, but the
 * scratch lives in one file-scope device array of MGT_STATIC_SCRATCH_BYTES
 * inside the library; every GPU that loads the library holds that array
 * until the process exits.  The call makes no cudaMalloc, cudaFree, pinned
 * host allocation or other allocating call, and needs no plan.
 *   desc: host; as for mgt_plan, with n_parts <= MGT_STATIC_MAX_PARTS.
 *   in, out: device arrays as for mgt_transpose.
 * Errors: MGT_EINVAL (bad descriptor or pointers), MGT_ENOMEM when the
 * default plan's workspace (mgt_plan's *workspace_bytes for the same
 * descriptor) exceeds MGT_STATIC_SCRATCH_BYTES -- roughly matrices of a few
 * million cells at most -- and MGT_ECUDA.
 * The first call on a device looks up the array's device address (with
 * that device current), and so does the first call after that device's
 * context was replaced (e.g. by cudaDeviceReset, which reloads the module);
 * make those calls before any stream capture.
 * All calls on a device share the one array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, or another
 * host thread) race and give wrong results; serialise them, e.g. on one
 * stream.  Device-detected errors: mgt_static_status. */
#define MGT_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
#define MGT_STATIC_MAX_PARTS 4096
int mgt_transpose_static(const mgt_desc *desc, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                         mgt_stream_t stream);

/* Synchronises stream and returns the device status word of the last
 * mgt_transpose_static on the current device (as mgt_read_status). */
int mgt_static_status(mgt_stream_t stream);

/* Memory-system probe (diagnostic; not part of a transpose).  The value
 * exchange of the view swap (Sec. 3, second step) permutes runs of values;
 * on one GPU the permutation can be walked in output order (random reads,
 * sequential writes: what mgt_transpose does) or in input order (sequential
 * reads, random writes).  This call times neither; it enqueues one kernel
 * that moves n_runs runs of run_bytes bytes in one of those orders, so a
 * caller can time the raw rates with events:
 *   mode 0  dst run r <- src run perm[r]     (gather)
 *   mode 1  dst run perm[r] <- src run r     (scatter)
 *   mode 2  ((uint32_t *)dst)[perm[r]] = r   (one 4-byte random write per run:
 *                                            the scatter's offset array)
 *   mode 3  dst run r <- src run r           (sequential copy)
 *   mode 4  as mode 0, the loads staged in shared memory with cp.async
 *           (more bytes in flight per thread than registers allow)
 *   mode 5  as mode 0 through the TMA engine: one bulk copy (cp.async.bulk)
 *           per run into shared memory, one bulk store per 32 output runs
 *           (run_bytes <= 1024)
 * src, dst: device, 16-byte aligned, n_runs * run_bytes bytes each (mode 2:
 * dst of n_runs * 4 bytes at least, src unused); perm: device, n_runs uint32
 * holding a permutation of [0, n_runs) (modes 0-2, 4, 5; the caller
 * guarantees it -- indices are not checked on the device).  run_bytes: a
 * multiple of 16 (mode 2: >= 4).  MGT_EINVAL for arguments out of range. */
int mgt_probe_runs(int mode, const void *src, void *dst, const uint32_t *perm, int64_t n_runs,
                   int32_t run_bytes, mgt_stream_t stream);

/* Mode 5 bounds every wait on a bulk copy; *count receives how many waits
 * ran out of polls on the current device since the library was loaded (the
 * kernel then stops early, so its output is incomplete).  Synchronises with
 * the device.  MGT_EINVAL for a null count. */
int mgt_probe_errors(unsigned *count);

/* The L2 fetch granularity hint of the calling thread's CUDA context on the
 * current device (cudaLimitMaxL2FetchGranularity: how many bytes L2 fetches
 * from DRAM on a miss, 0-128; the driver may clamp or ignore it).
 * *prev_bytes (may be NULL) receives the value before the call; set_bytes
 * >= 0 sets a new one for later launches, -1 only reads.  The hint is
 * context-wide and ends with the context.  MGT_EINVAL for set_bytes > 128,
 * MGT_ECUDA when the runtime refuses. */
int mgt_l2_fetch_granularity(int32_t set_bytes, int32_t *prev_bytes);

/* Minimal bytes of one transpose: the input read once plus the output
 * written once (used for throughput figures).  For a descriptor with
 * MGT_FLAG_VAR_WIDTH the value offsets are counted (8 (V + 1) bytes a side)
 * but not the value bytes, which the descriptor does not know: add
 * 2 * n_bytes. */
int64_t mgt_minimal_bytes(const mgt_desc *desc);

/* Human-readable text for an MGT_* code. */
const char *mgt_strerror(int code);

/* Library version string. */
const char *mgt_version(void);

/* The last failed CUDA call of this host thread behind an MGT_ECUDA: phase
 * or step name, CUDA error name and text.  Static storage per thread. */
const char *mgt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MGT_H */
