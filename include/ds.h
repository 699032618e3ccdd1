/*
 * ds.h -- C ABI of libds, a B300 (sm_103a) implementation of the separable
 * decimating FIR filter stage ("downscaler") of Rodrigues, Guyomarc'h and
 * Dekeyser, "Programming Massively Parallel Architectures using MARTE: a
 * Case Study" (arXiv:1103.4881).
 *
 * The operation (paper Sec. 3, "Case Study: H.263 Video Downscaling"): a
 * horizontal filter followed by a vertical filter; each maps packets of q
 * input pixels to p output pixels ("interpolating packets of 8 pixels both
 * row- and column-wise", 352 -> 132 per line at p/q = 3/8).  Every output is
 * a K-tap dot product over a window of its line, the windows laid out by an
 * Array-OL tiler (origin, paving, fitting) over a repetition space of
 * independent elementary tasks (Sec. 3.A, "Downscaler Model").
 *
 * Readings of what the paper leaves open (identical in every entry point):
 *   - n_out = floor(n_in * p / q) on each axis; the same ratio on both
 *     axes unless a plan is created with ds_plan_create_ex;
 *   - output o = r*p + j (block r, phase j) is centred on input coordinate
 *     r*q + (j + 1/2) q/p - 1/2 and reads the K pixels
 *     r*q + b_j ... r*q + b_j + K - 1, b_j = floor(centre_j) - K/2 + 1,
 *     each clamped to the frame (clamp-to-edge; ds_plan_create_ex can take
 *     them modulo the frame instead, the Array-OL reading of tilers);
 *   - taps: Lanczos-3 stretched by 6/K over the window, normalised to sum 1,
 *     computed in FP64 on the host; FP32 copies for float data, Q14 integers
 *     (round half up, residual on the largest tap) for uint8 data;
 *   - FP32 / FP16 data: FP32 accumulation in tap order t = 0..K-1, FP32
 *     intermediate, FP16 output rounded to nearest even;
 *   - uint8 data: integer accumulation, (acc + 8192) >> 14 (floor shift) and
 *     clamp to [0,255] after each pass, so the intermediate is a uint8 frame.
 *
 * Memory layout of every frame: dense row-major, no pitch; channels
 * interleaved (DS_U8_RGB: R,G,B bytes per pixel).  A batch of n frames is n
 * such frames back to back.  `in` / `out` are DEVICE pointers owned by the
 * caller unless a function says otherwise.  All launches are asynchronous on
 * the given stream (a cudaStream_t passed as void*; NULL = legacy default
 * stream).  No entry point synchronises the device unless it says so.
 *
 * Errors: functions return DS_OK (0) or a negative ds_status; functions that
 * return a pointer return NULL.  The reason is in ds_last_error() (a
 * thread-local string, valid until the next call on the same thread).
 *
 * Environment: DS_LOG=1 logs each plan's choices and every error to stderr
 * (prefix "[ds] "), DS_LOG=2 also every launch (class, jobs, tiles, grid);
 * read once per process.  DS_NO_TMA=1 sends new plans to the general
 * kernels; DS_TUNE_CACHE names the autotuner's cache file (Python side).
 */
#ifndef DS_H
#define DS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ds_plan ds_plan; /* opaque, immutable after creation (tuning aside) */

/* Decimation ratio p/q: lowest terms, 0 < p < q, p <= 16, q <= 64. */
typedef struct {
    int p, q;
} ds_ratio;

/* Element type; the channel count is folded into it. */
typedef enum {
    DS_F32 = 0,    /* 1 channel, float                                  */
    DS_F16 = 1,    /* 1 channel, IEEE half; FP32 accumulation            */
    DS_U8 = 2,     /* 1 channel, uint8; Q14 taps                         */
    DS_U8_RGB = 3  /* 3 interleaved channels, uint8; Q14 taps            */
} ds_dtype;

typedef enum {
    DS_OK = 0,
    DS_ERR_ARG = -1,         /* invalid argument                              */
    DS_ERR_NOMEM = -2,       /* host or device allocation failed              */
    DS_ERR_CUDA = -3,        /* a CUDA runtime/driver call failed             */
    DS_ERR_TIMEOUT = -4,     /* a kernel gave up a bounded wait (device flag) */
    DS_ERR_UNSUPPORTED = -5, /* valid, but not supported by this build        */
    DS_ERR_BOUNDS = -6       /* a bounds check failed (DS_CHECK_BOUNDS build) */
} ds_status;

/* ---------------------------------------------------------------------- */
/* Plans                                                                    */
/* ---------------------------------------------------------------------- */

/*
 * Create a plan for frames of in_h x in_w pixels filtered at `ratio` with
 * `taps` (K) taps per phase (Sec. 3; Sec. 3.A for the tiler).  Host only:
 * computes the phase windows and the FP64 / FP32 / Q14 tap tables and picks
 * the kernel; no device memory is allocated and no kernel runs.
 * Errors (NULL + ds_last_error): in_h or in_w < 1; ratio not in lowest terms
 * or not in (0,1) or p > 16 or q > 64; taps odd or outside [2,16]; unknown
 * dtype; an output extent of 0.
 */
ds_plan* ds_plan_create(int in_h, int in_w, ds_ratio ratio, int taps, ds_dtype dtype);

/* Boundary of the tilers: clamp-to-edge (the default reading), or modular
 * indexing, the Array-OL reading of tilers (Sec. 3.A: pattern elements are
 * taken modulo the array's shape). */
typedef enum {
    DS_CLAMP = 0,
    DS_WRAP = 1
} ds_boundary;

/*
 * Extended plan: each axis has its own ratio and tap count, for instance
 * the paper's CIF case, 352 -> 132 per line (3/8) and 288 -> 128 lines
 * (4/9) (Sec. 3).  The tap tables may be given.
 *   weights_h / weights_v: NULL = the Lanczos-3 taps of ds_plan_create;
 *     else a row-major [p][taps] FP64 table of that axis, copied into the
 *     plan and used as given (rows need not sum to 1).  uint8 plans use its
 *     Q14 rounding: q = floor(w * 16384 + 1/2), with the residual
 *     floor(16384 * row sum + 1/2) - sum(q) added to the largest tap of
 *     the row.
 * DS_CLAMP plans whose axes form a fast class (equal ratio and taps at 3/8
 * K=8, 1/2 K=6 or 2/3 K=6; or uint8 with H 3/8 K=8, V 4/9 K=8) run on the
 * fast fused kernel, with given taps too (a launch then carries the plan's
 * own tables); every other plan runs on the general kernels.
 * Errors (NULL + ds_last_error): those of ds_plan_create per axis; an
 * unknown boundary; a given tap that is not finite; for uint8, a Q14 tap
 * outside the int16 range or a row whose Q14 magnitudes sum past 65535
 * (sums must stay exact in FP32).
 */
typedef struct {
    int in_h, in_w;
    ds_ratio ratio_h;          /* along a row: packets of q pixels -> p */
    int taps_h;
    ds_ratio ratio_v;          /* along a column                        */
    int taps_v;
    ds_dtype dtype;
    ds_boundary boundary;
    const double* weights_h;   /* NULL or [ratio_h.p][taps_h]           */
    const double* weights_v;   /* NULL or [ratio_v.p][taps_v]           */
} ds_plan_desc;

ds_plan* ds_plan_create_ex(const ds_plan_desc* desc);

/* Release a plan (the end of the life of the downscaler's filter tasks,
 * Sec. 3.A; the paper has no API, this is the plan lifecycle of the C ABI).
 * The caller must make sure no launch using it is still running (synchronise
 * the streams it was used on first).  NULL is ignored. */
void ds_destroy(ds_plan* plan);

/* The arguments the plan was created with (any pointer may be NULL); p, q
 * and taps are those of the horizontal axis (ds_plan_get_axes has both). */
ds_status ds_plan_get_params(const ds_plan* plan, int* in_h, int* in_w, int* p, int* q, int* taps,
                             int* dtype);

/* Ratio and taps of both axes and the boundary (any pointer may be NULL). */
ds_status ds_plan_get_axes(const ds_plan* plan, int* p_h, int* q_h, int* taps_h, int* p_v, int* q_v,
                           int* taps_v, int* boundary);

/* Output extent floor(in*p/q) per axis and the channel count: the shape of
 * the output array of the tiler (Sec. 3.A: 352 -> 132 per line at 3/8, the
 * output pattern of p elements per repetition).  DS_ERR_ARG on a NULL plan;
 * NULL output pointers are skipped. */
ds_status ds_plan_out_shape(const ds_plan* plan, int* out_h, int* out_w, int* channels);

/* Input / output bytes of one frame. */
ds_status ds_plan_frame_bytes(const ds_plan* plan, size_t* in_bytes, size_t* out_bytes);

/*
 * Copy the plan's tap tables, each row-major [p][K]; any pointer may be NULL.
 * fp64: the exact taps; fp32: (float) of fp64 (used by DS_F32 / DS_F16);
 * q14: the Q14 integers (used by DS_U8 / DS_U8_RGB).  Also returns the
 * window start b_j of each phase in `window_start` ([p] ints) if not NULL.
 */
ds_status ds_plan_get_taps(const ds_plan* plan, double* fp64, float* fp32, short* q14,
                           int* window_start);

/* The same for one axis: axis 0 = horizontal (as ds_plan_get_taps), 1 =
 * vertical.  DS_ERR_ARG for another axis. */
ds_status ds_plan_get_axis_taps(const ds_plan* plan, int axis, double* fp64, float* fp32, short* q14,
                                int* window_start);

/*
 * Describe the execution choice as a short JSON object written into buf
 * (truncated to len bytes, always NUL-terminated): kernel, tile shape,
 * rows per tile, CTAs per SM.
 */
ds_status ds_plan_describe(const ds_plan* plan, char* buf, size_t len);

/*
 * Tile schedule of the fused kernel (the "launch topology" the paper derives
 * from the task multiplicity, Sec. 3.B.1): row_blocks = output row blocks
 * per tile (each block is p output rows), ctas_per_sm = resident CTAs per SM
 * of the persistent grid (0 = as many as fit).  Used by the autotuner.
 * A new plan has a per-class default band and no fixed band: a launch whose
 * work would not fill the GPU's pipelines at that band (one frame, a small
 * batch) then runs shorter bands.  After ds_plan_set_schedule every launch
 * uses row_blocks as given.  Either way the last tiles of a launch (about
 * two per pipeline) run at a quarter of the band, which shortens the end of
 * the launch.  The schedule never changes the results, only the time.
 * DS_ERR_ARG for row_blocks < 1 or ctas_per_sm < 0.
 */
ds_status ds_plan_set_schedule(ds_plan* plan, int row_blocks, int ctas_per_sm);
ds_status ds_plan_get_schedule(const ds_plan* plan, int* row_blocks, int* ctas_per_sm);

/*
 * The whole schedule, with the tile shape (Sec. 3.B.1, as above).  Every fast
 * kernel class is compiled in ds_plan_tile_shapes(plan) tile shapes (the
 * pipeline depth of a warp's shared-memory ring and the resident warps its
 * registers are budgeted for; ds_plan_describe shows them); plans on the
 * general kernels have none (0) and take only shape 0.
 *   row_blocks: output row blocks per tile; 0 = the class default band,
 *     shortened for launches too small to fill the GPU;
 *   ctas_per_sm: resident CTAs per SM; 0 = as many as fit;
 *   shape: 0 .. ds_plan_tile_shapes(plan) - 1 (0 = the default shape).
 * DS_ERR_ARG on NULL, negative fields or a shape out of range.
 */
typedef struct {
    int row_blocks;
    int ctas_per_sm;
    int shape;
} ds_schedule;
int ds_plan_tile_shapes(const ds_plan* plan);
ds_status ds_plan_set_schedule_ex(ds_plan* plan, const ds_schedule* schedule);
ds_status ds_plan_get_schedule_ex(const ds_plan* plan, ds_schedule* schedule);

/*
 * Autotuner (the launch topology of Sec. 3.B.1, measured instead of derived
 * from thresholds): time ds_run_frames(plan, in, out, n_frames) with CUDA
 * events on `stream`, `iters` launches per candidate after one warm-up, over
 *   1. every tile shape at the default band,
 *   2. fixed bands at the best shape (against the default adaptive band),
 *   3. fewer resident CTAs per SM at the best shape and band,
 * and keep the fastest schedule in the plan.  The GPU is first kept busy
 * with the default schedule (shape 0, adaptive band, full occupancy) for
 * about 30 ms, the default is timed first, and a candidate replaces the best
 * so far only when it is more than 1 % faster; a winner other than the
 * default is re-timed against it, alternately, three times each, and kept
 * only if its median is still more than 1 % faster.  So the result is never
 * slower than the default as measured, and clock drifts or noise between
 * equivalent schedules do not change the choice.  Every candidate produces
 * identical bits.
 * `in` / `out` are the caller's device buffers for n_frames frames; they are
 * written (out) during tuning.  Synchronises the stream.
 * res (if not NULL): the best schedule, its time and the default's (us per
 * launch), and the number of candidates timed.
 * ds_plan_autotune is the same with the band and time of the result only.
 * DS_ERR_ARG on NULL pointers, n_frames < 1 or iters < 1; on any other
 * failure the plan keeps the schedule it had.
 */
typedef struct {
    ds_schedule best;
    float best_us;
    float default_us;
    int candidates;
} ds_tune_result;
ds_status ds_plan_autotune_ex(ds_plan* plan, const void* in, void* out, int n_frames, void* stream,
                              int iters, ds_tune_result* res);
ds_status ds_plan_autotune(ds_plan* plan, const void* in, void* out, int n_frames, void* stream,
                           int iters, int* best_row_blocks, float* best_us);

/* ---------------------------------------------------------------------- */
/* Running                                                                  */
/* ---------------------------------------------------------------------- */

/*
 * Filter one frame (the downscaler's filter stage, Sec. 3: the horizontal
 * filter over every line, then the vertical filter over every column, each
 * a repetition of the Array-OL tiler of Sec. 3.A): in (in_h x in_w x C
 * elements) -> out (out_h x out_w x C), both passes fused in one kernel; the
 * intermediate stays on chip.  in and out must not overlap.
 * Fused launches take tile-scheduling counters from a ring of 512 slots; a
 * slot is reused only once the launch that last used it has completed (the
 * call waits for one when all 512 are in flight).  A fused launch inside a
 * stream capture that the caller started is refused (DS_ERR_UNSUPPORTED):
 * capture with ds_graph_create instead.
 * DS_ERR_ARG: NULL plan / pointer.  DS_ERR_CUDA: launch failure.
 */
ds_status ds_run(const ds_plan* plan, const void* in, void* out, void* stream);

/* Filter n_frames frames stored back to back (one launch; the frames are the
 * independent repetitions of the paper's task over its video, Sec. 3.A). */
ds_status ds_run_frames(const ds_plan* plan, const void* in, void* out, int n_frames,
                        void* stream);

/* One job of a batch: a frame (or n_frames frames back to back) of one plan. */
typedef struct {
    const ds_plan* plan;
    const void* in;
    void* out;
    int n_frames; /* 0 is read as 1 */
} ds_job;

/*
 * Filter a batch of jobs of any mix of plans (sizes, ratios, dtypes): the
 * repetitions of every job's tasks (Sec. 3.A) in one persistent launch per
 * kernel class and tile shape (one fast class = one dtype and one ratio and
 * tap count per axis); jobs whose plan needs the general kernel get their
 * own launches on the same stream.  Job descriptors travel in the launch parameters: no
 * device memory is allocated.  Batches beyond the per-launch descriptor limit
 * are split into several launches.  DS_ERR_ARG: n < 0, NULL jobs with n > 0,
 * NULL plan or pointer in a job.
 */
ds_status ds_batch_run(const ds_job* jobs, int n, void* stream);

/*
 * Autotuner of a batch (the launch topology of Sec. 3.B.1 for the whole
 * video's repetitions at once, measured instead of derived from
 * thresholds): as ds_plan_autotune_ex, but it times ds_batch_run(jobs, n,
 * stream) and applies each candidate to every fused-kernel plan of the
 * batch.  Tiles of all the batch's jobs share one launch per kernel class,
 * so a plan tuned alone does not see the others' tiles, bands or tail.  The
 * candidates: every tile shape that all those plans have, at the default
 * band; fixed bands at the best shape, up to the tallest plan's block rows;
 * then fewer resident CTAs per SM (one or two fewer, three quarters, half of
 * what fits each plan's kernel).  The same warm-up, 1 % margin and
 * alternating confirmation against the default keep the result no slower
 * than the default as measured.  The jobs' plans keep the chosen schedule
 * (a plan that also serves other batches runs those at it too); plans on the
 * general kernels keep theirs.  Output buffers are written during tuning.
 * Synchronises the stream.  res (if not NULL): the first fused plan's
 * schedule, the batch's time at the best schedule and at the default (us per
 * batch), and the number of candidates timed.  DS_ERR_ARG on NULL pointers,
 * n < 1 or iters < 1; DS_ERR_UNSUPPORTED when no job runs on the fused
 * kernel; on any other failure the plans keep the schedules they had.
 */
ds_status ds_batch_autotune(const ds_job* jobs, int n, void* stream, int iters, ds_tune_result* res);

/*
 * The unfused two-kernel form: a horizontal kernel writes the intermediate
 * (FP32 for float dtypes, uint8 for uint8 dtypes) to `workspace` in device
 * memory, a vertical kernel reads it back.  Same results as ds_run, bit for
 * bit.  workspace_bytes must be at least ds_plan_workspace_bytes(plan) *
 * n_frames.  DS_ERR_ARG otherwise.
 */
size_t ds_plan_workspace_bytes(const ds_plan* plan);
ds_status ds_run_unfused(const ds_plan* plan, const void* in, void* out, int n_frames,
                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * The unfused form without caller workspace, for callers that cannot
 * allocate device memory on the call path (a serving loop that must not stall
 * on cudaMalloc, an application with a device memory budget fixed at start-up,
 * a host program whose own allocator must own the device).  The paper has no
 * counterpart; this is a deployment variant of ds_run_unfused.
 * The intermediate lives in one fixed device array of
 * ds_static_workspace_bytes() (32 MiB) per GPU, held until the process exits;
 * the call allocates nothing.  DS_ERR_ARG when the plan's intermediate for
 * n_frames frames (ds_plan_workspace_bytes * n_frames) exceeds it.
 * The first call on a device looks up the array's device address (host
 * set-up, no allocation): make that first call before any stream capture.
 * The address is then kept for the life of the process; after
 * cudaDeviceReset (or anything else that tears down the device's primary
 * context) it is no longer valid, and this entry point must not be called
 * again in that process.
 * All calls share the array and it keeps the last call's contents (every
 * value a call reads it has written first); calls whose launches overlap on
 * the GPU -- on different streams or from different host threads -- race on
 * it and must be serialised by the caller.
 */
size_t ds_static_workspace_bytes(void);
ds_status ds_run_unfused_static(const ds_plan* plan, const void* in, void* out, int n_frames,
                                void* stream);

/*
 * Synchronise `stream` and read the device status word that kernels set
 * when a bounded wait gives up (or, in a DS_CHECK_BOUNDS build, when one of
 * the kernel's own bounds checks fails); the word is cleared by the read.
 * DS_ERR_TIMEOUT or DS_ERR_BOUNDS (what failed, and where, in
 * ds_last_error()) if it was set, DS_ERR_CUDA on an asynchronous CUDA error.
 */
ds_status ds_stream_check(void* stream);

/*
 * 1 if this library was built with DS_CHECK_BOUNDS: the fused kernel then
 * checks every shared-memory row read, border write, tensor copy and output
 * row against its buffer, and a failed check skips the access and sets the
 * device status word (see ds_stream_check).  0 for the normal build.
 */
int ds_bounds_checked(void);

/*
 * Test of the bounds-check report (DS_CHECK_BOUNDS builds): launch on
 * `stream` one warp that runs the kernels' check on an offset one past a
 * 64-byte buffer (no access is made), so the next ds_stream_check returns
 * DS_ERR_BOUNDS.  DS_ERR_UNSUPPORTED in the normal build.
 */
ds_status ds_debug_bounds_probe(void* stream);

/*
 * Test of the timeout path: launch on `stream` one warp that waits, with the
 * fused kernel's bounded wait, on an mbarrier that nothing completes (no
 * copy is issued, no thread arrives).  After limit_cycles SM clock cycles
 * (2.03e6 per ms at the B300's clock) it gives up and sets the device status
 * word, so the next ds_stream_check returns DS_ERR_TIMEOUT and the context
 * stays usable.  DS_ERR_ARG for a limit outside [0, 4e9].
 */
ds_status ds_debug_timeout_probe(long long limit_cycles, void* stream);

/*
 * Host-only self-check of the fused kernel's tile schedule for this plan:
 * walks every tile of a frame with the kernel's own index arithmetic and
 * verifies that TMA coordinates are aligned, every shared-memory read stays
 * inside the loaded window and never straddles a box, border pixels are
 * fixed up before use, the row stream delivers each frame row in order, the
 * register window holds exactly the (clamped) rows of every output block,
 * and every output element is written exactly once.  No device work.
 * DS_OK, or DS_ERR_ARG with the first violation in ds_last_error().  Plans
 * without a fast kernel: DS_OK.
 */
ds_status ds_debug_check_plan(const ds_plan* plan);

/* ---------------------------------------------------------------------- */
/* CUDA graphs                                                              */
/* ---------------------------------------------------------------------- */

typedef struct ds_graph ds_graph;

/*
 * Capture ds_batch_run(jobs, n, .) into a CUDA graph and instantiate it; the
 * job pointers are baked in.  NULL on error.  ds_graph_launch replays it on
 * `stream` (one graph launch for the whole batch; replays of one graph are
 * serialised by CUDA).  Each captured fused launch holds one of 512 tile-
 * scheduling slots until ds_graph_destroy, which must be called after the
 * graph's launches have completed; DS_ERR_UNSUPPORTED (NULL) when live graphs
 * hold all of them.  Direct launches share the other 512 slots round robin,
 * so at most 512 fused launches may be in flight at once.
 */
ds_graph* ds_graph_create(const ds_job* jobs, int n);
ds_status ds_graph_launch(ds_graph* graph, void* stream);
void ds_graph_destroy(ds_graph* graph);

/* ---------------------------------------------------------------------- */
/* End-to-end pipeline with host buffers                                    */
/* ---------------------------------------------------------------------- */

typedef struct ds_pipeline ds_pipeline;

/*
 * A host-to-host pipeline for one plan: frames are copied host -> device,
 * filtered and copied device -> host in chunks of `chunk_frames`, with
 * `depth` chunks in flight on separate streams so that copies in both
 * directions overlap the kernels (the transfer cost the paper measures in
 * Sec. 4).  Owns its device staging buffers and streams.  NULL on error.
 */
ds_pipeline* ds_pipeline_create(const ds_plan* plan, int chunk_frames, int depth);

/*
 * Filter n_frames frames from host memory `in` into host memory `out` and
 * wait for completion.  Page-locked (pinned) host buffers give overlapped
 * copies; pageable memory works but serialises.  DS_ERR_ARG on NULL.
 */
ds_status ds_pipeline_run(ds_pipeline* pipe, const void* in, void* out, int n_frames);
void ds_pipeline_destroy(ds_pipeline* pipe);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of single-frame requests                    */
/* ---------------------------------------------------------------------- */

/*
 * A request loop over a stream of frames (the paper applies its downscaler
 * to a video, frame after frame, and measures the whole application,
 * transfers included, Sec. 4; the paper has no serving API, this is the
 * C ABI's).  A request is one frame of any plan.  ds_server_run admits
 * queued requests while a stream slot is free and their bytes fit the
 * memory budget, launches each admitted group as one ds_batch_run on the
 * slot's stream, and keeps admitting as slots and memory free up, so groups
 * overlap on the device.  Plans stay resident in the caller's hands; the
 * server owns its streams, events and (copy mode) one device arena per slot.
 * The request path allocates nothing.
 *
 * ds_server_create: budget in bytes (inputs plus outputs of the admitted
 * requests; in the copy mode split into n_streams equal arenas, allocated at
 * the first copy-mode run), 1..64 stream slots, at most max_batch requests
 * per group.  NULL on error.  ds_server_destroy waits for its streams.
 */
typedef struct ds_server ds_server;

typedef struct {
    const ds_plan* plan;
    const void* in;    /* one frame: device memory, or host memory with DS_SERVE_COPIES (pinned
                          memory overlaps the copies) */
    void* out;         /* likewise */
    double arrival_s;  /* seconds after the start of the run (with DS_SERVE_REALTIME) */
} ds_request;

typedef struct {
    int completed, batches, max_batch, max_queue;
    long long launches;          /* kernel launches made by the run */
    double wall_s;
    size_t peak_admitted_bytes;
} ds_serve_stats;

enum {
    DS_SERVE_REALTIME = 1, /* requests arrive at their arrival_s; else all at once (saturation) */
    DS_SERVE_COPIES = 2,   /* in / out are host buffers: H2D copy, kernels, D2H copy per group */
    DS_SERVE_PLAIN = 4     /* the baseline: one plain fused launch per request on one stream */
};

ds_server* ds_server_create(size_t mem_budget_bytes, int n_streams, int max_batch);

/*
 * Serve n requests and return when all have completed.  latency_ms (NULL or
 * [n]): arrival -> observed completion of each request, in milliseconds
 * (with DS_SERVE_PLAIN: the end of the run, which waits once).  stats (NULL
 * or one): counts, the wall time and the launches.  DS_ERR_ARG for NULL
 * buffers, unknown flags or a request larger than the budget (copy mode:
 * than a slot's arena); DS_ERR_NOMEM if the arenas cannot be allocated;
 * DS_ERR_CUDA if a launch or copy fails (in-flight work is waited for
 * before returning).
 */
ds_status ds_server_run(ds_server* server, const ds_request* reqs, int n, int flags, double* latency_ms,
                        ds_serve_stats* stats);
void ds_server_destroy(ds_server* server);

/* ---------------------------------------------------------------------- */
/* Misc                                                                     */
/* ---------------------------------------------------------------------- */

/* Thread-local message of the last failure on this thread ("" if none).
 * Error reporting of the C ABI; the paper has no API. */
const char* ds_last_error(void);

/* Library version string. */
const char* ds_version(void);

/* Number of kernel launches this library made on this host thread since the
 * last call (the counter is reset by the call). */
long long ds_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* DS_H */
