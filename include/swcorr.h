/*
 * swcorr.h -- C ABI of the GB300 sliding-window inter-channel correlation
 * library (libswcorr.so).
 *
 * The library computes, for two equal-size grids x and y (Poyda & Zhizhin,
 * arXiv:1807.06507, Section 3: "both sets of data must be the same size"),
 * the Pearson correlation of every sliding window (Introduction, Eq. 1)
 * through the sums form (Section 1, Eq. 2):
 *
 *     c = (n Sxy - Sx Sy) / ( sqrt(n Sxx - Sx^2) * sqrt(n Syy - Sy^2) )
 *
 * with the five window sums Sx, Sy, Sxx, Syy, Sxy obtained by separable
 * sliding summation, one pass per dimension (Section 1, steps 1-4 and the
 * n-dimensional generalisation).  The result for a window is written to the
 * window's middle cell (Section 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Dimensions are listed outermost first (C order): for a 2-D grid
 *   shape = {rows, cols}, for 3-D {planes, rows, cols}; the last dimension
 *   is contiguous in memory.
 * - Window: k[d] cells along dimension d, centred: output centre i covers
 *   [i - floor((k-1)/2), i + floor(k/2)].  Border rule SWCORR_BORDER_CLIP:
 *   the window is clipped to the grid and n is the number of in-bounds cells
 *   (the paper writes -2 at borders instead; that mode is not provided).
 * - Stride ("step of the window", Introduction): output j has centre
 *   j * stride[d]; the output has ceil(shape[d] / stride[d]) cells per
 *   dimension.
 * - A window whose x (or y) values are all equal has zero variance and
 *   yields NaN.  This is the paper's equality check (Section 3, accuracy
 *   discussion), decided exactly.
 * - Results are float32 and clamped to [-1, 1].
 * - Pitches are in ELEMENTS per dimension (in_pitch[d] = distance between
 *   consecutive indices of dimension d); pitch[ndim-1] must be 1.  NULL means
 *   contiguous.
 *
 * Numerics
 * --------
 * - SWCORR_U16: the five sums are exact integers; c is evaluated from them
 *   with float32 rounding only in the last steps (|error| < 1e-6).
 * - SWCORR_F32: each input value is first offset by a per-block reference
 *   and rounded to a fixed-point grid of 2^-22 times the block's value range;
 *   from there on the sums are exact integers.  Integer-valued data whose
 *   block range is below 2^22 is represented exactly.
 *
 * Memory ownership and errors
 * ---------------------------
 * The caller owns every data buffer and keeps it alive until the work queued
 * on the given stream has completed.  The library owns plans (tensor-map
 * cache, a small device status block, staging buffers for host runs).
 * No call throws; each returns a status and records a detail message that
 * swcorr_last_error() returns (per thread).  Launch errors are reported
 * synchronously by the run call; device-side errors (a bounded wait that ran
 * out) are latched in the plan's status block and reported by
 * swcorr_plan_status() after the stream has been synchronised.
 *
 * Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 * default stream).
 */
#ifndef SWCORR_H
#define SWCORR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SWCORR_OK = 0,
  SWCORR_ERR_INVALID_ARG = 1, /* a shape, window, stride, pointer or pitch is invalid */
  SWCORR_ERR_UNSUPPORTED = 2, /* valid but not provided (e.g. ndim > 3, kw > 31) */
  SWCORR_ERR_ALIGNMENT = 3,   /* base address or pitch not 16-byte aligned */
  SWCORR_ERR_CUDA = 4,        /* a CUDA runtime/driver call failed */
  SWCORR_ERR_OOM = 5,         /* the library could not allocate what it needs */
  SWCORR_ERR_TIMEOUT = 6,     /* a bounded device wait gave up (kernel returned early) */
  SWCORR_ERR_NO_DEVICE = 7    /* no usable sm_103 device */
} swcorr_status;

typedef enum { SWCORR_U16 = 1, SWCORR_F32 = 2 } swcorr_dtype;

/* Border rule.
 *   SWCORR_BORDER_CLIP  : windows are clipped to the grid; n is the number of
 *                         in-grid cells (a reading: the paper writes -2 there).
 *   SWCORR_BORDER_PAPER : the paper's result convention (Section 3, the
 *                         paragraph on the result set): a window that reaches
 *                         past an edge of the grid gives -2, and so does a
 *                         window holding a missing value (a value <= -999) in
 *                         x or in y; other windows as with CLIP (they are whole).
 *                         1-D to 3-D: the fused kernel, then a pass that
 *                         writes the -2 outputs (the output must then be
 *                         contiguous); other plans: the general n-D path. */
typedef enum { SWCORR_BORDER_CLIP = 0, SWCORR_BORDER_PAPER = 1 } swcorr_border;

enum {
  /* Also write the five window sums (int64: Sx, Sy, Sxx, Syy, Sxy per output,
   * output-major, C order of the output grid) to the sums buffer passed to
   * swcorr_run: the exact integer sums of Section 1, steps 1-3.  uint16
   * plans with clipped windows (every kernel: 1-D, 2-D, 3-D and the general
   * path). */
  SWCORR_FLAG_EMIT_SUMS = 1u,
  /* Test hook for the failure path (not part of the paper's method): in a
   * 2-D uint16 plan whose inputs are read by TMA, the work item of the first
   * strip and row block announces its first row's copy but never issues it.
   * That warp's bounded wait gives up after about a second, it drains its
   * other copies and returns, and swcorr_plan_status reports
   * SWCORR_ERR_TIMEOUT; every other item completes normally and the context
   * stays usable.  Outputs of the stalled item are undefined. */
  SWCORR_FLAG_TEST_STALL = 2u,
  /* Ablation of the alternative the paper rejects (Section 1, last
   * paragraph): window sums from cumulative (summed-area) sums along every
   * dimension, by inclusion-exclusion over the window's corners, instead of
   * sliding sums.  Results are identical (the sums are exact modular
   * integers); only the cost differs.  Served by the general n-D path. */
  SWCORR_FLAG_SAT = 4u,
  /* Ablation of the fusion: run the general path (the paper's scheme of
   * Sections 1-2: products and sums materialised in device memory, one pass
   * per dimension) instead of the fused 1-D/2-D/3-D kernel.  Same results up
   * to float32 rounding (a float32 grid gets one fixed-point map instead of
   * one per block); only the cost differs. */
  SWCORR_FLAG_UNFUSED = 8u
};

typedef struct swcorr_plan_s* swcorr_plan;

/* Create a plan for one problem shape (the windowed correlation of two
 * equal-size grids, Section 3: both data sets have the same size; window
 * size and step, Introduction).
 *   out    : receives the plan (set to NULL on failure).
 *   ndim   : 1 to 8.  1-D, 2-D and 3-D grids run one fused kernel
 *            (Section 1, steps 1-4 in one pass over HBM; under the paper's
 *            border rule followed by a pass that writes the -2 outputs); more
 *            dimensions, SWCORR_FLAG_SAT and SWCORR_FLAG_UNFUSED run the
 *            general path (the steps as separate passes over materialised
 *            sums, one per dimension: Section 1's n-dimensional
 *            generalisation, Section 2's parallel phases).
 *   shape  : ndim extents, each >= 1 and at most 2^31 - 1024.
 *   k      : ndim window sizes, each >= 1 (an even k gives the window
 *            [i - k/2 + 1, i + k/2]).  The fused 2-D kernel takes odd widths
 *            up to 31 in the contiguous dimension, the fused 3-D one equal
 *            odd row and column sizes up to 15; uint16 windows of the fused
 *            kernels hold at most 32768 in-bounds cells.  Any other window
 *            shape runs on the general path (same results).
 *   stride : ndim steps >= 1, or NULL for all ones (Introduction: "given
 *            step").
 *   dtype  : SWCORR_U16 or SWCORR_F32 (x and y share it).
 *   border : SWCORR_BORDER_CLIP or SWCORR_BORDER_PAPER.
 *   flags  : SWCORR_FLAG_* bits.
 * Host-only work plus device attribute queries and the plan's device
 * allocations (a status block; the general path's sum buffers, 2 x 5 or 6
 * int64 per cell); no kernel is launched.  The plan owns its memory until
 * swcorr_plan_destroy. */
swcorr_status swcorr_plan_create(swcorr_plan* out, int ndim, const int64_t* shape,
                                 const int32_t* k, const int32_t* stride, swcorr_dtype dtype,
                                 swcorr_border border, uint32_t flags);

/* Launch parameters of a plan, as chosen by the autotuner (support
 * component; no counterpart in the paper).  0 in a field = the library's
 * built-in default.
 *   prefetch    : rows (2-D) in flight ahead of the row being summed: the
 *                 depth of the shared-memory staging ring (1..8).
 *   tile_rows   : least output rows (2-D) or planes (3-D) per work item, the
 *                 height of a tile; the halo of kh - 1 rows is re-read per
 *                 tile, so taller tiles read less but make fewer items.
 *   ctas_per_sm : cap on resident one-warp CTAs per SM used to size the
 *                 persistent grid (never above the kernel's occupancy).
 * Results do not depend on these values (uint16 results are bit-identical;
 * float32 results can differ in the last bits because the fixed-point
 * reference of a lane follows its tile). */
enum {
  SWCORR_TUNE_MAX_PREFETCH = 8,
  SWCORR_TUNE_MAX_TILE_ROWS = 4096,
  SWCORR_TUNE_MAX_CTAS_PER_SM = 32
};
typedef struct {
  int32_t prefetch;
  int32_t tile_rows;
  int32_t ctas_per_sm;
  int32_t reserved[5]; /* must be 0 */
} swcorr_tune;

/* swcorr_plan_create with explicit launch parameters (tune != NULL) instead
 * of the tune cache's entry for this device, ndim, dtype and k.  Values
 * outside the ranges above give SWCORR_ERR_INVALID_ARG.  Used by the
 * autotuner to time candidates.  No counterpart in the paper. */
swcorr_status swcorr_plan_create_tuned(swcorr_plan* out, int ndim, const int64_t* shape,
                                       const int32_t* k, const int32_t* stride, swcorr_dtype dtype,
                                       swcorr_border border, uint32_t flags, const swcorr_tune* tune);

/* The launch parameters a plan uses (after defaults and the cache).  No
 * counterpart in the paper.  SWCORR_ERR_INVALID_ARG for a NULL argument. */
swcorr_status swcorr_plan_tune(swcorr_plan p, swcorr_tune* out);

/* Tune cache: a JSON file ({"format": "swcorr-tune-1", "entries": [...]},
 * written by paper_1807_06507_gb300/autotune.py) that swcorr_plan_create and
 * swcorr_plan_batched consult.  This call (re)reads `path` (NULL or "": no
 * cache).  Without it, the first plan reads the file named by the
 * SWCORR_TUNE_FILE environment variable, if set.  A file that cannot be read
 * or does not parse is ignored as a whole (SWCORR_ERR_INVALID_ARG here, the
 * built-in defaults apply).  Thread-safe; plans already created keep their
 * parameters.  No counterpart in the paper. */
swcorr_status swcorr_set_tune_file(const char* path);

/* Cache lookup without a device (tests, tools): 1 and *out filled if the
 * loaded cache has an entry for (device, kind, ndim, k, dtype), else 0.
 * device NULL matches any device; batched != 0 looks up the batched plan's
 * entry (k ignored).  No counterpart in the paper. */
int swcorr_tune_lookup(const char* device, int batched, int ndim, const int32_t* k, swcorr_dtype dtype,
                       swcorr_tune* out);

/* Queue the correlation of device buffers x, y into device buffer c: for
 * every output window the five sums of x, y, x^2, y^2 and xy (Section 1,
 * steps 1-3) and Pearson's c from them (Section 1, Eq. 2: the sums form of
 * the classical formula of the Introduction), NaN for a window whose x or y
 * values are all equal (Section 3, accuracy paragraph), clamped to [-1, 1].
 *   x, y      : device pointers, 16-byte aligned, plan dtype.
 *   in_pitch  : ndim element pitches for x and y, or NULL (contiguous); the
 *               byte pitch of every outer dimension must be a multiple of 16.
 *   c         : device float32 output, ceil(shape[d]/stride[d]) per dim.
 *   out_pitch : ndim element pitches for c, or NULL (contiguous).
 *   sums      : device int64 buffer of 5 * (number of outputs) entries when the
 *               plan has SWCORR_FLAG_EMIT_SUMS, else NULL.
 *   stream    : cudaStream_t.
 * Returns after queuing (asynchronous).  Argument errors are returned
 * synchronously (SWCORR_ERR_INVALID_ARG, SWCORR_ERR_ALIGNMENT); device-side
 * ones are read with swcorr_plan_status after the stream has synchronised.
 * The caller owns x, y, c and sums and keeps them alive until the stream
 * work completes. */
swcorr_status swcorr_run(swcorr_plan p, const void* x, const void* y, const int64_t* in_pitch,
                         float* c, const int64_t* out_pitch, int64_t* sums, void* stream);

/* Same computation from HOST buffers (the paper's GPU timing in Section 3
 * includes the copies to and from the device; this call is that whole
 * job): copies x and y to plan-owned device
 * staging buffers, runs, copies c back and synchronises the stream.  Host
 * buffers are contiguous; pinned memory gives the fastest copies.  The plan
 * allocates its staging buffers on the first call (SWCORR_ERR_OOM on failure).
 * 2-D plans pipeline the copies and kernels over bands of rows.  When x, y
 * and c are all page-locked, that pipeline is recorded once as a CUDA graph
 * for those three pointers and replayed by later calls with the same
 * pointers (their contents are read at each call); other pointers record a
 * new graph.  In that case the kernels store c directly through its device
 * mapping (zero-copy) instead of a staging buffer and a copy back; c must
 * then not be read or written by the host until the call returns.  A plan is
 * not to be run from two host threads at once. */
swcorr_status swcorr_run_host(swcorr_plan p, const void* x, const void* y, float* c, void* stream);

/* One scene of a batched plan: one 2-D pair of channels of the paper's
 * all-windows correlation (Section 3), as many scenes of uneven sizes and
 * window shapes are correlated in one launch.  All scenes of a plan have the
 * plan's dtype (uint16 or float32); windows are square or rectangular
 * (k[0] rows, k[1] cols, k[1] odd and <= 31), stride 1, the clipped border.
 * Pointers are device pointers that must stay valid for every
 * swcorr_run_batched call on the plan. */
typedef struct {
  int64_t shape[2];     /* rows, cols */
  int32_t k[2];         /* window rows, cols */
  const void* x;        /* device, 16-byte aligned */
  const void* y;        /* device, 16-byte aligned */
  int64_t in_pitch;     /* elements between rows of x and y (>= cols; pitch in bytes a multiple of 16) */
  float* c;             /* device output, rows x cols */
  int64_t out_pitch;    /* elements between rows of c (>= cols) */
} swcorr_scene;

/* Plan one persistent launch over all scenes' tiles (a work queue ordered
 * largest-cost first; one kernel per class of window width), captured in a
 * CUDA graph on first run.  Copies the scene table; dtype is SWCORR_U16 or
 * SWCORR_F32 for every scene, with the same numerics as swcorr_run on that
 * dtype (float32: per-window certificate and exact recomputation).  flags
 * must be 0.  Errors: SWCORR_ERR_INVALID_ARG (NULL, bad shape or window,
 * pitch below the row), SWCORR_ERR_ALIGNMENT (base or row pitch not 16-byte
 * aligned), SWCORR_ERR_UNSUPPORTED (even or > 31 window width, uint16
 * windows above 32768 cells), SWCORR_ERR_OOM. */
swcorr_status swcorr_plan_batched(swcorr_plan* out, const swcorr_scene* scenes, int n_scenes,
                                  swcorr_dtype dtype, uint32_t flags);

/* swcorr_plan_batched with explicit launch parameters (see swcorr_tune;
 * tile_rows is the least number of output rows per work item).  No
 * counterpart in the paper. */
swcorr_status swcorr_plan_batched_tuned(swcorr_plan* out, const swcorr_scene* scenes, int n_scenes,
                                        swcorr_dtype dtype, uint32_t flags, const swcorr_tune* tune);

/* Launch the batched plan on a stream (graph launch; asynchronous).  The
 * paper correlates one scene per run; batching many is this library's
 * scheduling, with no counterpart in the paper.  SWCORR_ERR_INVALID_ARG
 * for a plan that is not batched. */
swcorr_status swcorr_run_batched(swcorr_plan p, void* stream);

/* Device-side status latched by the plan's kernels (read after the stream
 * has synchronised; reading resets it).  SWCORR_OK if nothing went wrong,
 * SWCORR_ERR_TIMEOUT if a bounded wait gave up (that work item's outputs are
 * undefined).  No counterpart in the paper. */
swcorr_status swcorr_plan_status(swcorr_plan p);

/* Diagnostic: number of windows the plan's kernels computed again since the
 * last call (uint16: windows whose second-moment sums could not be
 * certified below 2^32, recomputed exactly; float32: windows rewritten by
 * the second tier, which re-marches a lane or item whose fixed-point map
 * left a window uncertified, plus windows recomputed from their own cells);
 * reading resets it.  -1 on error.  No counterpart in the paper. */
int64_t swcorr_plan_fallbacks(swcorr_plan p);

/* No-allocation 2-D uint16 run, for callers that cannot allocate device
 * memory: code whose device memory is owned by its own pool allocator under a
 * fixed budget (e.g. a framework that reserved the GPU's memory up front), and
 * latency-critical loops that must not call cudaMalloc/cudaFree because those
 * calls can synchronise the whole device.  The paper has no counterpart: this
 * is a deployment variant of swcorr_run for a 2-D uint16 plan with stride 1,
 * computing the same results with the same kernel, but without a plan.
 *   rows, cols : grid size; kh, kw: window (kw odd, 1..31).
 *   x, y       : device uint16 grids (2-byte aligned); in_pitch elements
 *                between rows (<= 0 means cols).  c: device float32 output
 *                (4-byte aligned), out_pitch elements between rows (<= 0
 *                means cols).  stream: cudaStream_t.
 * The kernel's scratch (its status words) lives in a 256-byte file-scope
 * __device__ array of the library instead of a cudaMalloc'd block; every GPU
 * that loads the library holds that array until the process exits.  The
 * call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine); it rejects sizes beyond its limits (rows or cols > 2^31 - 1024,
 * or a kernel scratch larger than the array) with SWCORR_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  The
 * address is kept for the process: after cudaDeviceReset() on a device, do
 * not use this call on that device again.  Every call shares the array and
 * clears its status words before launching, so calls whose work overlaps on
 * the GPU (different streams, no ordering between them) race on it.
 * Asynchronous: returns after queuing.  Device-side errors (a bounded wait
 * that gave up, leaving outputs of that work item undefined) are not
 * reported here: read them with swcorr_noalloc_status. */
swcorr_status swcorr_run2d_u16_noalloc(int64_t rows, int64_t cols, int32_t kh, int32_t kw, const void* x,
                                       const void* y, int64_t in_pitch, float* c, int64_t out_pitch,
                                       void* stream);

/* Status of the no-allocation runs queued on `stream` since the last call:
 * waits for the stream, copies the status words out of the static array
 * (into host memory on the call's stack; nothing is allocated), clears them,
 * and returns SWCORR_ERR_TIMEOUT if a kernel's bounded wait gave up, else
 * SWCORR_OK.  *fallbacks (if not NULL) receives the number of windows the
 * kernel recomputed through its exact per-window path (-1 on error).  The
 * paper has no counterpart. */
swcorr_status swcorr_noalloc_status(void* stream, int64_t* fallbacks);

/* Number of output windows the plan computes per run (the product of
 * ceil(shape[d] / stride[d])).  -1 for NULL. */
int64_t swcorr_plan_outputs(swcorr_plan p);

/* Release a plan (NULL is ignored).  Waits for nothing: the caller must have
 * synchronised the streams the plan ran on.  No counterpart in the paper. */
void swcorr_plan_destroy(swcorr_plan p);

/* Name of a status code (static string).  No counterpart in the paper. */
const char* swcorr_status_string(swcorr_status s);

/* Detail text of the last failing call on this thread ("" if none).  No
 * counterpart in the paper. */
const char* swcorr_last_error(void);

/* Library version, e.g. "swcorr 0.1.0 sm_103a".  No counterpart in the
 * paper. */
const char* swcorr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWCORR_H */
