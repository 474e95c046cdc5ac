/*
 * swift.h -- C ABI of the GB300 (sm_103a) SWiFT-IR block-matching library.
 *
 * The library computes the "swim" matching step of SWiFT-IR (Wetzel et al.,
 * Sec. III): for each pair of apodised match windows, the forward 2D
 * transforms of both windows, their frequency-domain product with its
 * amplitudes rescaled by a power-law whitening exponent (phases untouched),
 * the inverse transform (the pixel-level match response of Fig. 2), the peak
 * of that response (the relative shift), the peak's signal-to-noise ratio as a
 * Z score against the background, and a subpixel peak position.
 *
 * Every step runs in this library's own CUDA kernels; there is no CPU path.
 *
 * Conventions shared by every entry point
 *   - All image, origin, level, affine and result arrays are DEVICE pointers
 *     owned by the caller.  A plan owns only its tables and its workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and do not synchronise the host.
 *   - Argument errors are detected on the host before any launch and return a
 *     status other than SWIFT_OK with nothing written.  Launch failures return
 *     SWIFT_ERR_CUDA.  Per-window data problems are reported in
 *     swift_result.status, never as a call error.
 *   - The calls of one plan share its workspace, so they are ordered among
 *     themselves on the device: a call made on a stream other than the
 *     plan's previous call first makes its stream wait for that call's work
 *     (an event the plan records after every call).  Calls captured into a
 *     CUDA graph are not ordered this way; swift_plan_replay orders the
 *     replays.  A plan is not thread-safe.  No entry point throws.
 */
#ifndef SWIFT_H_
#define SWIFT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SWIFT_OK = 0,
  SWIFT_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is invalid      */
  SWIFT_ERR_UNSUPPORTED = 2, /* valid, but not built (e.g. a window size)    */
  SWIFT_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed         */
  SWIFT_ERR_OOM = 4,         /* a plan table could not be allocated          */
  SWIFT_ERR_TIMEOUT = 5,     /* a device-side bounded wait gave up           */
  SWIFT_ERR_CAPACITY = 6     /* more windows than swift_match_batch_noalloc's
                                static scratch holds                         */
} swift_status;

/* Apodisation: the paper's cosine taper (Sec. III, "apodization").  HANN is
 * the periodic Hann window, a[k] = (1 - cos(2 pi k / n)) / 2, and equals
 * TUKEY with alpha = 1; TUKEY(alpha) is flat in the middle with raised-cosine
 * ramps of alpha*n/2 samples at each edge.  The 2D taper is a[y] a[x]. */
typedef enum { SWIFT_APOD_NONE = 0, SWIFT_APOD_HANN = 1, SWIFT_APOD_TUKEY = 2 } swift_apod;

/* Element type of the input images. */
typedef enum { SWIFT_IN_U8 = 0, SWIFT_IN_F32 = 1 } swift_dtype;

/* Arithmetic of the transforms.  FP32 is the plain form (radix-16/8
 * butterflies on the FP32 units).  BF16X2 and FP16X2 compute every 1D DFT
 * on the tensor cores, one warp per transform, by the four-step
 * factorisation n = 16 x (n/16): both small DFTs are mma.sync products with
 * operands split into hi + lo 16-bit parts (products hi*hi + hi*lo + lo*hi,
 * FP32 accumulation) and FP32 twiddles between them (FP16X2 scales each
 * transform's input by a power of two to stay in FP16's range).  Statistics,
 * SNR and the subpixel fit are the FP32 form's FP64-accumulated kernels in
 * every precision.  BF16X2 / FP16X2 support window sizes 128 and 256 and the
 * plain (unwarped) forward only. */
typedef enum { SWIFT_PREC_FP32 = 0, SWIFT_PREC_BF16X2 = 1, SWIFT_PREC_FP16X2 = 2 } swift_precision;

/* Per-window status codes (swift_result.status). */
enum {
  SWIFT_WIN_OK = 0,
  SWIFT_WIN_OUT_OF_BOUNDS = 1, /* a window leaves its image                     */
  SWIFT_WIN_FLAT = 2,          /* all pixels of either window are equal         */
  SWIFT_WIN_NONFINITE = 3,     /* a NaN or infinity in either (float) window    */
  SWIFT_WIN_TIMEOUT = 4        /* a staged window load did not complete within
                                  its bounded wait; outputs are not valid      */
};

/* One matching configuration (one pyramid level), Sec. III:
 *   n                    window side; 64, 128, 256 or 512 (512: streaming
 *                        schedule, FP32, unwarped forward only)
 *   whiten_exponent      w in [0, 1]: magnitudes of the cross-power spectrum
 *                        C = M conj(R) are raised to 1 - w (G = C |C|^-w);
 *                        0 = plain correlation, 1 = phase-only correlation
 *   apod, tukey_alpha    taper (alpha in (0, 1], used by TUKEY only)
 *   snr_exclusion_radius pixels within this wrapped Euclidean distance of the
 *                        peak are left out of the SNR background; in
 *                        [0, n/4)                                            */
typedef struct {
  int32_t n;
  float whiten_exponent;
  int32_t apod;
  float tukey_alpha;
  float snr_exclusion_radius;
} swift_level;

/* An image (section) or a stack of patches, row-major, on the device.
 *   data    device pointer to uint8 or float32 elements (the plan's dtype)
 *   pitch   elements between consecutive rows
 *   stride  elements between consecutive images of a stack: the K sections
 *           averaged into a reference model (Sec. III, "remod"), or the
 *           patches of patch mode
 *   height, width  image size in pixels (ignored in patch mode)
 *   count   number of sections averaged into each window (>= 1); the window
 *           is then their mean.  Use 1 for the moving image.                 */
typedef struct {
  const void* data;
  int64_t pitch;
  int64_t stride;
  int32_t height;
  int32_t width;
  int32_t count;
} swift_image;

/* A batch of window pairs.
 *   ref, mov     HOST arrays of n_levels images: level l's windows are cut
 *                from ref[l] (reference, possibly a K-section model) and
 *                mov[l] (moving)
 *   ref_origin   device int32 [B][2] (y, x) window origins in ref; NULL in
 *                patch mode
 *   mov_origin   device int32 [B][2] origins in mov; NULL in patch mode
 *   level        device int32 [B] level of each window; NULL = all level 0
 *   n_windows    B >= 0 (0 is a no-op)
 *   patch_mode   0: windows are cut from images at the origins;
 *                1: window b of level l is the n x n patch starting at
 *                   data + b * stride (pitch = n) of ref[l] / mov[l]
 *   affine       device float [B][6] or NULL.  When set (section mode only),
 *                moving-window pixel (i, j) is the bilinear sample of mov[l]
 *                at origin + c + [[a_yy, a_yx], [a_xy, a_xx]] (i - c, j - c)
 *                + (t_y, t_x), c = n/2, for theta = (a_yy, a_yx, t_y, a_xy,
 *                a_xx, t_x) -- a locally affine warp of the window (Sec. III,
 *                mir's affine triangles).  A window whose warped corners
 *                leave [0, h-1] x [0, w-1] is OUT_OF_BOUNDS.  The first call
 *                with warps (or the first backward) allocates the plan's
 *                extra workspace; make it before capturing the stream.
 *   level_offsets HOST int64 [n_levels + 1] or NULL.  When set, the windows
 *                are sorted by level: level l's windows are b in
 *                [level_offsets[l], level_offsets[l + 1]), with
 *                level_offsets[0] = 0 and level_offsets[n_levels] = B
 *                (non-decreasing).  Each level's launches then cover only
 *                its own windows instead of scanning the whole batch for
 *                them; `level` may be NULL (forward calls only: warped
 *                windows and the backward need `level`).  A capture bakes
 *                the offsets into the graph.                                 */
typedef struct {
  const swift_image* ref;
  const swift_image* mov;
  const int32_t* ref_origin;
  const int32_t* mov_origin;
  const int32_t* level;
  int64_t n_windows;
  int32_t patch_mode;
  const float* affine;
  const int64_t* level_offsets;
} swift_batch;

/* Result of one window pair (32 bytes).
 *   dy, dx   integer peak of the match response as a signed shift in
 *            [-n/2, n/2): the moving window's content sits at
 *            reference + (dy, dx).  Ties go to the smallest row-major index.
 *   sy, sx   subpixel shift: integer peak plus a separable three-point
 *            parabola offset in [-1/2, 1/2] per axis (0 if not concave)
 *   snr      (peak - mean_bg) / std_bg over background pixels farther than
 *            the exclusion radius from the peak (population std);
 *            +inf if std_bg = 0 and the peak is above the mean
 *   peak     match response at the peak; the response is
 *            Re(IDFT(G)) / n^2, so an exact shift under phase-only matching
 *            gives 1 - 1/n^2
 *   status   SWIFT_WIN_* ; outputs are 0 unless status is SWIFT_WIN_OK      */
typedef struct {
  int32_t dy, dx;
  float sy, sx;
  float snr;
  float peak;
  int32_t status;
  int32_t reserved;
} swift_result;

typedef struct swift_plan_s* swift_plan;

/* Create a plan for up to n_levels (1..16) matching levels.  Builds the taper
 * and twiddle tables (FP64 on the host, stored as FP32 on the current device).
 * max_windows bounds n_windows of later calls (> 0).  Returns
 * SWIFT_ERR_UNSUPPORTED for a window size or precision this build lacks
 * (BF16X2 / FP16X2 with a level whose n is not 128 or 256).  A reduced-
 * precision plan returns SWIFT_ERR_UNSUPPORTED from the affine-warped
 * forward and from swift_match_backward.
 * On success *out receives the plan; on failure *out is set to NULL. */
swift_status swift_plan_create(const swift_level* levels, int32_t n_levels, swift_dtype in,
                               swift_precision prec, int64_t max_windows, swift_plan* out);

/* Release a plan's tables (NULL is a no-op).  The caller must make sure no
 * launch that uses the plan is still running. */
swift_status swift_plan_destroy(swift_plan plan);

/* Forward match of a batch (Sec. III, the swim step): one result per window
 * written to out (device, [n_windows]).  Stream-ordered, no host sync. */
swift_status swift_match_batch(swift_plan plan, const swift_batch* batch, swift_result* out,
                               void* stream);

/* Forward match without any device allocation.
 *
 * For callers that cannot call cudaMalloc: code running inside another
 * allocator's callback, real-time loops that must not change their memory
 * after start-up, or processes whose device memory pool belongs to a
 * framework.  No plan is needed and nothing is allocated: the scratch this
 * path needs (window statistics, row spectra, whitened inverse-column data,
 * the match response) lives in one 24 MiB file-scope device array that every
 * GPU which loads the library holds until the process exits.  At every call
 * a small kernel on `stream` computes the taper, twiddle and taper-transform
 * tables of `level` straight into that array (no host buffer is read), so a
 * call can be captured into a CUDA graph and replayed (after the set-up call
 * below).  The paper has no
 * counterpart: this is a
 * deployment variant of swift_match_batch for a single level (batch->level
 * must be NULL); it runs the same streaming kernels and gives the same
 * results.
 *
 * Limits: at most floor((24 MiB - 9216 B) / per-window bytes) windows per
 * call: 7 windows of 512 x 512, 31 of 256 x 256, 127 of 128 x 128, 510 of
 * 64 x 64.  Larger
 * batches return SWIFT_ERR_CAPACITY before any work is queued; split them.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before capturing any stream into a
 * CUDA graph.  The kept address belongs to the device's context: after
 * cudaDeviceReset on that device, do not call this entry point again in the
 * same process.
 *
 * Sharing: all calls on a device use the same array and it keeps the last
 * call's contents (its per-window finalize counters start at zero and every
 * call leaves them at zero; nothing else in it has to hold any value).  Calls that overlap
 * on the GPU (different streams, or different host threads without ordering)
 * race on it and corrupt each other's results; order them on one stream. */
swift_status swift_match_batch_noalloc(const swift_level* level, swift_dtype in, const swift_batch* batch,
                                       swift_result* out, void* stream);

/* Backward of the match: gradients of
 *     L = sum_b grad_peak[b] * peak_b + grad_snr[b] * snr_b
 * with respect to the affine warp of every moving window (batch->affine, or
 * the identity warp when NULL) and to each level's whitening exponent.  The
 * peak index of each window (and with it the SNR background set) is held
 * fixed: the argmax has no derivative.  The forward is recomputed from the
 * inputs (no state is kept between calls).  Windows whose status is not OK
 * get zero gradients.
 *   grad_peak, grad_snr   device float [B]
 *   grad_affine           device float [B][6], same order as the warp
 *   grad_w                device float [n_levels] (summed over the batch)
 * Section mode only.  Stream-ordered; may allocate the plan's extra workspace
 * on its first call. */
swift_status swift_match_backward(swift_plan plan, const swift_batch* batch, const float* grad_peak,
                                  const float* grad_snr, float* grad_affine, float* grad_w, void* stream);

/* Forward schedules of a level (FP32 plans; the BF16X2 / FP16X2 forms have
 * their own five-kernel schedule).
 *   FUSED       one kernel per level: each window's field lives in the shared
 *               memory of one CTA (64 x 64) or of a cluster of 2 (128 x 128)
 *               or 8 (256 x 256) CTAs, with the row/column redistributions
 *               through distributed shared memory
 *   STREAM      kernels of independent CTAs per slice of a level's windows,
 *               passing each window's intermediates through the plan's
 *               workspace.  Up to 256 x 256 three: rows (each row block
 *               records its sums and flatness), column pairs (the records
 *               combined, the means removed in the spectrum, the whitening)
 *               and inverse rows (the last block of each window finalizes
 *               it), plus a finalize kernel for exclusion radii of 8 px and
 *               more; 512 x 512 five (statistics, rows, columns, inverse
 *               rows, finalize)
 *   PERSISTENT  the same five steps as work items of ONE kernel for every
 *               level that has this schedule: CTAs claim items in a fixed
 *               order from a queue and wait (bounded) for the items they
 *               depend on; each window's intermediates live in a ring of
 *               workspace slots small enough to stay in L2.  Windows of up to
 *               256 x 256.  Results equal the STREAM schedule's bit for bit.
 *               A wait that runs out (about 2 s) stops the launch's remaining
 *               work: those windows report SWIFT_WIN_TIMEOUT.  The workspace
 *               grows to the largest batch matched (a call that must grow it
 *               may not be captured into a graph: swift_plan_capture makes an
 *               uncaptured call first)
 *   DEFAULT     FUSED for 64 x 64, STREAM for 128 x 128 and larger
 * A forward call spreads its launch units (each fused launch, each
 * streaming slice, in every precision; the affine-warped forward excepted)
 * over lanes: the call's stream and one auxiliary stream of
 * the plan, each lane with its own part of the workspace, so that one unit's
 * tail overlaps another's head.  The auxiliary lane waits for the work queued
 * on the call's stream before the call, and the call's stream waits for the
 * auxiliary lane at its end: the call stays one stream-ordered unit (also
 * inside a captured graph).  See swift_plan_set_lanes. */
typedef enum {
  SWIFT_SCHED_DEFAULT = 0,
  SWIFT_SCHED_FUSED = 1,
  SWIFT_SCHED_STREAM = 2,
  SWIFT_SCHED_PERSISTENT = 3
} swift_schedule;

/* Choose the forward schedule of one level. */
swift_status swift_plan_set_schedule(swift_plan plan, int32_t level, int32_t schedule);

/* Autotuner: on this batch (CUDA events; synchronises the host) it times
 * the fused and streaming schedules of every level present, then the whole
 * call with those per-level picks against one persistent launch of every
 * level that has it, at each skew of the persistent work order (4, 8, 12,
 * 16 windows between consecutive steps of a window: larger skews leave more
 * items between a producer and its consumer, smaller ones keep a smaller
 * ring in L2), then the chosen schedules with one lane and with two, and
 * keeps the fastest for later calls.  `chosen` (host int32
 * [n_levels], may be NULL) receives the schedule of each level.  On return
 * `out` holds the batch's results under the chosen schedules. */
swift_status swift_plan_autotune(swift_plan plan, const swift_batch* batch, swift_result* out, void* stream,
                                 int32_t* chosen);

/* Skew of the persistent schedule's work order (1..16; default 16): stage k
 * of a level's j-th window sits at time j + k * skew.  Larger skews leave
 * more items between a producer and its consumer (fewer waits), smaller ones
 * keep fewer windows in flight (a smaller ring of workspace slots, 5 * skew +
 * 4, to hold in L2).  The autotuner sets it too. */
swift_status swift_plan_set_skew(swift_plan plan, int32_t skew);

/* Lanes of the plan's forward calls (1 or 2; default 2; the autotuner sets
 * it too; the affine-warped forward always uses one).  With 1 every launch
 * goes to the call's stream and a streaming slice holds up to
 * S = min(max_windows, 2048) windows.  With 2 each level's windows are split
 * into slices of about half the level (at least 256 windows, at most S, or
 * S / 2 when S windows of the plan's largest size pass 2 GiB of workspace),
 * each going to the less loaded lane; the workspace holds one such part per
 * lane.  The results do not depend on the lanes.  SWIFT_ERR_INVALID_ARG for
 * other values. */
swift_status swift_plan_set_lanes(swift_plan plan, int32_t lanes);
/* The plan's current lanes, into *lanes (host int32). */
swift_status swift_plan_get_lanes(swift_plan plan, int32_t* lanes);

/* How the streaming row kernel loads uint8 section windows (Sec. II: the
 * windows cut from the two images): 0 by plain loads only (16-byte vectors
 * where a window's rows start on a 16-byte boundary, else byte loads); 1 (the
 * default) through tensor-map (TMA) tile copies for the windows whose rows
 * start off a 16-byte boundary in either image, plain vectors for the rest;
 * 2 through tensor-map copies for every window.  A tile copy takes the rows
 * of one row block from the 16-byte chunk holding the window's first column
 * (so the copy starts aligned whatever the origin) into shared memory, and
 * the kernel reads the window from the origin's offset in the chunk.  Tile
 * copies need 16-byte aligned image addresses, pitches and widths and a
 * one-section reference; other images load as with 0.  The results do not
 * depend on the mode.  SWIFT_ERR_INVALID_ARG for other values. */
swift_status swift_plan_set_row_tma(swift_plan plan, int32_t mode);
/* The plan's current mode, into *mode (host int32). */
swift_status swift_plan_get_row_tma(swift_plan plan, int32_t* mode);

/* Capture one forward call on `batch` (all its levels) into a CUDA graph
 * owned by the plan; swift_plan_replay then re-runs it with one graph
 * launch.  Pointers and sizes are baked into the graph: replay matches the
 * same buffers (whose contents may change).  `stream` must not be the legacy
 * default stream.  A new capture replaces the previous one. */
swift_status swift_plan_capture(swift_plan plan, const swift_batch* batch, swift_result* out, void* stream);
swift_status swift_plan_replay(swift_plan plan, void* stream);

/* Per-kernel timing.  While enabled, every forward launch records CUDA
 * events on its stream around each kernel (a ring of 1024 launch records);
 * swift_plan_timings synchronises on them and returns, per kernel slot, the
 * summed device time in ms and the number of launches since the last read
 * (after more than 1024 launch records, the most recent 1024 only), then
 * starts over.  Slots: 0 statistics, 1 row transforms, 2 column
 * transforms + whitening, 3 inverse row transforms, 4 finalize (the
 * streaming schedule, and the same five kernels of the BF16X2 / FP16X2
 * forms; a streaming slice whose finalize is folded into its inverse rows --
 * n <= 256, exclusion radius below 8 px -- launches no finalize kernel and
 * counts none), 5 fused kernel, 6 persistent launch (its clearing of the
 * work queue included), 7 unused.  kernel_ms and launches are host arrays of
 * 8.  With two lanes (swift_plan_set_lanes) launches of different slices
 * overlap, so each launch's time includes the GPU it shared. */
swift_status swift_plan_set_timing(swift_plan plan, int32_t enable);

/* Test hook for the bounded-wait failure path (not for production use).
 * While enabled, the FP32 streaming schedule's row staging by asynchronous
 * copies counted on an mbarrier (bulk copies of aligned float32 rows, and the
 * tensor-map tile copies of uint8 rows, swift_plan_set_row_tma) expects 16
 * bytes more than its copies deliver, so its wait gives up after its bound
 * (about 2 s, then about 2 s more for copies in flight) and every such window
 * reports SWIFT_WIN_TIMEOUT.  Nothing faults or hangs; the stream and the
 * plan stay usable, and calls after disabling it give normal results.
 * Windows loaded by plain loads, the fused schedule and the tensor-core forms
 * do not use this staging and are unaffected. */
swift_status swift_plan_set_test_stall(swift_plan plan, int32_t enable);

/* Test hook for the persistent schedule's bounded waits (not for production
 * use).  While `window` >= 0, the row-transform items of that window (its
 * position in the launch's sequence of windows: the batch order for a batch
 * without levels) never report completion, and every wait of the launch
 * gives up after about 10 ms instead of 2 s.  The wait for that window's
 * rows runs out, the launch stops its remaining work, and the windows not
 * finished by then report SWIFT_WIN_TIMEOUT.  Nothing faults or hangs; the
 * plan stays usable.  -1 turns the hook off. */
swift_status swift_plan_set_test_hold(swift_plan plan, int64_t window);

/* Test hook for the window guard (not for production use).  While enabled,
 * the statistics kernel of the FP32 streaming schedule (512 x 512 levels:
 * smaller windows take their statistics in the row kernel, which derives the
 * status word itself) reports windows of other levels as OK without reading
 * them -- the state a raced or stale workspace could leave.  The row kernels re-check every window's level and
 * bounds from the batch's own arrays (swift_window_check) before turning an
 * origin into an address, so such a window is still skipped and its result
 * record is left as it was. */
swift_status swift_plan_set_test_stale_status(swift_plan plan, int32_t enable);
swift_status swift_plan_timings(swift_plan plan, float* kernel_ms, int32_t* launches);

/* ------------------------------------------------------------------------
 * Rendering step ("mir": Sec. III module list, Sec. IV).  The paper renders
 * aligned sections from the linear least-squares solution of the swim
 * correspondence points, as texture mapping of a triangulated mesh whose
 * triangles are each locally affine, each fitted to the points in and around
 * it.
 *
 * A correspondence is q (output / reference frame), p (source section, the
 * matching point) and a weight w >= 0, all (y, x): q and p are float32 [P][2],
 * w float32 [P], device pointers.  An affine maps output to source,
 * p = A q + t, stored as double[6] = (a_yy, a_yx, t_y, a_xy, a_xx, t_x).
 * Fits minimise sum_i w_i |A q_i + t - p_i|^2 in FP64.
 * ------------------------------------------------------------------------ */

/* Triangle mesh: ny x nx square cells of side `cell` (>= 8) from the integer
 * output-frame corner (origin_y, origin_x); each cell is split by its main
 * diagonal into triangle 2 (cy nx + cx) + 0, holding the pixels with
 * (x - x0) >= (y - y0), and + 1, holding the others. */
typedef struct {
  int32_t origin_y, origin_x;
  int32_t cell;
  int32_t ny, nx;
} swift_mesh;

/* Fit status (per group / triangle). */
enum {
  SWIFT_FIT_OK = 0,
  SWIFT_FIT_FALLBACK = 1,  /* triangle support degenerate: the all-points affine was used */
  SWIFT_FIT_DEGENERATE = 2 /* fewer than three non-collinear weighted points: identity   */
};

/* Correspondences from forward-match results (the swim step's output): for
 * window b, q = ref_origin[b] + n/2 (the reference window centre),
 * p = mov_origin[b] + n/2 + (sy, sx) (where that content sits in the moving
 * section) and w = snr when status is SWIFT_WIN_OK and snr is finite and
 * >= min_snr, else w = 0 (and p = the moving centre): the SNR-weighted least
 * squares.  All device pointers: results [B], origins int32 [B][2], q and p
 * float32 [B][2], w float32 [B]. */
swift_status swift_correspondences(const swift_result* results, const int32_t* ref_origin,
                                   const int32_t* mov_origin, int64_t n_windows, int32_t n, float min_snr, float* q,
                                   float* p, float* w, void* stream);

/* One weighted least-squares affine per group: group g owns points
 * [offsets[g], offsets[g+1]) (offsets: device int64 [n_groups + 1]).
 * theta: device double [n_groups][6]; status: device int32 [n_groups].  A
 * group is degenerate (identity written) when its weights sum to 0 or its
 * weighted points are (nearly) collinear: det(Sqq) <= 1e-9 (tr Sqq / 2)^2 for
 * the weighted centred second moments Sqq.  Stream-ordered. */
swift_status swift_fit_affine(const float* q, const float* p, const float* w, const int64_t* offsets,
                              int32_t n_groups, double* theta, int32_t* status, void* stream);

/* The same fit as an update: theta holds each group's previous affine on
 * entry; an OK group overwrites it, a degenerate group keeps it (status
 * SWIFT_FIT_DEGENERATE).  This is how the registration loop keeps a section's
 * affine when its matches do not support a new one, without a host round
 * trip.  Same arguments and errors as swift_fit_affine. */
swift_status swift_fit_affine_update(const float* q, const float* p, const float* w, const int64_t* offsets,
                                     int32_t n_groups, double* theta, int32_t* status, void* stream);

/* One affine per mesh triangle (theta: device double [2 ny nx][6], status:
 * device int32 [2 ny nx]), each fitted to the points within Chebyshev
 * distance `band` (>= 0, output pixels) of the closed triangle: the
 * triangle's own area plus a surrounding band (band = cell takes in the
 * neighbouring triangles).  Degenerate supports take the all-points affine
 * (SWIFT_FIT_FALLBACK), or the identity when that is degenerate too. */
swift_status swift_mesh_fit(const float* q, const float* p, const float* w, int64_t n_points,
                            const swift_mesh* mesh, int32_t band, double* theta, int32_t* status, void* stream);

/* Render records of a mesh: one 32-byte record per triangle, computed from
 * theta (as written by swift_mesh_fit) in FP64 once per mesh.  records: device
 * buffer of 32 x 2 ny nx bytes, 16-byte aligned, owned by the caller; its
 * layout is private to the library. */
swift_status swift_render_prepare(const double* theta, const swift_mesh* mesh, void* records, void* stream);

/* Texture-map one source section (src: a uint8 / float32 image, height and
 * width >= 2, pitch in elements) through the mesh into out (device,
 * [out_h][out_pitch] elements of out_dtype): output pixel (y, x) belongs to
 * the triangle of its cell (cells clamped to the mesh) and takes the bilinear
 * sample of the source at A (y, x) + t, or `fill` where that point leaves
 * [0, h-1] x [0, w-1].  out_dtype SWIFT_IN_F32 stores the sample;
 * SWIFT_IN_U8 stores it rounded half to even and clamped to [0, 255].
 * records from swift_render_prepare with the same mesh.  Sample points are an
 * integer base plus an FP32 fraction, so their error stays ~1e-4 px at any
 * section coordinate.  Limits: out_h, out_w, |origin| and the mesh extent
 * (cell x cells) at most 2^20 pixels (else SWIFT_ERR_INVALID_ARG). */
swift_status swift_render(const swift_image* src, swift_dtype dtype, const void* records, const swift_mesh* mesh,
                          void* out, swift_dtype out_dtype, int32_t out_h, int32_t out_w, int64_t out_pitch,
                          float fill, void* stream);

/* ------------------------------------------------------------------------
 * Pyramid and model steps around the match ("iscale" and "remod", Sec. III
 * module list and model averaging).
 * ------------------------------------------------------------------------ */

/* Box-mean downsampling by an integer factor (1..64): out (y, x) is the mean
 * of the factor x factor block at (factor y, factor x); partial edge blocks
 * are dropped, so out is floor(H / f) x floor(W / f) (rows <= 65535, else
 * SWIFT_ERR_UNSUPPORTED).  uint8: exact integer mean rounded half to even;
 * float32: float32 block sum in row-major order divided by f^2.  out has the
 * source's type, device memory, out_pitch elements per row.  A source with
 * count > 1 is a batch of images `stride` elements apart, downsampled in one
 * launch into consecutive output planes of out_pitch x floor(H / f)
 * elements. */
swift_status swift_downsample(const swift_image* src, swift_dtype dtype, int32_t factor, void* out, int64_t out_pitch,
                              void* stream);

/* Z-averaged models of a uint8 section stack (device: section j at
 * stack + j * stride, rows `pitch` bytes apart): model z (device, at
 * out + z * out_stride elements, rows out_pitch elements apart) is the mean
 * of the sections j in [z - k, z + k], j != z, with valid[j] != 0 (valid:
 * device uint8 [n_sections], NULL = all valid); with no such section it is
 * section z itself.  out_dtype SWIFT_IN_F32: float32(integer sum) /
 * float32(count), one IEEE division; SWIFT_IN_U8: the exact mean rounded half
 * to even.  height <= 65535. */
swift_status swift_zmodel(const uint8_t* stack, int64_t stride, int32_t n_sections, int32_t height, int32_t width,
                          int64_t pitch, int32_t k, const uint8_t* valid, void* out, swift_dtype out_dtype,
                          int64_t out_stride, int64_t out_pitch, void* stream);

/* Set the whitening exponent of one level for later calls (w in [0, 1]). */
swift_status swift_plan_set_whitening(swift_plan plan, int32_t level, float w);

/* Human-readable name of a status code (static string). */
/* The window guard that every kernel applies before it turns an origin into
 * an address: a window of side n whose level index is `level` belongs to a
 * launch of level `want_level`, and its reference window at ref_origin (y, x)
 * and moving window at mov_origin (y, x) lie inside images of ref_h x ref_w
 * and mov_h x mov_w pixels.  Host function (no GPU needed).
 * Returns SWIFT_WIN_OK (0), SWIFT_WIN_OUT_OF_BOUNDS (1), or -1 for a window
 * of another level (skipped: no result is written for it by that launch). */
int32_t swift_window_check(int32_t n, int32_t level, int32_t want_level, const int32_t* ref_origin,
                           const int32_t* mov_origin, int32_t ref_h, int32_t ref_w, int32_t mov_h, int32_t mov_w);

const char* swift_status_string(swift_status s);

/* Library version string, e.g. "swift-gb300 0.1 sm_103a". */
const char* swift_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWIFT_H_ */
