/*
 * hrc.h -- C ABI of the GB300 Holographic Radiance Cascades (HRC) library.
 *
 * The library computes the 2D fluence F(p) of Eq. 1 (Sec. 3) by the HRC
 * method of Sec. 4: directly traced intervals T_0..T_2 (Sec. 4.2, Eq. 9),
 * the acceleration structure T_3..T_N built by interval extension (Sec. 4.1,
 * Eqs. 18-20), the merge down the cascades R_{N-1}..R_0 (Eqs. 13-17) and the
 * sum over four quadrants (Algorithm 1, procedure Lighting), plus the exact
 * adjoint of all of it.  Options of a context add the Eq. 21 cross blur
 * (hrc_set_cross_blur), multiple bounces (hrc_fluence_bounces), offscreen
 * light as R_N from an environment map (hrc_set_environment) or from a
 * caller-supplied table (hrc_set_top_radiance), and per-channel extinction
 * (hrc_set_channel_extinction); all are off by default.
 *
 * Data conventions (shared by every entry point):
 *   - Images are row-major: emission e[C][H][W] (the per-unit-length source
 *     term integrated in Eq. 4), extinction sigma_t[H][W] (Eq. 2, per pixel
 *     length, one channel shared by all C colours unless per-channel
 *     extinction is enabled: then [C][H][W]), fluence F[C][H][W].
 *     Pixel (x, y) is the unit square [x, x+1] x [y, y+1]; its probe sits at
 *     the centre.  Cells outside the grid are vacuum with no emission.
 *   - Unless stated otherwise, tensor pointers are DEVICE pointers to
 *     contiguous fp32 data, 16-byte aligned.  The library never frees or
 *     keeps ownership of caller memory.
 *   - A context owns every scratch buffer (all T and R levels, gradients).
 *     It allocates them in hrc_create / hrc_create_batched and in the set-up
 *     calls that enable an option (hrc_set_precision for FP64,
 *     hrc_set_cross_blur, hrc_reserve_bounces, hrc_set_environment,
 *     hrc_set_top_radiance, hrc_set_channel_extinction).  Compute calls
 *     allocate no buffer; the first call with a new set of pointers (or a
 *     new configuration) captures and instantiates a CUDA graph of the
 *     pass, which the driver allocates, and later calls with the same
 *     pointers replay it.  A
 *     context keeps eight such graphs (the oldest is replaced).  When at
 *     least six of them were never replayed (the caller's tensors move
 *     every call), a pass with a new pointer set is launched directly
 *     instead of captured, unless that set was seen in the last sixteen
 *     such passes; so a caller whose tensors move every step pays about the
 *     direct-launch cost (hrc_set_graphs(ctx, 0)), and one whose tensors
 *     recur gets graphs.
 *   - Compute calls are asynchronous on the context's stream: HRC_OK means
 *     "enqueued".  Argument errors are reported synchronously; an
 *     asynchronous CUDA error surfaces as HRC_ECUDA on a later call.
 *   - NaN / Inf inputs are accepted and propagate; negative sigma_t is not
 *     rejected (the formulas are analytic in sigma_t).
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - hrc_last_error returns a static description of the last failure.
 */
#ifndef HRC_H
#define HRC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hrc_ctx hrc_ctx;

typedef enum {
    HRC_OK = 0,
    HRC_EINVAL = 1,    /* bad argument (size, null pointer, misalignment)      */
    HRC_ENOMEM = 2,    /* device allocation failed                              */
    HRC_ECUDA = 3,     /* CUDA launch or runtime error                          */
    HRC_ESTATE = 4,    /* call out of order (e.g. backward before forward)      */
    HRC_ETIMEOUT = 5,  /* a bounded device-side wait gave up (its launch ended
                          early; reported by hrc_sync / hrc_batched_sync /
                          hrc_noalloc_sync)                                      */
    HRC_EBOUNDS = 6    /* a device-side bounds check fired (debug builds)       */
} hrc_status;

typedef enum {
    HRC_FP32 = 0,       /* intervals and fluence stored and computed in fp32          */
    HRC_FP16_LOGT = 1,  /* radiance/fluence stored fp16, transmittance as fp32
                           tau = -ln T; arithmetic in fp32 (Sec. 5 stores fp16)   */
    HRC_BF16_LOGT = 2,  /* as above with bf16 radiance/fluence storage              */
    HRC_FP64_TEST = 3   /* fp64 everywhere; only for finite-difference checks via
                           hrc_fluence_f64 / hrc_fluence_backward_f64              */
} hrc_precision;

/* Create a context for one W x H scene with `channels` colours
 * (1 <= channels <= 4, W, H >= 1).  `cascades` <= 0 selects
 * N = ceil(log2 U) per quadrant frame (U = W for +-x, U = H for +-y; Sec. 4.2);
 * a positive value caps N (R_cascades is then taken as 0, as R_N is).
 * Allocates every buffer of the forward and backward passes on the current
 * device.  Returns HRC_EINVAL / HRC_ENOMEM / HRC_ECUDA on failure (*out = 0). */
hrc_status hrc_create(int W, int H, int channels, int cascades, hrc_ctx **out);

/* CUDA graphs of whole passes (default 1): with 1, each pass is captured
 * once per set of pointers and configuration and replayed afterwards (eight
 * graphs per context); with 0, every call launches its kernels directly
 * (no capture, no graph memory; about 0.1 ms more launch time per 1024^2
 * frame).  hrc_graph_captures returns how many graphs the context (and its
 * per-channel contexts) has captured so far, -1 for NULL. */
hrc_status hrc_set_graphs(hrc_ctx *ctx, int enable);
long long hrc_graph_captures(const hrc_ctx *ctx);

/* Release the context and its device buffers (synchronises its stream). */
hrc_status hrc_destroy(hrc_ctx *ctx);

/* Stream for all later calls (a cudaStream_t; NULL = legacy default stream). */
hrc_status hrc_set_stream(hrc_ctx *ctx, void *cuda_stream);

/* Storage precision of the interval and fluence buffers (see hrc_precision).
 * Switching to HRC_FP64_TEST allocates its fp64 buffers once. */
hrc_status hrc_set_precision(hrc_ctx *ctx, hrc_precision prec);

/* Launch schedule (a tuning knob; results are identical for every value):
 * 0 = every kernel launch covers the four quadrant frames (level-major);
 * 1 = the frames run one after another, so that each level's producer and
 *     consumer meet in L2;
 * 2 = the four frames' chains (trace, merge up, merge down) run as four
 *     parallel branches of the pass (context-owned streams, forked from and
 *     joined to the caller's stream; parallel paths of the captured graph),
 *     so that one frame's launch fills the SMs while another's drains; the
 *     fluence sum follows the join.  With per-launch timing on, and in the
 *     level recomputation of the backward, 2 runs as 0.
 * Default 0. */
hrc_status hrc_set_schedule(hrc_ctx *ctx, int schedule);

/* Launch configuration of a single-scene context (tuning knobs; results are
 * identical for every setting):
 *   schedule: as hrc_set_schedule (0, 1 or 2);
 *   groups:   v per thread in the merge-up kernel: 1 = a pair, 2 = two pairs
 *             blockDim apart, 4 = four consecutive v;
 *   threads:  threads per block of the merge and adjoint-merge kernels
 *             (64, 128, 256 or 512);
 *   vmajor:   grid order of those kernels: 0 = rows in gridDim.x, v-blocks
 *             in gridDim.y; 1 = the reverse (allowed while 4 (W + H) <= 65535,
 *             the gridDim.y limit for the adjoint's level-0 rows);
 *   mdown:    merge-down kernel (fp32 / fp16 / bf16): 0 = every thread loads
 *             its operands; 1 = each block's rows are staged in shared
 *             memory by bulk (TMA) copies completed on an mbarrier; 2 = one
 *             persistent launch for every level (as many 128-thread blocks
 *             as fit on every SM take row segments from a ticket counter;
 *             level-to-level dependencies are tracked by per-column
 *             completion counters with bounded waits; not with schedule 2).
 *             FP64 always uses 0.
 * Defaults {0, 1, 128, 0, 0}; hrc_autotune picks one. */
typedef struct hrc_launch_config {
    int schedule, groups, threads, vmajor, mdown;
} hrc_launch_config;

/* Read / set the launch configuration.  Setting it forgets the borrowed
 * forward inputs (run hrc_fluence again before hrc_fluence_backward).
 * HRC_EINVAL for a value outside the ranges above. */
hrc_status hrc_get_launch_config(const hrc_ctx *ctx, hrc_launch_config *cfg);
hrc_status hrc_set_launch_config(hrc_ctx *ctx, const hrc_launch_config *cfg);

/* Autotuner: times every launch configuration (schedule x groups x threads x
 * grid order, as hrc_launch_config) with forward passes over the context's
 * own staging buffers (the timing does not depend on the data), keeps the
 * fastest, and writes its ms per frame to *best_ms (may be NULL).
 * Synchronous.  Results do not depend on the configuration.  Single-scene
 * contexts in fp32 / fp16 / bf16; the borrowed forward inputs are forgotten
 * (run hrc_fluence again before hrc_fluence_backward). */
hrc_status hrc_autotune(hrc_ctx *ctx, float *best_ms);

/* Forward pass, Algorithm 1 (Lighting) without the Eq. 21 blur:
 * out[c][y][x] = sum over the four quadrant frames of R_0([u+1, v], 1/2).
 * emission [C][H][W], sigma_t [H][W], out [C][H][W]: device fp32.
 * The context remembers (borrows) emission and sigma_t for the backward
 * pass; the caller keeps them alive and unchanged until then. */
hrc_status hrc_fluence(hrc_ctx *ctx, const float *emission, const float *sigma_t, float *out);

/* Same computation from HOST buffers: copies emission and sigma_t to
 * context-owned device buffers, runs hrc_fluence, copies the fluence back to
 * `out` (host) and waits for the stream.  Host buffers may be pageable or
 * pinned (pinned is faster).  A later hrc_fluence_backward borrows the
 * context's own device copies. */
hrc_status hrc_fluence_host(hrc_ctx *ctx, const float *emission, const float *sigma_t, float *out);

/* Adjoint of the last hrc_fluence on this context: given dLoss/dF (grad_F,
 * [C][H][W]), writes dLoss/d emission ([C][H][W]) and dLoss/d sigma_t
 * ([H][W]).  Outputs are overwritten, not accumulated.  By default it reads
 * the intervals T_n / R_n that the last forward left in the context's
 * buffers; with hrc_set_backward_recompute(ctx, 1) it first recomputes them
 * from the borrowed inputs.  Either way it re-traces the borrowed inputs,
 * which must be unchanged since that forward; it may be called several
 * times (another grad_F) without a new forward.  Enqueue it on the forward's
 * stream, or order the two streams.  HRC_ESTATE if no forward ran on this
 * context. */
hrc_status hrc_fluence_backward(hrc_ctx *ctx, const float *grad_F, float *grad_emission,
                                float *grad_sigma_t);

/* Backward strategy of a context (single-scene or batched): 0 (default) =
 * read the levels the forward left in the buffers; 1 = recompute every
 * level T_0..T_N, R_1..R_{N-1} from the borrowed inputs at the start of
 * each backward, so that the backward depends on no forward-time storage:
 * it differentiates at the inputs' contents at the time of the backward.
 * For unchanged inputs the gradients are the same either way; recomputing
 * costs about one forward pass. */
hrc_status hrc_set_backward_recompute(hrc_ctx *ctx, int on);

/* Cross blur (Sec. 4.2, Eq. 21), applied after the fluence sum by every
 * later hrc_fluence / hrc_fluence_host / hrc_fluence_f64 on a single-scene
 * context, and differentiated by the matching backward.  Each pixel becomes
 * the mean of itself (weight 4) and its four edge neighbours (weight 1
 * each), leaving out neighbours outside the grid and those whose opacity
 * 1 - exp(-sigma_t) differs from the pixel's by more than `threshold`; the
 * kept weights are renormalised, so the interior with every neighbour kept
 * is exactly 1/8 [0 1 0; 1 4 1; 0 1 0].  The paper does not state the
 * opacity measure or threshold; 0.5 is this library's default reading.
 * The kept set is piecewise constant in sigma_t, so the blur adds nothing
 * to dLoss/d sigma_t; its adjoint is the transpose for fixed sigma_t.
 *   enable:    0 = off (the default), 1 = on;
 *   threshold: opacity difference in [0, 1] (1 keeps every neighbour).
 * The first enable allocates one context-owned buffer of W * H * C doubles
 * (the unblurred fluence, and dLoss/d(unblurred fluence) in the backward).
 * HRC_EINVAL for other values or on a batched context; HRC_ENOMEM if the
 * buffer does not fit.  hrc_fluence_noalloc never blurs. */
hrc_status hrc_set_cross_blur(hrc_ctx *ctx, int enable, float threshold);
hrc_status hrc_get_cross_blur(const hrc_ctx *ctx, int *enable, float *threshold);

/* Per-channel extinction (the paper keeps T as C-vectors, Sec. 5).  With
 * per_channel = 1, every later call on this single-scene context takes
 * sigma_t as [C][H][W] (channel c has its own extinction) and returns
 * dLoss/d sigma_t as [C][H][W]; with 0 (the default) sigma_t is one [H][W]
 * plane shared by the channels.  Once the transmittance is per channel,
 * every step of the method (Merge, the Eq. 20 blend, the merge down, the
 * fluence sum, the cross blur, the bounce source) acts channel by channel,
 * so the context runs C single-channel contexts (created by the first
 * enable, each with its own level buffers: C radiances and C
 * transmittances per entry in all) on its stream; its settings (stream,
 * precision, launch configuration, backward strategy, cross blur, bounce
 * reservation, timing, environment map row c for channel c) are mirrored
 * into them.  Channel planes whose address is not 16-byte aligned (W * H
 * not a multiple of 4) pass through context-owned staging buffers.
 * hrc_copy_level answers HRC_ESTATE in this mode.  HRC_EINVAL on a batched
 * context or for other values; HRC_ENOMEM if the channel contexts do not
 * fit. */
hrc_status hrc_set_channel_extinction(hrc_ctx *ctx, int per_channel);

/* Environment map (footnote 1 of Sec. 4.2): light arriving from outside
 * the grid, with nothing outside that absorbs or emits.  env is a device
 * array [C][M] (fp32, 16-byte aligned): the radiance seen along the image
 * look angle theta_m = 2 pi (m + 1/2) / M, theta measured from +x (along a
 * row) towards +y (down the rows), linearly interpolated between samples
 * and periodic.  Every later forward and backward on this single-scene
 * context takes R_N(p, i) = A_N(i) env(direction of v_N(i)) and, for an R
 * lookup outside the grid, the sum of its level-N descendants (what the
 * recursion gives when continued outside through vacuum).  The map is
 * converted into a per-frame, per-level table when this call runs (the
 * stream is synchronised; env may be freed afterwards) and is held fixed
 * by the backward (no gradient with respect to it).  env = NULL removes
 * the map (R_N = 0 again).  The first map allocates the table
 * (12 * 4 * 2^(N+1) * C bytes).  HRC_EINVAL on a batched context or for M
 * outside [1, 2^20]; a forward must run again before a backward. */
hrc_status hrc_set_environment(hrc_ctx *ctx, const float *env, int M);

/* Top-level radiance supplied by the caller (footnote 1 of Sec. 4.2: the
 * light from outside the grid enters only through R_N, which another method
 * -- cone tracing an offscreen scene, a sky model -- may compute).  top is a
 * device array [4][K][C] (fp32): top[(q K + j) C + c] is R_N of cone j of
 * quadrant frame q at its top level N_q (j < 2^N_q; K >= 2^N for the largest
 * N of the context), i.e. the radiance integrated over the cone between the
 * frame directions v_N(j) and v_N(j + 1), v_N(k) = (2^N, 2k - 2^N) in frame
 * coordinates (u along +x, -x, +y, -y image axes and v along +y, +y, +x, +x
 * for q = 0 .. 3).  The values do not depend on the probe; an R lookup
 * outside the grid at a lower level sees the sum of its level-N
 * descendants, as with an environment map, which this call replaces (and
 * hrc_set_environment replaces it; either with NULL removes both).  The
 * values are held fixed in the adjoint.  Synchronous; allocates the table
 * once.  With per-channel extinction, channel c takes its own values.
 * HRC_EINVAL for a batched context or K out of range. */
hrc_status hrc_set_top_radiance(hrc_ctx *ctx, const float *top, int K);

/* Multiple diffuse bounces (Sec. 4.2: the output fluence fed into another
 * iteration of the method; Fig. 14).  Bounce 0 is hrc_fluence on
 * `emission`; bounce k + 1 runs it on
 *     e_{k+1} = emission + albedo * sigma_t * F_k / (2 pi),
 * the source of isotropic single scattering in 2D with a per-pixel,
 * per-channel albedo (the scattering fraction of sigma_t; values in [0, 1)
 * converge as bounces grow).  The paper gives no formula for the feedback;
 * this is this library's reading.  Each bounce includes the cross blur
 * when it is enabled.  `out` receives F_bounces ([C][H][W]).
 *
 * hrc_reserve_bounces allocates the context-owned buffers for up to
 * `max_bounces` (0 .. 64; 2 max_bounces + 2 planes of W * H * C doubles):
 * the e_k and F_k of the last bounce forward, which its backward reads, and
 * the backward's scratch.  It must be called before the first bounce call;
 * a larger count reallocates (synchronising the stream).  HRC_EINVAL on a
 * batched context or a count out of range; HRC_ENOMEM if they do not fit.
 *
 * hrc_fluence_bounces: device pointers, 16-byte aligned; albedo is
 * [C][H][W].  The pointers are borrowed until the next forward (as for
 * hrc_fluence).  HRC_EINVAL for bounces outside [0, reserved],
 * HRC_ESTATE without a reservation or in HRC_FP64_TEST (use the _f64
 * variant there).
 *
 * hrc_fluence_bounces_backward: adjoint of the last hrc_fluence_bounces on
 * this context: dLoss/d emission, d sigma_t ([H][W]) and d albedo
 * ([C][H][W]) from dLoss/dF_bounces, overwritten, by the reverse of every
 * bounce (the last one reads the levels its forward left, unless
 * hrc_set_backward_recompute is on or a backward since has reused the
 * buffers; every earlier bounce recomputes its levels from the stored
 * e_k).  HRC_ESTATE if the last forward on the context was not a bounce
 * forward.  A plain hrc_fluence_backward after a bounce forward is
 * HRC_ESTATE too.
 *
 * hrc_bounce_source writes out = emission + albedo * sigma_t * fluence /
 * (2 pi) on the context's stream (one bounce per frame, "temporally":
 * feed the previous frame's fluence into this frame's emission). */
hrc_status hrc_reserve_bounces(hrc_ctx *ctx, int max_bounces);
hrc_status hrc_fluence_bounces(hrc_ctx *ctx, const float *emission, const float *sigma_t, const float *albedo,
                               int bounces, float *out);
hrc_status hrc_fluence_bounces_backward(hrc_ctx *ctx, const float *grad_F, float *grad_emission,
                                        float *grad_sigma_t, float *grad_albedo);
hrc_status hrc_fluence_bounces_f64(hrc_ctx *ctx, const double *emission, const double *sigma_t,
                                   const double *albedo, int bounces, double *out);
hrc_status hrc_fluence_bounces_backward_f64(hrc_ctx *ctx, const double *grad_F, double *grad_emission,
                                            double *grad_sigma_t, double *grad_albedo);
hrc_status hrc_bounce_source(hrc_ctx *ctx, const float *emission, const float *sigma_t, const float *albedo,
                             const float *fluence, float *out);

/* Waits for the context's stream and reports whether a bounded device-side
 * wait of its kernels (the trace kernels' tensor-copy waits, the bulk-copy
 * merge down, the persistent merge down's dependency waits; its per-channel
 * contexts' too) gave up since the last call: HRC_ETIMEOUT, that launch
 * ended early and its outputs are incomplete.  The status word belongs to
 * this context alone and is cleared by this call.  A block that gave up
 * first waits once more, with a much longer bound, for the copies it had
 * issued; if even that runs out the message (hrc_last_error) says so, and
 * the results of later launches on this device are then suspect (a late
 * copy could still land in the shared memory of another block). */
hrc_status hrc_sync(hrc_ctx *ctx);

/* Test hook for the bounded device-side waits: with extra_bytes > 0
 * (0..4096) the trace and the mdown = 1 merge down arm their copy barriers
 * with that many bytes more than they copy, and the mdown = 2 persistent
 * merge down publishes no finished item, so their waits run out after
 * `limit_ns` (<= 0 restores the default, 2 s) and hrc_sync reports
 * HRC_ETIMEOUT instead of a kernel hanging.  {0, 0} restores normal
 * operation; the context stays usable. */
hrc_status hrc_debug_bulk_wait(hrc_ctx *ctx, int extra_bytes, long long limit_ns);

/* FP64 instance of hrc_fluence / hrc_fluence_backward (device fp64 buffers,
 * same layouts); requires hrc_set_precision(ctx, HRC_FP64_TEST). */
hrc_status hrc_fluence_f64(hrc_ctx *ctx, const double *emission, const double *sigma_t, double *out);
hrc_status hrc_fluence_backward_f64(hrc_ctx *ctx, const double *grad_F, double *grad_emission,
                                    double *grad_sigma_t);

/* Batched context: n scenes of sizes W[i] x H[i], one channel count.  The
 * scenes' tensors are packed back to back; hrc_scene_offsets gives the
 * element offsets (n + 1 entries each: emission/out offsets in floats of the
 * [C][H][W] blocks, sigma offsets in floats of the [H][W] blocks). */
hrc_status hrc_create_batched(int n, const int *W, const int *H, int channels, int cascades,
                              hrc_ctx **out);
hrc_status hrc_scene_offsets(const hrc_ctx *ctx, long long *emis_off, long long *sigma_off);

/* As hrc_create_batched, with the interval storage precision chosen at
 * creation (HRC_FP32, HRC_FP16_LOGT or HRC_BF16_LOGT), so the buffers are
 * sized for that precision's layout.  A later hrc_set_precision to a larger
 * layout reallocates them. */
hrc_status hrc_create_batched_prec(int n, const int *W, const int *H, int channels, int cascades,
                                   hrc_precision prec, hrc_ctx **out);

/* Forward / backward of every scene of a batched context in one persistent,
 * CUDA-graph-launched kernel; same semantics as the single-scene calls.
 * HRC_ETIMEOUT if a bounded device-side dependency wait gave up. */
hrc_status hrc_fluence_batched(hrc_ctx *ctx, const float *emission, const float *sigma_t, float *out);
hrc_status hrc_fluence_backward_batched(hrc_ctx *ctx, const float *grad_F, float *grad_emission,
                                        float *grad_sigma_t);

/* Allocation-free forward pass.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- a frame callback
 * running under an engine-owned memory budget, code whose host framework
 * must own every device allocation, or a plugin in a process that forbids
 * new device allocations after start-up (cudaMalloc also synchronises the
 * device, which a real-time frame loop cannot afford).
 *
 * Computes exactly what hrc_fluence computes (fp32, cascades chosen
 * automatically) for one W x H grid with `channels` colours, on
 * `cuda_stream` (NULL = legacy default stream), without a context.  The
 * caller passes the device buffers emission [C][H][W], sigma_t [H][W] and
 * out [C][H][W] (fp32, 16-byte aligned).  Every intermediate level lives in
 * one fixed file-scope device array of HRC_NOALLOC_SCRATCH_BYTES bytes,
 * which every GPU that loads the library holds until the process exits.
 *
 * Limits: 1 <= W, H <= HRC_NOALLOC_MAX_SIDE and 1 <= channels <= 4; larger
 * requests return HRC_EINVAL with a message from hrc_last_error(NULL).
 * No cudaMalloc, cudaFree or other allocating routine is called.
 * Set-up: the first call on each device (made with that device current)
 * resolves the array's device address and writes a constant arc table into
 * it with a synchronous copy; make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents (every level is fully rewritten before it is read, so nothing
 * needs clearing); calls that overlap on the GPU -- on different streams
 * or different host threads -- race on it and must be serialised by the
 * caller. */
#define HRC_NOALLOC_MAX_SIDE 128
#define HRC_NOALLOC_SCRATCH_BYTES 20443392ULL
hrc_status hrc_fluence_noalloc(int W, int H, int channels, const float *emission, const float *sigma_t,
                               float *out, void *cuda_stream);

/* Completion status of hrc_fluence_noalloc on the current device: waits for
 * `cuda_stream`, then reads and clears the no-alloc path's own status word
 * (a word inside the fixed array, shared by every no-alloc call on the
 * device and by no context).  HRC_ETIMEOUT when a bounded copy wait of a
 * call since the last check gave up (that call's fluence is incomplete;
 * its message says whether copies could still have been in flight), else
 * HRC_OK.  Allocates nothing.  The one-time set-up of hrc_fluence_noalloc
 * is redone automatically if the array's device address changes (e.g.
 * after cudaDeviceReset); a caller that resets the device must make the
 * next no-alloc call before any stream capture, as for the first. */
hrc_status hrc_noalloc_sync(void *cuda_stream);

/* Test hook for hrc_noalloc_sync: later hrc_fluence_noalloc calls arm the
 * trace's copy barrier with `extra_bytes` (0..4096) that never arrive and
 * bound its wait by `limit_ns` (<= 0 restores the default, 2 s), so the
 * wait gives up; (0, 0) restores normal operation. */
hrc_status hrc_noalloc_debug_wait(int extra_bytes, long long limit_ns);

/* Waits for the batched context's stream and reports the status of its
 * last persistent launch: HRC_ETIMEOUT if a bounded dependency wait gave
 * up (the launch then ended early and its outputs are incomplete). */
hrc_status hrc_batched_sync(hrc_ctx *ctx);

/* Tuning of the persistent launch: resident blocks per SM (0 = as many as
 * fit) and the ticket order within each stage (0 = input order, 1 = largest
 * scene first).  Results are identical for every setting. */
hrc_status hrc_batched_tune(hrc_ctx *ctx, int blocks_per_sm, int order);

/* Schedule of a batched pass, both captured and replayed as one CUDA graph:
 * 0 (default) = the tile steps of all scenes as multi-scene launches around
 * one persistent launch that runs every scene's merge cascade from a
 * ticket queue with bounded dependency waits; 1 = every scene's own
 * per-level launch sequence (as a single-scene pass), the scenes spread
 * largest first over 8 streams forked from and joined to the caller's
 * stream, so that kernels of different scenes overlap; 2 = level-major
 * multi-scene launches: one launch per stage (each merge-up level, each
 * merge-down level, the fluence sum; each adjoint level) covering every
 * scene that has it, the tile steps as multi-scene tile launches.  Results
 * are identical for all three. */
hrc_status hrc_batched_schedule(hrc_ctx *ctx, int schedule);

/* Test hook for the bounded waits: `withhold_counter` >= 0 makes that stage
 * counter never publish, so the stages after it time out after
 * `spin_limit` polls (about 128 ns each; <= 0 restores the default, about
 * 2 s) and the launch ends with HRC_ETIMEOUT instead of hanging. */
hrc_status hrc_batched_debug(hrc_ctx *ctx, int withhold_counter, long long spin_limit);

/* Introspection for tests: copies level n of quadrant frame q (0..3) from
 * the last forward into `dst` (device fp32).  which = 0: T_n as
 * [U_n][2^n+1][V][C+1] (C radiances then the transmittance T, linear even in
 * the log-T precisions); which = 1: R_n as [U_n][2^n][V][C].  Entries no
 * fluence depends on are NaN, as the library never computes them: column
 * x = 0 of every level (the sum of Algorithm 1 reads R_0 at u + 1, and
 * column 0 feeds only column 0 of the levels next to it), the even columns
 * of T_0 (level 0 reads T_0 only at odd columns, Eq. 14) and the odd
 * directions of T_1 at even columns (Eqs. 15-17 read even directions).  The forward does not store R_0
 * either (the fluence sum computes it in place); this call recomputes it from
 * T_0, T_1 and R_1 of the last forward.  *count receives the element count;
 * dst may be NULL to query it.  HRC_EINVAL if the level does not exist. */
hrc_status hrc_copy_level(hrc_ctx *ctx, int q, int which, int n, float *dst, long long *count);

/* Number of kernel launches the last compute call enqueued. */
int hrc_last_launch_count(const hrc_ctx *ctx);

/* Per-launch timing.  With timing enabled, every kernel a compute call
 * enqueues is bracketed by CUDA events on the context's stream: enable = 1
 * launches the kernels directly (no graph; each record then also holds
 * that launch's host-side launch latency), enable = 2 captures the pass
 * into a CUDA graph whose event-record nodes bracket each kernel, and
 * replays it, enable = 3 does the same with one record per phase (the
 * consecutive launches of one kind, with no event node between them: the
 * phase timed as the graphs of normal operation run it; `level` is then
 * the phase's first level and `launches` its launch count), 0 switches
 * timing off.
 * hrc_get_timing synchronises the stream and fills up to `cap` records of
 * the last compute call; it returns the number of records (or -1 on error).
 * `kind`: 0 trace T_0..T_2, 1 merge up, 2 merge down, 3 fluence sum,
 * 4 adjoint sum, 5 adjoint merge down, 6 adjoint merge up, 7 adjoint trace,
 * 8 batched persistent kernel, 9 other, 10 cross blur, 11 adjoint cross blur,
 * 12 bounce source update, 13 its adjoint.  `bytes` is the launch's
 * algorithmic traffic (each array it consumes read once, each array it
 * produces written once). */
typedef struct { int kind; int level; float ms; double bytes; int launches; } hrc_kernel_time;
hrc_status hrc_set_timing(hrc_ctx *ctx, int enable);
int hrc_get_timing(hrc_ctx *ctx, hrc_kernel_time *out, int cap);

/* Static description of the last error on ctx (or of the last failed
 * creation when ctx is NULL). */
const char *hrc_last_error(const hrc_ctx *ctx);

/* Library version string. */
const char *hrc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HRC_H */
