/*
 * af.h - C ABI of the B300 (sm_103a) lens-aware differentiable-beamforming
 * autofocus library.
 *
 * The library runs one autofocus iteration of Frey et al., "Lens-Aware
 * Differentiable Beamforming for In Vivo Distributed Aberration Correction
 * with Curvilinear Transducers", on one GPU:
 *
 *   af_forward : Sec. III-A exit points at c_med (Eq. 8, Fermat), Eq. 1 ray
 *                sums through the slowness grid, Eq. 2-4 apodization, Eq. 5
 *                subaperture DAS with phase rotation, the CMPE focusing loss
 *                (Sec. II-D) and Eq. 10-12 regularisation.
 *   af_adjoint : dL/ds by a hand-written adjoint of af_forward (Fig. 1g),
 *                exit points and masks held constant.
 *   af_step    : the Eq. 9 update of the sound speed, run as Adam on c in km/s.
 *
 * Conventions shared by every entry point
 *  - Units are SI (m, s, s/m, Hz).  z grows into the tissue.
 *  - Host pointers (const double* in af_config) are read during af_plan only.
 *  - Every d_* pointer is caller-owned DEVICE memory on the current device;
 *    the library never frees it.  The plan owns its own workspaces.
 *  - Calls are asynchronous on the plan's stream (the cudaStream_t passed to
 *    af_plan; NULL = legacy default stream).  Outputs are valid once that
 *    stream has reached the call.  The kernels of af_forward / af_adjoint /
 *    af_step are programmatic dependent launches: each waits on the device
 *    for the work before it on the stream to finish before touching memory,
 *    so stream order holds as for plain launches.
 *  - Errors are returned as af_status codes and never thrown; af_last_error()
 *    returns a message for the last failing call of the calling thread.
 *    Argument and shape errors are detected on the host before any launch.
 *  - A plan is not thread-safe; use one plan per host thread.
 */
#ifndef AF_H
#define AF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct af_plan_s *af_plan_t;

typedef enum {
    AF_OK = 0,
    AF_ERR_ARG = 1,          /* NULL pointer, non-finite or out-of-range scalar */
    AF_ERR_SHAPE = 2,        /* inconsistent sizes (e.g. n_elem % sub_width != 0) */
    AF_ERR_DTYPE = 3,        /* unknown iq_dtype, or a scale array missing for a 16-bit dtype */
    AF_ERR_CUDA = 4,         /* a CUDA runtime call failed (message names it) */
    AF_ERR_NUMERIC = 5,      /* non-positive or non-finite slowness seen on the device */
    AF_ERR_TIMEOUT = 6,      /* a bounded device wait (tensor-core completion) ran out */
    AF_ERR_UNSUPPORTED = 7,  /* valid but outside what this build implements */
    AF_ERR_STATE = 8         /* call order violated (e.g. af_adjoint before af_forward) */
} af_status;

/* storage of the demodulated channel data Psi */
enum { AF_IQ_C64 = 0,        /* interleaved float32 (re, im) */
       AF_IQ_BF16 = 1,       /* interleaved bfloat16 (re, im), times a per-transmit float scale */
       AF_IQ_F16 = 2 };      /* interleaved float16 (re, im), times a per-transmit float scale */

/* lens model */
enum { AF_LENS_BENT_RAY = 0, /* Eq. 7-8: Fermat exit point on a curved lens surface */
       AF_LENS_NONE = 1,     /* Eq. 1 straight rays from the element (with t_ttp: the
                                conventional model of Eq. 6) */
       AF_LENS_PLANAR = 2 }; /* Eq. 7-8 with a flat lens (linear array) */

/* update rule of af_step */
enum { AF_OPT_ADAM = 0,      /* Eq. 9 with Adam moments (beta1, beta2, eps) on c */
       AF_OPT_GD = 1 };      /* Eq. 9 as printed: c <- c - lr dL/dc (m, v unused) */

/* apodization */
enum { AF_APOD_FNUMBER = 0,  /* |x'| <= z' / (2F), z' > 0 (usual f-number reading of Eq. 4) */
       AF_APOD_PRINTED = 1 };/* |x'| <= (F/2) z', z' > 0 (Eq. 4 as printed) */

/*
 * Problem description (host memory, copied by af_plan).
 *
 * Array (Sec. II-A): element a at (elem_x[a], elem_z[a]); its orientation is
 *   Eq. 3 from its neighbours (end elements: linear extrapolation).
 * Lens (Sec. II-B, III-B, Table I): AF_LENS_BENT_RAY: outer surface = arc of
 *   radius lens_radius about (arc_cx, arc_cz), concentric with the elements;
 *   AF_LENS_PLANAR: outer surface = the line z = lens_z, every element above it
 *   (elem_z < lens_z) and every pixel below it (arc_cx, arc_cz, lens_radius
 *   unused); sound speed c_lens; t_ttp is added to every round-trip delay
 *   (Eq. 6-7).
 * Image points r_Omega: n_patch patches of patch_npix pixels, patch-major
 *   (pixel p belongs to patch p / patch_npix), at (pix_x[p], pix_z[p]).
 * Slowness grid (Sec. III-A): node (i, j) at (x0 + i dx, z0 + j dz),
 *   stored row-major s[j * nx + i]; Keys bicubic interpolation; nseg ray
 *   segments (nseg + 1 endpoints) from the exit point to the pixel,
 *   1 <= nseg <= AF_MAX_NSEG (larger values: AF_ERR_UNSUPPORTED).
 *   Every pixel and the lens surface over the aperture must lie inside the
 *   grid box.
 * Channel data Psi[t][r][n] (Eq. 5): n_samp samples per (transmit, receive)
 *   pair, sample n at time t0 + n / fs, demodulation frequency fd.
 * Subapertures: blocks of sub_width consecutive elements; image
 *   B_ij = transmit block i, receive block j.
 * Table II: rho_thresh, fnum, nseg, w1, kx1, kz1, w2, kx2, kz2, lr, as printed.
 *   Eq. 9-11 act on the sound speed in units of c_unit m/s (1000: km/s) with
 *   positions in mm: kx1, kz1 in c_unit/mm, kx2, kz2 in c_unit/mm^2, lr in
 *   c_unit per step.  Table II's values read this way allow gradients of
 *   10 m/s per mm and take Adam steps of 3 m/s (phantom) or 50 m/s (in vivo).
 * Update (Eq. 9) on c = 1 / (c_unit s): optimizer AF_OPT_ADAM (Adam with beta1,
 *   beta2, eps) or AF_OPT_GD (the plain gradient step as printed).
 */
#define AF_MAX_NSEG 65535

typedef struct {
    int n_elem;
    const double *elem_x, *elem_z;
    int lens_mode;
    double arc_cx, arc_cz, lens_radius, c_lens, t_ttp, lens_z;
    int apod_mode;
    double fnum;
    int n_patch, patch_npix;
    const double *pix_x, *pix_z;
    int nx, nz;
    double x0, z0, dx, dz;
    int nseg;
    int n_samp;
    double fs, fd, t0;
    int iq_dtype;
    int sub_width;
    double rho_thresh;
    double w1, kx1, kz1, w2, kx2, kz2;
    double lr, beta1, beta2, eps, c_unit;
    int optimizer;
} af_config;

/* Host-only validation of a configuration (no CUDA call).  Returns AF_OK or
 * the first error found; af_last_error() names it. */
af_status af_check_config(const af_config *cfg);

/* Host-only: device bytes af_plan will allocate for this configuration. */
af_status af_workspace_bytes(const af_config *cfg, size_t *bytes);

/* Validate cfg, copy the geometry to the device of the calling thread and
 * allocate the plan's workspaces.  stream: a cudaStream_t (or NULL). */
af_status af_plan(const af_config *cfg, void *stream, af_plan_t *out);

/* Forward pass (Eq. 1-8, Eq. 10-12 and the CMPE of Sec. II-D): loss of Eq. 12
 * at slowness d_slowness.
 *  d_iq        Psi, [n_elem][n_elem][n_samp] complex, layout per iq_dtype.
 *              Must stay valid and unchanged until the matching af_adjoint.
 *  d_iq_scale  [n_elem] float per-transmit scale for 16-bit dtypes, else NULL.
 *  d_slowness  [nz][nx] float, s/m, all > 0.
 *  d_loss      [4] float written: {L, L_CMPE, R_TV, R_SV}. */
af_status af_forward(af_plan_t plan, const void *d_iq, const float *d_iq_scale,
                     const float *d_slowness, float *d_loss);

/* Adjoint of the last af_forward (Fig. 1g): d_grad [nz][nx] = dL/ds (s/m)^-1.
 * Delays are recomputed from the stored one-way tables, not stored per pair. */
af_status af_adjoint(af_plan_t plan, float *d_grad);

/* Eq. 9 update of c = 1 / (c_unit s) (step counts from 1): AF_OPT_ADAM updates
 * d_slowness, d_adam_m, d_adam_v ([nz][nx] float each) in place; AF_OPT_GD updates
 * d_slowness only (d_adam_m and d_adam_v may then be NULL). */
af_status af_step(af_plan_t plan, const float *d_grad, float *d_slowness,
                  float *d_adam_m, float *d_adam_v, int step);

/* One whole iteration: af_forward + af_adjoint + af_step. */
af_status af_iterate(af_plan_t plan, const void *d_iq, const float *d_iq_scale,
                     float *d_slowness, float *d_grad, float *d_adam_m,
                     float *d_adam_v, int step, float *d_loss);

/* ---- autofocus jobs from host memory (Sec. III-A: N_i iterations per acquisition) ----
 * A job uploads one acquisition's channel data and initial map, runs n_iter
 * af_iterate steps (Adam step index 1..n_iter, moments starting at zero) and reads
 * back the final map and loss.  af_job_submit only enqueues: the upload goes on a
 * copy stream owned by the plan, into one of two device buffers (the one the job
 * before last used, once that job has finished), and the rest on the plan's stream,
 * so a job submitted while another runs has its channel data uploaded under the
 * running job's iterations.  Each job's initial-map copy is ordered before the next
 * job's channel data on the copy engine.
 *  - Host buffers are read and written asynchronously: they must stay valid and
 *    unchanged until af_job_wait.  Pinned memory (cudaHostAlloc / cudaHostRegister)
 *    gives the overlap; pageable memory works but the copies then serialise.
 *  - Device memory: af_job_reserve allocates 2 x the channel data
 *    (n_elem^2 n_samp x 8 bytes for AF_IQ_C64, x 4 for 16-bit), 2 x n_elem floats,
 *    4 grids of nz x nx floats and 4 floats, once per plan; af_destroy frees them.
 *  - Errors: argument errors are reported before anything is enqueued; a CUDA error
 *    or an af_iterate error returns at once (work already enqueued stays queued).
 *
 * af_job_reserve: creates the job buffers, copy stream and events (idempotent;
 *   af_job_submit calls it when needed).
 * af_job_submit:
 *   h_iq        Psi in host memory, layout per the plan's iq_dtype (as af_forward).
 *   h_iq_scale  [n_elem] per-transmit scale for 16-bit dtypes (host), else NULL.
 *   h_s0        [nz][nx] initial slowness (host), s/m.
 *   n_iter      iterations, >= 1.
 *   h_s_out     [nz][nx] final slowness (host), or NULL for no read back.
 *   h_loss_out  [4] loss of the last iteration {L, L_CMPE, R_TV, R_SV} (host), or NULL.
 * af_job_wait: waits for every submitted job and returns af_sync_status. */
af_status af_job_reserve(af_plan_t plan);
af_status af_job_submit(af_plan_t plan, const void *h_iq, const float *h_iq_scale, const float *h_s0,
                        int n_iter, float *h_s_out, float *h_loss_out);
af_status af_job_wait(af_plan_t plan);

/* Release the plan's device memory (job buffers included).  NULL is accepted. */
af_status af_destroy(af_plan_t plan);

/* ---- batches of independent acquisitions (one job, one graph launch) ----
 * A batch owns one plan per configuration, each on a non-blocking stream of its
 * own, so the members run concurrently.  `stream` is the caller's stream: the
 * batch calls fork from it and join back to it (stream order is kept; it may be
 * the legacy default stream).  Errors as af_plan; on failure nothing is kept. */
typedef struct af_batch_s *af_batch_t;
af_status af_batch_plan(int n, const af_config *const *cfgs, void *stream, af_batch_t *out);
/* Member k's plan (owned by the batch) for the per-plan getters and settings. */
af_status af_batch_plan_of(af_batch_t batch, int k, af_plan_t *out);
/* One af_iterate of every member.  Each argument is a host array of n device
 * pointers, member k's buffers as in af_iterate; d_iq_scale may be NULL when no
 * member has 16-bit data.  Asynchronous; no allocation. */
af_status af_batch_iterate(af_batch_t batch, const void *const *d_iq, const float *const *d_iq_scale,
                           float *const *d_s, float *const *d_grad, float *const *d_m,
                           float *const *d_v, int step, float *const *d_loss);
/* Record n_iter iterations of every member (Adam steps first_step ..
 * first_step + n_iter - 1) into one CUDA graph by stream capture; nothing runs.
 * The graph keeps the device pointers: keep the buffers for its launches.
 * AF_ERR_STATE if a member's stage timing is on.  Replaces a previous graph. */
af_status af_batch_capture(af_batch_t batch, const void *const *d_iq, const float *const *d_iq_scale,
                           float *const *d_s, float *const *d_grad, float *const *d_m,
                           float *const *d_v, float *const *d_loss, int first_step, int n_iter);
/* Launch the captured graph, ordered after the caller stream's earlier work and
 * before its later work.  AF_ERR_STATE if nothing was captured. */
af_status af_batch_launch(af_batch_t batch);
/* Release the batch, its plans, streams and graph.  NULL is accepted. */
af_status af_batch_destroy(af_batch_t batch);

/* Move the image points of a plan (same n_patch x patch_npix, host arrays, read
 * during the call).  Used by the global-speed sweep of Sec. II-C / III-A, whose
 * dynamic grid scales pixel and kernel positions with the active speed.  The
 * same validation as af_plan applies (inside the grid box, outside the lens);
 * synchronises the plan's stream. */
af_status af_set_pixels(af_plan_t plan, const double *pix_x, const double *pix_z);

/* Global-speed sweep (Sec. II-C, III-A; Fig. 3): L_CMPE of the uniform map 1/c0
 * for each of the n_speeds speeds in h_speeds (host, m/s), one forward pass each,
 * all queued on the plan's stream without host round trips between speeds.
 *  dynamic = 1: the dynamic CMPE grid.  Before the pass at c0 every patch keeps
 *    its direction from the lens centre (its lateral position for a flat lens),
 *    its depth below the lens surface is multiplied by k = c0 / c_ref, and its
 *    pixels' offsets from the patch centre (the mean of its pixels) by k, so
 *    each patch observes the same echoes at every c0.  The plan's pixels are
 *    those of c_ref.  Every moved pixel set is validated on the host first (the
 *    checks of af_set_pixels; the grid box must cover them).  dynamic = 0: the
 *    plan's pixels at every speed.
 *  d_cmpe [n_speeds] float (device): L_CMPE per speed; d_active [n_speeds] int
 *    (device, may be NULL): active CMPE terms per speed.
 * Afterwards the plan's pixels are restored and the next af_forward starts
 * without an exit-angle warm start.  Needs a curved or flat lens surface for
 * dynamic = 1 (AF_ERR_ARG otherwise).  The two extreme speeds are validated
 * before any work is queued; a speed in between that fails stops the sweep
 * with the error, with the plan's pixels restored and earlier speeds' results
 * written.  Each speed's exit solve starts from the previous speed's exit angles. */
af_status af_sweep(af_plan_t plan, const void *d_iq, const float *d_iq_scale, const double *h_speeds,
                   int n_speeds, double c_ref, int dynamic, float *d_cmpe, int *d_active);

/* Waits for the plan's stream and returns AF_ERR_NUMERIC if a kernel flagged
 * a non-positive or non-finite slowness since the last call, else AF_OK. */
af_status af_sync_status(af_plan_t plan);

/* ---- introspection of the last af_forward / af_adjoint (device outputs) ---- */

/* One-way delays T[e][p] (s, element -> lens -> pixel, Eq. 7-8 + Eq. 1) as
 * double, and the apodization bits h_e(r_p) (Eq. 4), both [n_elem][npix].
 * Either pointer may be NULL. */
af_status af_get_delays(af_plan_t plan, double *d_T, uint8_t *d_apod);

/* Lens exit points, [n_elem][npix] float: the exit angle (rad, about the arc
 * centre) for AF_LENS_BENT_RAY, the exit x (m, on the line z = lens_z) for
 * AF_LENS_PLANAR, 0 for AF_LENS_NONE. */
af_status af_get_exit_angles(af_plan_t plan, float *d_phi);

/* Subaperture images B[b][p] as interleaved float (re, im), b = i*nsub + j,
 * [nsub*nsub][npix][2]. */
af_status af_get_images(af_plan_t plan, float *d_B);

/* CMPE cross terms z[P][k] ([n_patch][npair][2] float) and correlation mask
 * bits ([n_patch][npair] uint8); *h_n_active (host) = number of set bits.
 * Any pointer may be NULL.  Synchronises the plan's stream. */
af_status af_get_cmpe(af_plan_t plan, float *d_z, uint8_t *d_mask, int *h_n_active);

/* Images of the last af_forward, [npix] float each (either may be NULL):
 *  d_bmode       |sum_ij B_ij(p)|, the full-aperture DAS envelope (Figs. 2, 4);
 *  d_cmpe_image  integrated CMPE (Sec. IV): sum over the common-midpoint pairs
 *                of |arg(B_ij(p) conj(B_i+1,j-1(p)))|, per pixel.
 * A plan over a dense pixel grid gives the full field of view. */
af_status af_get_bmode(af_plan_t plan, float *d_bmode, float *d_cmpe_image);

/* Image-quality metrics of the last af_forward (Sec. III-F, Model Evaluation;
 * the paper defines MAE and cites the other metrics, read here as follows).
 * S_j(p) = sum_i B_ij(p) is the image of receive subaperture j.
 *  cf_mean      mean over the background of |sum_j S_j|^2 / (n_sub sum_j |S_j|^2)
 *               (coherence factor over receive subapertures);
 *  loc          mean over j of Re sum_p S_j conj(S_j+1) /
 *               sqrt(sum_p |S_j|^2 sum_p |S_j+1|^2), p over the background
 *               (lag-one coherence over receive subapertures);
 *  cmcc         mean over patches and common-midpoint pairs of the CMPE
 *               correlation coefficient rho;
 *  contrast_db  20 log10(mean_in / mean_out) of the envelope |sum_ij B_ij|;
 *  cnr          |mean_in - mean_out| / sqrt(var_in + var_out) (population
 *               variances);
 *  gcnr         1 - sum_b min(h_in(b), h_out(b)), h the normalised histograms of
 *               the envelope over nbins equal bins spanning its range over both
 *               regions (generalized CNR).
 * d_roi [npix] uint8 (device): 1 target region, 2 background, 0 unused.
 * Quantities of an empty region are NaN.  Allocates and frees its own device
 * scratch (about (2 n_sub + 8) x npix floats); synchronises the plan's stream.
 * Errors: AF_ERR_ARG (NULL, nbins outside [2, 65536]), AF_ERR_STATE (no forward
 * pass yet), AF_ERR_CUDA. */
typedef struct {
    double cf_mean, loc, cmcc, contrast_db, cnr, gcnr, mean_in, mean_out;
    long long n_in, n_out;
} af_metrics;
af_status af_image_metrics(af_plan_t plan, const uint8_t *d_roi, int nbins, af_metrics *h_out);

/* Sound-speed MAE (Sec. III-F): mean over the plan's pixels of
 * |1 / bicubic(s, r_p) - c_true[p]| (Keys a = -1/2, clamp to edge, the
 * interpolation of Sec. III-A).  d_s [nz][nx] and d_c_true [npix] float on the
 * device; the result is written to *h_mae (host).  Synchronises the plan's
 * stream; allocates npix floats of scratch. */
af_status af_speed_mae(af_plan_t plan, const float *d_s, const float *d_c_true, double *h_mae);

/* ---- patch-sharded runs (one acquisition over several GPUs) ----
 * L_CMPE (Sec. II-D) is a sum over patches normalised by the total number M of
 * active terms, so a problem whose patches are split over several plans (one per
 * GPU, each with its own patch subset and the same grid, array and channel data)
 * needs two exchanges per iteration:
 *   af_forward on every plan;  af_cmpe_totals -> d_totals[2] = {sum over the plan's
 *   active terms of |arg z|, number of active terms} (device doubles);  sum the
 *   totals over the plans (e.g. an all-reduce);  af_set_cmpe_totals with the sums:
 *   the plan's L_CMPE = sum / max(1, M) and its adjoint's normalisation become those
 *   of the whole problem, and d_loss ([4] float, may be NULL) is rewritten as
 *   af_forward writes it;  af_adjoint on every plan;  sum the d_grad of the plans;
 *   af_step with the summed gradient on every plan (identical updates).
 * Give the regularisers (w1, w2) to one plan only, or their gradient is counted
 * once per plan.  Both calls are asynchronous on the plan's stream and need an
 * earlier af_forward (AF_ERR_STATE).  No counterpart in the paper, which runs on
 * one device. */
af_status af_cmpe_totals(af_plan_t plan, double *d_totals);
af_status af_set_cmpe_totals(af_plan_t plan, const double *d_totals, float *d_loss);

/* dL/dB[b][p] (= dL/dRe B + j dL/dIm B) of the last af_adjoint,
 * [nsub*nsub][npix][2] float. */
af_status af_get_image_grad(af_plan_t plan, float *d_G);

/* dL/dT[e][p] of the last af_adjoint, [n_elem][npix] float. */
af_status af_get_delay_grad(af_plan_t plan, float *d_g);

/* Host: counters of the last af_forward (synchronises the stream):
 *  [0] apodized (element, pixel) pairs, [1] exit solves that fell back to
 *  float64, [2] active CMPE terms, [3] number of CMPE pairs per patch. */
af_status af_get_counters(af_plan_t plan, long long *h_counters);

/* Per-stage device timing with CUDA events recorded on the plan's stream.
 * af_set_timing(plan, 1) clears the record and starts recording every kernel
 * stage of later calls; 0 stops.  af_get_stage_times synchronises the stream
 * and writes, per stage, the summed milliseconds (h_ms) and launch counts
 * (h_count) since recording started.  Stages (AF_NSTAGES = 8):
 *  0 grid statistics (c_med, Eq. 10-11)   1 delays (Eq. 1-4, 8)
 *  2 DAS forward (Eq. 5)                   3 CMPE forward + loss
 *  4 (none: dL/dB is formed in stage 5)   5 DAS adjoint with dL/dB
 *  6 ray adjoint + gradient reduction      7 Adam update (Eq. 9)
 *  8 lens-surrogate inference (when enabled) */
#define AF_NSTAGES 9
af_status af_set_timing(af_plan_t plan, int enable);
af_status af_get_stage_times(af_plan_t plan, float *h_ms, int *h_count);

/* ---- allocation-free CMPE loss ----
 *
 * No counterpart in the paper: an extra entry point for callers that cannot
 * allocate device memory while they run (a real-time pipeline that reserves
 * all of its GPU memory at start-up, or a host framework that owns the device
 * allocator).  It computes L_CMPE of caller-provided subaperture images with
 * the same reading of the CMPE as af_forward, using no plan and no allocation:
 * its scratch (per-patch partial sums) is a fixed array of
 * AF_NOALLOC_MAX_PATCHES x 16 bytes inside the library's device memory, held
 * by every GPU that loads the library until the process exits.
 *  d_B        images, [nsub*nsub][n_patch*patch_npix][2] float (as af_get_images)
 *  d_loss     [1] float, written with L_CMPE
 *  d_n_active [1] int, number of active CMPE terms, or NULL
 *  stream     cudaStream_t (NULL = legacy default stream)
 * Every call looks up the scratch array's device address on the current device
 * (no allocation); the first call on a device may load the library's device code
 * there, so make it before any stream capture.  All calls share the scratch: calls that
 * overlap on the GPU race, so order them on one stream.  n_patch above
 * AF_NOALLOC_MAX_PATCHES returns AF_ERR_UNSUPPORTED.  No cudaMalloc/cudaFree. */
#define AF_NOALLOC_MAX_PATCHES 16384
af_status af_cmpe_loss_noalloc(const float *d_B, int nsub, int n_patch, int patch_npix,
                               double rho_thresh, float *d_loss, int *d_n_active, void *stream);

/* ---- learned lens surrogate (MLP on the tensor cores) ----
 * A 4-layer MLP (4 -> 128 -> 128 -> 128 -> 2, tanh) standing in for the exit-
 * point solve of Eq. 8: inputs element angle, pixel radius, pixel angle
 * relative to the element (about the arc centre) and c_med; outputs the exit
 * angle offset and the lens transit time.  The 128 x 128 layers run as bf16
 * tcgen05 MMAs with f32 accumulation (forward and backward).  No counterpart in
 * the paper, which solves Eq. 8 directly.
 *
 * af_surrogate_train: requires one earlier af_forward (its apodization defines
 *   the validated pairs).  Draws n_samples configurations inside the f-number
 *   cone with c in [1400, 1650] m/s, labels them with the float64 exact solver,
 *   trains `epochs` passes of Adam (batch tiles_per_step x 128, cosine decay
 *   from lr), then validates on every apodized pair at six speeds and marks
 *   pairs whose delay error exceeds lambda/50 (1 / (50 fd)) for the exact
 *   solver.  h_report[8] = {final training loss, rms exit-angle error (rad),
 *   max delay error (s), max lens-time error (s), fallback fraction, samples,
 *   tolerance (s), optimisation steps}.  Allocates and frees temporaries.
 * af_surrogate_enable: 1 = af_forward uses the surrogate's exit angle (exact
 *   solver on marked pairs; path lengths are always computed exactly), 0 = off.
 * af_surrogate_eval: exit angle (rad) and lens time (s) of every (element,
 *   pixel) pair at medium speed c, into [n_elem][npix] float arrays.
 * af_surrogate_params: copy the AF_MLP_NPARAM float parameters out (set = 0)
 *   or in (set = 1).  Layout: W1[128][4], b1[128], W2[128][128], b2[128],
 *   W3[128][128], b3[128], W4[2][128], b4[2].
 * af_surrogate_grad: gradient of the training loss (mean over the n samples of
 *   the squared error of both normalised outputs) at the current parameters
 *   for a caller batch d_X[n][4], d_Y[n][2] (normalised), n a multiple of 128;
 *   *h_loss receives the loss.  Parameters are not changed. */
#define AF_MLP_NPARAM 33922
af_status af_surrogate_train(af_plan_t plan, long long n_samples, int epochs, int tiles_per_step, float lr,
                             unsigned long long seed, double *h_report);
af_status af_surrogate_enable(af_plan_t plan, int enable);
af_status af_surrogate_eval(af_plan_t plan, float c, float *d_phi, float *d_tlens);
af_status af_surrogate_params(af_plan_t plan, float *d_params, int set);
af_status af_surrogate_grad(af_plan_t plan, const float *d_X, const float *d_Y, int n, float *d_grad,
                            float *h_loss);

/* ---- BF16 tensor-core GEMM (building block of the lens-surrogate MLP) ----
 * D[M][N] (float) = sum_k A(m,k) B(n,k) on the sm_103a tensor cores (tcgen05,
 * f32 accumulation in tensor memory).  A is bf16 [M][K] (a_mn_major = 0) or
 * [K][M] (1); B is bf16 [N][K] (b_mn_major = 0) or [K][N] (1); D is [M][N].
 * M, N multiples of 128, K a multiple of 64, operands 16-byte aligned.
 * *d_err (device int, caller-zeroed) is set to 1 if an MMA completion wait
 * timed out.  No counterpart in the paper: it is the building block of the
 * learned lens-time model (the MLP surrogate below). */
af_status af_gemm_bf16(const void *d_A, const void *d_B, float *d_D, int M, int N, int K,
                       int a_mn_major, int b_mn_major, int *d_err, void *stream);

/* Test hook for the bounded waits of the tensor-core kernels (af_gemm_bf16, the
 * lens-surrogate training and inference).  Each waits for its MMAs with a bounded
 * number of tries; on a timeout it reports the error (*d_err = 1 for
 * af_gemm_bf16, AF_ERR_TIMEOUT from af_surrogate_train), waits again with the
 * default bound for the MMAs in flight, frees its tensor memory and returns.
 * tries >= 0 sets the number of tries of that first wait for every such kernel the
 * process launches afterwards (0: it gives up at once, so a test can run the
 * error path); tries < 0 restores the default (2^26 tries, about a second).  No
 * counterpart in the paper. */
af_status af_set_wait_limit(int tries);

/* Ray adjoint: flush window of the shared-memory fixed-point grids, in rays of
 * the largest |dL/dT|.  A CTA adds its integer grids into the global one before
 * a block of rays whose summed |dL/dT| / max|dL/dT| would take the total since
 * its last flush past this window.  The default (and maximum) is the window the
 * fixed-point scale is sized for; rays > that maximum set the maximum, 0 flushes
 * before every block.  A smaller window only flushes more often: the integer
 * sums, and so dL/ds, do not change (a test uses it to run the flush path on
 * small problems).  AF_ERR_ARG for a NULL plan or rays < 0 (or NaN).  No
 * counterpart in the paper. */
af_status af_set_ray_flush_budget(af_plan_t plan, double rays);

/* Measured FP32 lane rate of the current device: lane-operations (one fused
 * multiply-add on one lane) per second of a plain, dependency-free FMA loop over
 * 8 CTAs per SM, timed with CUDA events on `stream`.  It is the denominator of
 * the rooflines of this library's kernels, which are bound by FP32 issue.
 * d_sink: one device float the kernel may write (it keeps the loop from being
 * removed).  *h_rate (host) receives the rate; synchronises the stream.  No
 * counterpart in the paper. */
af_status af_fp32_lane_rate(float *d_sink, void *stream, double *h_rate);

/* Message of the last failing call on this host thread ("" if none). */
const char *af_last_error(void);

/* Static name of a status code. */
const char *af_status_string(af_status s);

#ifdef __cplusplus
}
#endif
#endif /* AF_H */
