// Internal declarations of the sm_103a autofocus library: device geometry,
// the plan, float-float helpers and the host-side launchers of each kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "af.h"

// Apodization-off sentinel stored in the integer sample field of a one-way
// delay entry: any round trip that uses it lands below sample 0 and is
// skipped by the gather, so h_t h_r = 0 needs no separate mask lookup.
#define AF_APOD_OFF (-(1 << 29))

// Geometry and scalars every kernel reads (passed by value).
struct AfGeom {
    int ne, npix, nsub, W, nb, npair, n_patch, patch_npix;
    int ns, nx, nz, ng, nseg, pitch;         // pitch = padded grid row length (>= nx + 4, odd)
    int lens_mode, apod_mode;
    float arc_cx, arc_cz, RL, fnum_inv2, fnum_half;
    float lens_z;                            // flat lens: outer surface z = lens_z
    float x0, z0, inv_dx, inv_dz;
    float inv_c_lens;                        // for the FP64 fallback solve
    float fs, wd;                            // sample rate, 2 pi fd
    float fs_clens_hi, fs_clens_lo;          // fs / c_lens as float-float
    float off_hi, off_lo;                    // (t_ttp - t0) fs / 2 as float-float
    float rfd_hi, rfd_lo;                    // fd / fs as float-float
    float cyc0;                              // frac(fd t0 / 2)
    float rho_thresh;
    float inv_nseg, inv_nseg1;               // 1/N, 1/(N+1)
    // regularisation (Eq. 10-11): speed in units of c_unit m/s (km/s), positions in mm
    float w1, kx1, kz1, w2, kx2, kz2, hx_mm, hz_mm;
    float na_inv, nb_inv;                    // 1 / number of difference terms
    float fix_scale;                         // ray-adjoint fixed-point scale times max |dL/dT|
    float ray_flush_budget;                  // ray adjoint: flush window in rays of max |dL/dT| (<= kRayFlushBudget)
    float c_unit, inv_c_unit;                // Eq. 9-11 act on c = 1 / (c_unit s)
    float lr, beta1, beta2, omb1, omb2, eps; // Adam on that c; omb = 1 - beta, formed in double
    int optimizer;                           // AF_OPT_ADAM or AF_OPT_GD
};

constexpr int kStatBlocks = 64;     // CTAs of the grid-statistics partial sums
// partial sums of one grid-statistics CTA: {sum 1/s, Eq. 10 terms, Eq. 11 terms, bad-value flag}
struct alignas(32) StatPart {
    double c, a, b, bad;
};
constexpr int kTimingCap = 4096;   // recorded stage launches per timing window
constexpr size_t kMaxGridSmemBytes = 200 * 1024;   // largest padded slowness grid held in shared memory

// ray adjoint: pixels per work item, the window the fixed-point scale is sized
// for (kRayItemsPerFlush items, kRayFlushRays rays, each with the largest
// |dL/dT|; the kernel flushes when the rays since its last flush reach that
// window by their |dL/dT|), and the largest pair of integer grid copies it keeps
// in shared memory
constexpr int kRayGroup = 3;
constexpr int kRayItemsPerFlush = 1024;
constexpr double kRayFlushRays = (double)kRayItemsPerFlush * kRayGroup;
// Flush budget, in rays of the largest |dL/dT|: the window kRayFlushRays that the
// fixed-point scale is set for, kept a little below it against float rounding of
// the running bound.  Each ray also counts kRayRoundShare of a full ray: a full
// ray may add ~2^30 / kRayFlushRays (~3.5e5) units to a node, 1/1024 of that is
// ~340 units, more than the <= 33 units its rounding to integers can add.
constexpr float kRayFlushBudget = 0.999f * (float)kRayFlushRays;
constexpr float kRayRoundShare = 1.0f / 1024.0f;
constexpr size_t kRayDualMaxBytes = 180 * 1024;
struct DelayShape {
    bool pairs;          // grid as float2 node pairs (i, i + 2) or scalar
    int threads, blocks;
    size_t smem;
};
struct RayAdjShape {
    bool dual;           // two grid copies (row pitch 1 and 31 mod 32) or one
    int threads, blocks;
    size_t smem;         // dynamic shared memory per CTA
};

// lens-surrogate MLP: parameter count (4->128->128->128->2) and normalisation
#define AF_MLP_NPARAM 33922
struct MlpNorm {
    float th_c, th_s;      // element angle: (th_e - th_c) * th_s
    float r_c, r_s;        // pixel radius
    float dp_s;            // pixel angle relative to the element
    float c_c, c_s;        // medium speed
    float y0_s;            // exit-angle offset = y0 * y0_s (rad)
    float y1_c, y1_s;      // lens time = y1_c + y1 * y1_s (s)
};
struct MlpGeom {           // sampling region and lens constants (float64)
    double re, RL, inv_c_lens;
    double th_lo, th_hi, z_lo, z_hi, cone, c_lo, c_hi;
};

// Plan-owned device scalars.
struct AfScal {
    double cmpe_sum;     // sum over active CMPE terms of |arg z| (numerator of L_CMPE)
    float sbar;          // 1 / c_med, c_med = mean(1/s)  (Sec. III-A)
    float rtv, rsv;      // Eq. 10, Eq. 11
    float lcmpe;         // CMPE loss
    float inv_m;         // 1 / max(1, number of active CMPE terms)
    int n_active;
    int numeric_flag;    // set when a slowness is non-positive or non-finite
    int fp64_solves;     // exit solves that fell back to float64
    int n_apod;          // apodized (element, pixel) pairs
    int gmax_bits;       // max |dL/dT| of the last adjoint (float bits, >= 0)
    int mlp_err;         // a tensor-core completion wait of the MLP timed out
    int ray_next;        // next item block of the ray adjoint (zero between launches)
    unsigned stat_done;  // CTAs of the grid statistics done (zero between launches)
    unsigned cmpe_done;  // CTAs of the CMPE forward done (zero between launches)
    unsigned delay_done; // CTAs of the delay kernel done (zero between launches)
    unsigned long long delay_next;   // next (element, pixel) item of the delay kernel (zero between launches)
};

struct AfJobs;          // jobs from host memory (af_job_*): staging buffers, copy stream, events

struct af_plan_s {
    AfGeom g;
    af_config cfg;       // scalar copy of the configuration (host pointers cleared)
    double *host_ex, *host_ez;   // element positions kept for re-validation
    double *host_px, *host_pz;   // current pixel positions (re-validation, sweep)
    cudaStream_t stream;
    int device, sm_count;
    size_t smem_grid;    // bytes of the padded slowness grid in shared memory
    DelayShape delay;    // delay-kernel launch shape (grid layout, threads, CTAs)
    RayAdjShape rayadj;  // ray-adjoint launch shape (grid layout, threads, CTAs)
    // geometry
    float4 *elem;        // (x, z, cos theta_a, sin theta_a)  theta_a from Eq. 3
    float2 *elem_pol;    // (polar angle about the arc centre, radius)
    float2 *pix;         // (x, z)
    float2 *pix_pol;     // (polar angle, radius)
    // global-speed sweep (af_sweep): the plan's pixels while the sweep moves them,
    // per-patch centre geometry of the dynamic grid, a uniform slowness map
    float2 *pix_base, *pix_pol_base;
    double *sweep_geo;   // [n_patch][5] {centre x, centre z, unit x, unit z, distance}
    float *s_sweep;      // [ng]
    // workspaces
    float *phi;          // [ne][npix] exit angles
    float4 *D;           // [ne][npix] {sample index (int bits), fraction, Re P, Im P}
    int2 *nrange;        // [npix] {min n, min -n} over the pixel's live one-way sample indices n
    float2 *B, *G;       // [nb][npix] images and dL/dB
    float2 *z;           // [n_patch][npair] CMPE cross terms
    uint8_t *mask;       // [n_patch][npair]
    double *patch_sum;   // [n_patch] sum m |arg z|
    int *patch_cnt;      // [n_patch] sum m
    float *gdel;         // [ne][npix] dL/dT
    long long *gpad;     // [padded grid] fixed-point accumulator of the ray adjoint (all CTAs)
    AfScal *scal;
    StatPart *stat_part; // [kStatBlocks] partial sums of the grid statistics
    float *loss_out;     // last caller loss buffer
    const void *iq;      // last forward's inputs (kept for the adjoint)
    const float *iq_scale;
    const float *slowness;
    int iq_dtype;
    bool have_phi, have_fwd, have_adj;
    // lens surrogate
    float *mlp_p, *mlp_m, *mlp_v, *mlp_g;   // f32 parameters, Adam moments, last gradient
    void *mlp_w2b, *mlp_w3b;                // bf16 copies of the two tensor-core layers
    uint8_t *sur_fb;                        // [ne][npix] 1 = use the exact solver
    MlpNorm mlp_norm;
    MlpGeom mlp_geom;
    bool use_surrogate, sur_trained;
    AfJobs *jobs;        // created by af_job_reserve (or the first af_job_submit)
    // stage timing: a ring of (start, stop) event pairs per recorded launch
    bool timing;
    int n_rec;
    int rec_stage[kTimingCap];
    cudaEvent_t ev[2 * kTimingCap];
};

// ---- float-float arithmetic (Dekker / Knuth error-free transformations) ----
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float err = (a - (s - bb)) + (b - bb);
    return {s, err};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)   // |a| >= |b|
{
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b)
{
    float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.hi, b.hi);
    float lo = s.lo + a.lo + b.lo;
    return ff_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = ff_two_sum(a.hi, b);
    return ff_fast_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = ff_two_prod(a.hi, b.hi);
    float lo = p.lo + fmaf(a.hi, b.lo, a.lo * b.hi);
    return ff_fast_two_sum(p.hi, lo);
}
// sqrt(a) for a > 0 (one Newton correction of the float32 root)
__device__ __forceinline__ ff ff_sqrt(ff a)
{
    float r = sqrtf(a.hi);
    float e = fmaf(-r, r, a.hi) + a.lo;
    return ff_fast_two_sum(r, e / (2.0f * r));
}
// |(ax - bx, az - bz)| with float32 inputs, exact differences
__device__ __forceinline__ ff ff_dist(float ax, float az, float bx, float bz)
{
    ff dx = ff_two_sum(ax, -bx), dz = ff_two_sum(az, -bz);
    ff x2 = ff_two_prod(dx.hi, dx.hi);
    x2.lo = fmaf(2.0f * dx.hi, dx.lo, x2.lo);
    ff z2 = ff_two_prod(dz.hi, dz.hi);
    z2.lo = fmaf(2.0f * dz.hi, dz.lo, z2.lo);
    return ff_sqrt(ff_add(x2, z2));
}

// Keys cubic-convolution weights (a = -1/2) for taps -1, 0, 1, 2 at fraction t,
// factored with u = 1 - t: w0 = -t u^2 / 2, w3 = -t^2 u / 2,
// w1 = 1 - 5/2 t^2 + 3/2 t^3, and w2 = 1 - w0 - w1 - w3 (the weights sum to 1).
__device__ __forceinline__ void keys_weights(float t, float w[4])
{
    const float u = 1.0f - t;
    const float m = (-0.5f * t) * u;
    w[0] = m * u;
    w[3] = m * t;
    w[1] = fmaf(t * t, fmaf(1.5f, t, -2.5f), 1.0f);
    w[2] = (1.0f - m) - w[1];
}

// Keys weights of the two axes at once on the packed FP32 pipe: w[a] = (wx[a],
// wz[a]) for t = (tx, tz), the same round-to-nearest steps as keys_weights
__device__ __forceinline__ void keys_weights2(float2 t, float2 (&w)[4])
{
    const float2 one = make_float2(1.0f, 1.0f), neg = make_float2(-1.0f, -1.0f);
    const float2 u = __ffma2_rn(neg, t, one);
    const float2 m = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), t), u);
    w[0] = __fmul2_rn(m, u);
    w[3] = __fmul2_rn(m, t);
    w[1] = __ffma2_rn(__fmul2_rn(t, t), __ffma2_rn(make_float2(1.5f, 1.5f), t, make_float2(-2.5f, -2.5f)), one);
    w[2] = __ffma2_rn(neg, w[1], __ffma2_rn(neg, m, one));
}

// Programmatic dependent launch.  The kernels of an iteration are launched by
// launch_dependent(), so the GPU prepares a kernel's launch while the kernel
// before it in the stream is still running.  Such a kernel calls pdl_wait()
// before its first access to global memory: it returns once the kernel before
// has completed and its writes are visible (a no-op in a kernel launched without
// the attribute).  The kernel before triggers the launch implicitly when it
// completes.  An explicit trigger at the start of every CTA
// (griddepcontrol.launch_dependents) made a step 30 us slower on the 128-element
// workload; the implicit one makes it 12 us faster than plain launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t stream, Args... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// records the message returned by af_last_error() and returns st
af_status af_set_error(af_status st, const char *fmt, ...);

// tries of the first tensor-core completion wait (af_set_wait_limit; default about a second)
uint32_t af_wait_tries();

// releases a plan's job buffers, stream and events (af_destroy)
void jobs_release(af_plan_t pl);

// ---- launchers (each in its own .cu file) ----
cudaError_t launch_grid_stats(af_plan_t pl, const float *s);
cudaError_t launch_delays(af_plan_t pl, const float *s);
cudaError_t launch_das_forward(af_plan_t pl);
cudaError_t launch_cmpe_forward(af_plan_t pl, float *loss);
cudaError_t launch_cmpe_backward(af_plan_t pl);
cudaError_t launch_cmpe_totals(af_plan_t pl, double *out);
cudaError_t launch_cmpe_set_totals(af_plan_t pl, const double *in, float *loss);
cudaError_t launch_das_adjoint(af_plan_t pl);
cudaError_t launch_ray_adjoint(af_plan_t pl, const float *s, float *grad);
cudaError_t launch_adam(af_plan_t pl, const float *grad, float *s, float *m, float *v, int step);
cudaError_t launch_export_delays(af_plan_t pl, double *T, uint8_t *apod);
cudaError_t launch_images(af_plan_t pl, float *bmode, float *cimg);
// host copies of the pixel positions; the centre geometry of the dynamic grid
void sweep_patch_geometry(const af_config *c, const double *px, const double *pz, double *geo);
void sweep_moved_pixels(const af_config *c, const double *px, const double *pz, const double *geo, double k,
                        double *out_x, double *out_z);
DelayShape delays_shape(size_t smem_scalar, int sm_count);
cudaError_t mlp_setup_attributes();
cudaError_t mlp_refresh_bf16(af_plan_t pl);
cudaError_t mlp_init_params(af_plan_t pl, uint64_t seed);
cudaError_t mlp_generate(af_plan_t pl, long count, uint64_t seed, float4 *X, float2 *Y);
cudaError_t mlp_train_step(af_plan_t pl, const float4 *X, const float2 *Y, long first, int ntiles, float lr,
                           int step, float *lpart, float *gpart);
cudaError_t mlp_infer(af_plan_t pl, float c_fixed, const uint8_t *fb, float *phi_out, float *tl_out);
cudaError_t mlp_validate(af_plan_t pl, double c, const float *phi_s, const float *tl_s, double tol, uint8_t *fb,
                         unsigned long long *stats);
RayAdjShape rayadj_shape(int nx, int nz, int pitch, int sm_count);
