// C ABI of the autofocus library (declared in include/af.h): argument
// validation, plan construction (device geometry and workspaces) and the call
// sequence of one iteration.  Everything numeric runs in the kernels of the
// sibling .cu files; this file only validates, allocates and launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "af_internal.cuh"

namespace {

thread_local char g_err[512] = "";

af_status fail(af_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

af_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(AF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define AF_CUDA(call)                                         \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);   \
    } while (0)

bool is_fin(double x) { return std::isfinite(x); }

// float-float split of a double
void split_ff(double v, float *hi, float *lo)
{
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
}

long long n_pairs(const af_config *c)
{
    const int n = c->n_elem / c->sub_width;
    return n >= 3 ? (long long)(n - 1) * (n - 2) : 0;
}

// padded row length: two edge nodes on each side, rounded up to an odd number
// of floats so that successive rows start in different shared-memory banks
int padded_pitch(int nx) { return (nx + 4) | 1; }

size_t padded_grid_bytes(const af_config *c)
{
    return (size_t)padded_pitch(c->nx) * (size_t)(c->nz + 4) * sizeof(float);
}

constexpr size_t kMaxGridSmem = 200 * 1024;

// Run one stage launcher, bracketed by events when timing is on.
template <typename F>
cudaError_t staged(af_plan_t pl, int stage, F &&launch)
{
    const bool rec = pl->timing && pl->n_rec < kTimingCap;
    if (rec) {
        cudaError_t e = cudaEventRecord(pl->ev[2 * pl->n_rec], pl->stream);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch();
    if (e != cudaSuccess) return e;
    if (rec) {
        e = cudaEventRecord(pl->ev[2 * pl->n_rec + 1], pl->stream);
        if (e != cudaSuccess) return e;
        pl->rec_stage[pl->n_rec++] = stage;
    }
    return cudaSuccess;
}

}  // namespace

af_status af_set_error(af_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

extern "C" {

const char *af_last_error(void) { return g_err; }

const char *af_status_string(af_status s)
{
    switch (s) {
    case AF_OK: return "AF_OK";
    case AF_ERR_ARG: return "AF_ERR_ARG";
    case AF_ERR_SHAPE: return "AF_ERR_SHAPE";
    case AF_ERR_DTYPE: return "AF_ERR_DTYPE";
    case AF_ERR_CUDA: return "AF_ERR_CUDA";
    case AF_ERR_NUMERIC: return "AF_ERR_NUMERIC";
    case AF_ERR_TIMEOUT: return "AF_ERR_TIMEOUT";
    case AF_ERR_UNSUPPORTED: return "AF_ERR_UNSUPPORTED";
    case AF_ERR_STATE: return "AF_ERR_STATE";
    }
    return "AF_ERR_UNKNOWN";
}

af_status af_check_config(const af_config *c)
{
    g_err[0] = 0;
    if (!c) return fail(AF_ERR_ARG, "config is NULL");
    if (c->n_elem < 1) return fail(AF_ERR_SHAPE, "n_elem = %d < 1", c->n_elem);
    if (!c->elem_x || !c->elem_z) return fail(AF_ERR_ARG, "elem_x / elem_z is NULL");
    if (c->sub_width < 1) return fail(AF_ERR_SHAPE, "sub_width = %d < 1", c->sub_width);
    if (c->n_elem % c->sub_width) return fail(AF_ERR_SHAPE, "n_elem %d is not a multiple of sub_width %d", c->n_elem, c->sub_width);
    if (c->sub_width != 1 && c->sub_width != 2 && c->sub_width != 4 && c->sub_width != 8 && c->sub_width != 16)
        return fail(AF_ERR_UNSUPPORTED, "sub_width %d not in {1, 2, 4, 8, 16}", c->sub_width);
    if (c->n_elem / c->sub_width > 32) return fail(AF_ERR_UNSUPPORTED, "more than 32 subapertures (%d)", c->n_elem / c->sub_width);
    if (c->n_elem > 1024) return fail(AF_ERR_UNSUPPORTED, "n_elem %d > 1024", c->n_elem);
    if (c->n_patch < 0 || c->patch_npix < 1) return fail(AF_ERR_SHAPE, "n_patch %d / patch_npix %d", c->n_patch, c->patch_npix);
    if (c->n_patch > 0 && (!c->pix_x || !c->pix_z)) return fail(AF_ERR_ARG, "pix_x / pix_z is NULL");
    if (c->nx < 2 || c->nz < 2) return fail(AF_ERR_SHAPE, "grid %d x %d smaller than 2 x 2", c->nx, c->nz);
    if (padded_grid_bytes(c) > kMaxGridSmem) return fail(AF_ERR_UNSUPPORTED, "grid %d x %d does not fit in shared memory", c->nx, c->nz);
    if (!(c->dx > 0) || !(c->dz > 0) || !is_fin(c->x0) || !is_fin(c->z0)) return fail(AF_ERR_ARG, "bad grid spacing / origin");
    if (c->nseg < 1) return fail(AF_ERR_ARG, "nseg = %d < 1", c->nseg);
    if (c->n_samp < 2) return fail(AF_ERR_SHAPE, "n_samp = %d < 2", c->n_samp);
    if (!(c->fs > 0) || !is_fin(c->fs) || !is_fin(c->fd) || !is_fin(c->t0) || !is_fin(c->t_ttp))
        return fail(AF_ERR_ARG, "bad fs / fd / t0 / t_ttp");
    if (c->iq_dtype != AF_IQ_C64 && c->iq_dtype != AF_IQ_BF16 && c->iq_dtype != AF_IQ_F16)
        return fail(AF_ERR_DTYPE, "unknown iq_dtype %d", c->iq_dtype);
    if (c->lens_mode != AF_LENS_BENT_RAY && c->lens_mode != AF_LENS_NONE) return fail(AF_ERR_ARG, "unknown lens_mode %d", c->lens_mode);
    if (c->apod_mode != AF_APOD_FNUMBER && c->apod_mode != AF_APOD_PRINTED) return fail(AF_ERR_ARG, "unknown apod_mode %d", c->apod_mode);
    if (!(c->fnum > 0) || !is_fin(c->fnum)) return fail(AF_ERR_ARG, "fnum must be > 0");
    if (!is_fin(c->rho_thresh)) return fail(AF_ERR_ARG, "rho_thresh not finite");
    const double regs[] = {c->w1, c->kx1, c->kz1, c->w2, c->kx2, c->kz2, c->lr};
    for (double r : regs)
        if (!(r >= 0) || !is_fin(r)) return fail(AF_ERR_ARG, "regulariser weights, thresholds and lr must be finite and >= 0");
    if (!(c->beta1 >= 0 && c->beta1 < 1) || !(c->beta2 >= 0 && c->beta2 < 1) || !(c->eps > 0) || !(c->c_ref > 0))
        return fail(AF_ERR_ARG, "bad Adam parameters");
    const long long npix = (long long)c->n_patch * c->patch_npix;
    const long long nsub = c->n_elem / c->sub_width;
    if ((long long)c->n_elem * npix >= (1LL << 31) || nsub * nsub * npix >= (1LL << 31))
        return fail(AF_ERR_UNSUPPORTED, "too many pixels");
    const double gx1 = c->x0 + (c->nx - 1) * c->dx, gz1 = c->z0 + (c->nz - 1) * c->dz;
    auto inside = [&](double x, double z) { return x >= c->x0 && x <= gx1 && z >= c->z0 && z <= gz1; };
    double emin = 1e300, emax = -1e300, remax = 0;
    for (int a = 0; a < c->n_elem; ++a) {
        if (!is_fin(c->elem_x[a]) || !is_fin(c->elem_z[a])) return fail(AF_ERR_ARG, "element %d not finite", a);
        const double th = atan2(c->elem_x[a] - c->arc_cx, c->elem_z[a] - c->arc_cz);
        emin = fmin(emin, th);
        emax = fmax(emax, th);
        remax = fmax(remax, hypot(c->elem_x[a] - c->arc_cx, c->elem_z[a] - c->arc_cz));
        if (c->lens_mode == AF_LENS_NONE && !inside(c->elem_x[a], c->elem_z[a]))
            return fail(AF_ERR_ARG, "element %d outside the slowness grid", a);
    }
    if (c->lens_mode == AF_LENS_BENT_RAY) {
        if (!(c->c_lens > 0) || !is_fin(c->c_lens) || !is_fin(c->arc_cx) || !is_fin(c->arc_cz))
            return fail(AF_ERR_ARG, "bad lens parameters");
        if (!(c->lens_radius >= remax * (1 - 1e-7)))
            return fail(AF_ERR_ARG, "lens_radius %.9g below the element radius %.9g", c->lens_radius, remax);
    }
    double pmin = emin, pmax = emax;
    for (long long p = 0; p < npix; ++p) {
        const double x = c->pix_x[p], z = c->pix_z[p];
        if (!is_fin(x) || !is_fin(z)) return fail(AF_ERR_ARG, "pixel %lld not finite", p);
        if (!inside(x, z)) return fail(AF_ERR_ARG, "pixel %lld outside the slowness grid", p);
        if (c->lens_mode == AF_LENS_BENT_RAY) {
            if (!(hypot(x - c->arc_cx, z - c->arc_cz) > c->lens_radius))
                return fail(AF_ERR_ARG, "pixel %lld inside the lens", p);
            const double th = atan2(x - c->arc_cx, z - c->arc_cz);
            pmin = fmin(pmin, th);
            pmax = fmax(pmax, th);
        }
    }
    if (c->lens_mode == AF_LENS_BENT_RAY) {
        // every possible exit point lies on the lens arc between the extreme angles
        for (int k = 0; k <= 256; ++k) {
            const double th = pmin + (pmax - pmin) * k / 256.0;
            if (!inside(c->arc_cx + c->lens_radius * sin(th), c->arc_cz + c->lens_radius * cos(th)))
                return fail(AF_ERR_ARG, "lens surface at angle %.6f rad outside the slowness grid", th);
        }
    }
    return AF_OK;
}

af_status af_workspace_bytes(const af_config *c, size_t *bytes)
{
    af_status st = af_check_config(c);
    if (st != AF_OK) return st;
    if (!bytes) return fail(AF_ERR_ARG, "bytes is NULL");
    const size_t ne = c->n_elem, npix = (size_t)c->n_patch * c->patch_npix;
    const size_t nsub = ne / c->sub_width, nb = nsub * nsub, npair = (size_t)n_pairs(c);
    const size_t ng = (size_t)c->nx * c->nz;
    size_t b = 0;
    b += ne * (sizeof(float4) + sizeof(float2)) + npix * 2 * sizeof(float2);
    b += ne * npix * (sizeof(float) + sizeof(float4) + sizeof(float));   // phi, D, gdel
    b += 2 * nb * npix * sizeof(float2);                                  // B, G
    b += (size_t)c->n_patch * npair * (sizeof(float2) + 1);               // z, mask
    b += (size_t)c->n_patch * (sizeof(double) + sizeof(int));
    b += 148 * 8 * ng * sizeof(float);                                     // partial grids (upper bound)
    b += sizeof(AfScal);
    *bytes = b;
    return AF_OK;
}

af_status af_destroy(af_plan_t pl)
{
    if (!pl) return AF_OK;
    for (int k = 0; k < 2 * kTimingCap; ++k)
        if (pl->ev[k]) cudaEventDestroy(pl->ev[k]);
    void *ptrs[] = {pl->elem, pl->elem_pol, pl->pix, pl->pix_pol, pl->phi, pl->D, pl->B, pl->G, pl->z,
                    pl->mask, pl->patch_sum, pl->patch_cnt, pl->gdel, pl->gpart, pl->gpad, pl->scal};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete pl;
    return AF_OK;
}

af_status af_plan(const af_config *c, void *stream, af_plan_t *out)
{
    if (!out) return fail(AF_ERR_ARG, "out is NULL");
    *out = nullptr;
    af_status st = af_check_config(c);
    if (st != AF_OK) return st;

    af_plan_t pl = new af_plan_s();
    memset(pl, 0, sizeof(*pl));
    pl->stream = (cudaStream_t)stream;
    pl->iq_dtype = c->iq_dtype;
    AfGeom &g = pl->g;
    const int ne = c->n_elem, npix = c->n_patch * c->patch_npix;
    g.ne = ne;
    g.npix = npix;
    g.W = c->sub_width;
    g.nsub = ne / c->sub_width;
    g.nb = g.nsub * g.nsub;
    g.npair = (int)n_pairs(c);
    g.n_patch = c->n_patch;
    g.patch_npix = c->patch_npix;
    g.ns = c->n_samp;
    g.nx = c->nx;
    g.nz = c->nz;
    g.ng = c->nx * c->nz;
    g.nseg = c->nseg;
    g.pitch = padded_pitch(c->nx);
    g.lens_mode = c->lens_mode;
    g.apod_mode = c->apod_mode;
    g.arc_cx = (float)c->arc_cx;
    g.arc_cz = (float)c->arc_cz;
    g.RL = (float)c->lens_radius;
    g.fnum_inv2 = (float)(1.0 / (2.0 * c->fnum));
    g.fnum_half = (float)(0.5 * c->fnum);
    g.x0 = (float)c->x0;
    g.z0 = (float)c->z0;
    g.inv_dx = (float)(1.0 / c->dx);
    g.inv_dz = (float)(1.0 / c->dz);
    g.inv_c_lens = c->lens_mode == AF_LENS_BENT_RAY ? (float)(1.0 / c->c_lens) : 0.0f;
    g.fs = (float)c->fs;
    g.wd = (float)(2.0 * 3.14159265358979323846 * c->fd);
    if (c->lens_mode == AF_LENS_BENT_RAY) split_ff(c->fs / c->c_lens, &g.fs_clens_hi, &g.fs_clens_lo);
    split_ff(0.5 * (c->t_ttp - c->t0) * c->fs, &g.off_hi, &g.off_lo);
    split_ff(c->fd / c->fs, &g.rfd_hi, &g.rfd_lo);
    {
        double cyc = 0.5 * c->fd * c->t0;
        g.cyc0 = (float)(cyc - floor(cyc));
    }
    g.rho_thresh = (float)c->rho_thresh;
    g.inv_nseg = (float)(1.0 / c->nseg);
    g.inv_nseg1 = (float)(1.0 / (c->nseg + 1));
    g.w1 = (float)c->w1;
    g.kx1 = (float)c->kx1;
    g.kz1 = (float)c->kz1;
    g.w2 = (float)c->w2;
    g.kx2 = (float)c->kx2;
    g.kz2 = (float)c->kz2;
    g.hx_mm = (float)(c->dx * 1e3);
    g.hz_mm = (float)(c->dz * 1e3);
    {
        const long na = (long)(c->nx - 1) * c->nz + (long)c->nx * (c->nz - 1);
        const long nbv = (long)(c->nx > 2 ? c->nx - 2 : 0) * c->nz + (long)c->nx * (c->nz > 2 ? c->nz - 2 : 0);
        g.na_inv = na > 0 ? (float)(1.0 / na) : 0.0f;
        g.nb_inv = nbv > 0 ? (float)(1.0 / nbv) : 0.0f;
    }
    {
        // one ray adds at most |dL/dT| (5 cell diagonals + L / (N + 1)) to a node; a flush
        // window holds 8 rounds of 256 rays; single contributions stay below 2^21
        const double diag = sqrt(c->dx * c->dx + c->dz * c->dz);
        const double lmax = sqrt(pow((c->nx - 1) * c->dx, 2) + pow((c->nz - 1) * c->dz, 2));
        const double per_ray = 5.0 * diag + lmax / (c->nseg + 1);
        const double window = 8.0 * 256.0 * per_ray;
        const double s1 = ldexp(1.0, 30) / window;
        const double s2 = ldexp(1.0, 21) * (c->nseg + 1) / lmax;
        g.fix_scale = (float)fmin(s1, s2);
    }
    g.c_ref = (float)c->c_ref;
    g.lr = (float)c->lr;
    g.beta1 = (float)c->beta1;
    g.beta2 = (float)c->beta2;
    g.omb1 = (float)(1.0 - c->beta1);
    g.omb2 = (float)(1.0 - c->beta2);
    g.eps = (float)c->eps;

    // host geometry: Eq. 3 orientation (end elements extrapolated), polar coordinates
    std::vector<float4> elem(ne);
    std::vector<float2> elem_pol(ne), pix((size_t)npix), pix_pol((size_t)npix);
    std::vector<double> th(ne, 0.0);
    for (int a = 1; a + 1 < ne; ++a)
        th[a] = -atan((c->elem_z[a + 1] - c->elem_z[a - 1]) / (c->elem_x[a + 1] - c->elem_x[a - 1]));
    if (ne >= 3) {
        th[0] = 2 * th[1] - th[2];
        th[ne - 1] = 2 * th[ne - 2] - th[ne - 3];
    }
    for (int a = 0; a < ne; ++a) {
        elem[a] = make_float4((float)c->elem_x[a], (float)c->elem_z[a], (float)cos(th[a]), (float)sin(th[a]));
        const double ux = c->elem_x[a] - c->arc_cx, uz = c->elem_z[a] - c->arc_cz;
        elem_pol[a] = make_float2((float)atan2(ux, uz), (float)hypot(ux, uz));
    }
    for (int p = 0; p < npix; ++p) {
        pix[p] = make_float2((float)c->pix_x[p], (float)c->pix_z[p]);
        const double vx = c->pix_x[p] - c->arc_cx, vz = c->pix_z[p] - c->arc_cz;
        pix_pol[p] = make_float2((float)atan2(vx, vz), (float)hypot(vx, vz));
    }

    auto bail = [&](af_status s) { af_destroy(pl); return s; };
    cudaError_t e;
#define AF_ALLOC(ptr, bytes)                                                     \
    do {                                                                         \
        size_t _b = (bytes);                                                     \
        e = cudaMalloc((void **)&(ptr), _b > 0 ? _b : 16);                       \
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc " #ptr));     \
    } while (0)
    e = cudaGetDevice(&pl->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    const size_t nep = (size_t)ne * npix, nbp = (size_t)g.nb * npix;
    const size_t nzp = (size_t)g.n_patch * g.npair;
    AF_ALLOC(pl->elem, ne * sizeof(float4));
    AF_ALLOC(pl->elem_pol, ne * sizeof(float2));
    AF_ALLOC(pl->pix, npix * sizeof(float2));
    AF_ALLOC(pl->pix_pol, npix * sizeof(float2));
    AF_ALLOC(pl->phi, nep * sizeof(float));
    AF_ALLOC(pl->D, nep * sizeof(float4));
    AF_ALLOC(pl->gdel, nep * sizeof(float));
    AF_ALLOC(pl->B, nbp * sizeof(float2));
    AF_ALLOC(pl->G, nbp * sizeof(float2));
    AF_ALLOC(pl->z, nzp * sizeof(float2));
    AF_ALLOC(pl->mask, nzp);
    AF_ALLOC(pl->patch_sum, g.n_patch * sizeof(double));
    AF_ALLOC(pl->patch_cnt, g.n_patch * sizeof(int));
    AF_ALLOC(pl->scal, sizeof(AfScal));
    pl->smem_grid = padded_grid_bytes(c);
    pl->delay_blocks = pl->sm_count * delays_blocks_per_sm(pl->smem_grid);
    pl->rayadj_blocks = pl->sm_count * rayadj_blocks_per_sm(pl->smem_grid);
    AF_ALLOC(pl->gpart, (size_t)pl->rayadj_blocks * g.ng * sizeof(float));
    AF_ALLOC(pl->gpad, (size_t)pl->rayadj_blocks * pl->smem_grid);
#undef AF_ALLOC
    e = cudaMemcpy(pl->elem, elem.data(), ne * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->elem_pol, elem_pol.data(), ne * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && npix) e = cudaMemcpy(pl->pix, pix.data(), npix * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && npix) e = cudaMemcpy(pl->pix_pol, pix_pol.data(), npix * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(pl->scal, 0, sizeof(AfScal));
    if (e == cudaSuccess) e = cudaMemset(pl->gdel, 0, (nep ? nep : 1) * sizeof(float));
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan upload"));
    *out = pl;
    return AF_OK;
}

af_status af_forward(af_plan_t pl, const void *iq, const float *scale, const float *s, float *loss)
{
    g_err[0] = 0;
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!iq || !s || !loss) return fail(AF_ERR_ARG, "d_iq, d_slowness and d_loss must be non-NULL");
    if (pl->iq_dtype != AF_IQ_C64 && !scale) return fail(AF_ERR_DTYPE, "16-bit channel data needs d_iq_scale");
    pl->iq = iq;
    pl->iq_scale = scale;
    pl->slowness = s;
    pl->loss_out = loss;
    AF_CUDA(staged(pl, 0, [&] { return launch_grid_stats(pl, s); }));
    AF_CUDA(staged(pl, 1, [&] { return launch_delays(pl, s); }));
    AF_CUDA(staged(pl, 2, [&] { return launch_das_forward(pl); }));
    AF_CUDA(staged(pl, 3, [&] { return launch_cmpe_forward(pl, loss); }));
    pl->have_fwd = true;
    pl->have_adj = false;
    return AF_OK;
}

af_status af_adjoint(af_plan_t pl, float *grad)
{
    g_err[0] = 0;
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!grad) return fail(AF_ERR_ARG, "d_grad is NULL");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "af_adjoint called before af_forward");
    AF_CUDA(staged(pl, 4, [&] { return launch_cmpe_backward(pl); }));
    AF_CUDA(staged(pl, 5, [&] { return launch_das_adjoint(pl); }));
    AF_CUDA(staged(pl, 6, [&] { return launch_ray_adjoint(pl, pl->slowness, grad); }));
    pl->have_adj = true;
    return AF_OK;
}

af_status af_step(af_plan_t pl, const float *grad, float *s, float *m, float *v, int step)
{
    g_err[0] = 0;
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!grad || !s || !m || !v) return fail(AF_ERR_ARG, "d_grad, d_slowness, d_adam_m, d_adam_v must be non-NULL");
    if (step < 1) return fail(AF_ERR_ARG, "step = %d < 1", step);
    AF_CUDA(staged(pl, 7, [&] { return launch_adam(pl, grad, s, m, v, step); }));
    return AF_OK;
}

af_status af_iterate(af_plan_t pl, const void *iq, const float *scale, float *s, float *grad,
                     float *m, float *v, int step, float *loss)
{
    af_status st = af_forward(pl, iq, scale, s, loss);
    if (st != AF_OK) return st;
    st = af_adjoint(pl, grad);
    if (st != AF_OK) return st;
    return af_step(pl, grad, s, m, v, step);
}

af_status af_sync_status(af_plan_t pl)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    AF_CUDA(cudaStreamSynchronize(pl->stream));
    int flag = 0;
    AF_CUDA(cudaMemcpy(&flag, &pl->scal->numeric_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        AF_CUDA(cudaMemset(&pl->scal->numeric_flag, 0, sizeof(int)));
        return fail(AF_ERR_NUMERIC, "non-positive or non-finite slowness");
    }
    return AF_OK;
}

af_status af_get_delays(af_plan_t pl, double *T, uint8_t *apod)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "no forward pass yet");
    AF_CUDA(launch_export_delays(pl, T, apod));
    return AF_OK;
}

af_status af_get_exit_angles(af_plan_t pl, float *phi)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "no forward pass yet");
    const size_t n = (size_t)pl->g.ne * pl->g.npix;
    if (n == 0) return AF_OK;
    if (!phi) return fail(AF_ERR_ARG, "d_phi is NULL");
    AF_CUDA(cudaMemcpyAsync(phi, pl->phi, n * sizeof(float), cudaMemcpyDeviceToDevice, pl->stream));
    return AF_OK;
}

af_status af_get_images(af_plan_t pl, float *B)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "no forward pass yet");
    const size_t n = (size_t)pl->g.nb * pl->g.npix;
    if (n == 0) return AF_OK;
    if (!B) return fail(AF_ERR_ARG, "d_B is NULL");
    AF_CUDA(cudaMemcpyAsync(B, pl->B, n * sizeof(float2), cudaMemcpyDeviceToDevice, pl->stream));
    return AF_OK;
}

af_status af_get_cmpe(af_plan_t pl, float *z, uint8_t *mask, int *n_active)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "no forward pass yet");
    const size_t nzp = (size_t)pl->g.n_patch * pl->g.npair;
    if (z && nzp) AF_CUDA(cudaMemcpyAsync(z, pl->z, nzp * sizeof(float2), cudaMemcpyDeviceToDevice, pl->stream));
    if (mask && nzp) AF_CUDA(cudaMemcpyAsync(mask, pl->mask, nzp, cudaMemcpyDeviceToDevice, pl->stream));
    if (n_active) {
        AF_CUDA(cudaStreamSynchronize(pl->stream));
        AF_CUDA(cudaMemcpy(n_active, &pl->scal->n_active, sizeof(int), cudaMemcpyDeviceToHost));
    }
    return AF_OK;
}

af_status af_get_image_grad(af_plan_t pl, float *G)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_adj) return fail(AF_ERR_STATE, "no adjoint pass yet");
    const size_t n = (size_t)pl->g.nb * pl->g.npix;
    if (n == 0) return AF_OK;
    if (!G) return fail(AF_ERR_ARG, "d_G is NULL");
    AF_CUDA(cudaMemcpyAsync(G, pl->G, n * sizeof(float2), cudaMemcpyDeviceToDevice, pl->stream));
    return AF_OK;
}

af_status af_get_delay_grad(af_plan_t pl, float *gd)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_adj) return fail(AF_ERR_STATE, "no adjoint pass yet");
    const size_t n = (size_t)pl->g.ne * pl->g.npix;
    if (n == 0) return AF_OK;
    if (!gd) return fail(AF_ERR_ARG, "d_g is NULL");
    AF_CUDA(cudaMemcpyAsync(gd, pl->gdel, n * sizeof(float), cudaMemcpyDeviceToDevice, pl->stream));
    return AF_OK;
}

af_status af_set_timing(af_plan_t pl, int enable)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (enable && !pl->ev[0]) {
        for (int k = 0; k < 2 * kTimingCap; ++k) AF_CUDA(cudaEventCreate(&pl->ev[k]));
    }
    pl->timing = enable != 0;
    pl->n_rec = 0;
    return AF_OK;
}

af_status af_get_stage_times(af_plan_t pl, float *ms, int *count)
{
    if (!pl || !ms || !count) return fail(AF_ERR_ARG, "NULL argument");
    for (int k = 0; k < AF_NSTAGES; ++k) { ms[k] = 0.0f; count[k] = 0; }
    AF_CUDA(cudaStreamSynchronize(pl->stream));
    for (int r = 0; r < pl->n_rec; ++r) {
        float t = 0.0f;
        AF_CUDA(cudaEventElapsedTime(&t, pl->ev[2 * r], pl->ev[2 * r + 1]));
        ms[pl->rec_stage[r]] += t;
        count[pl->rec_stage[r]] += 1;
    }
    return AF_OK;
}

af_status af_get_counters(af_plan_t pl, long long *h)
{
    if (!pl || !h) return fail(AF_ERR_ARG, "NULL argument");
    AF_CUDA(cudaStreamSynchronize(pl->stream));
    AfScal sc;
    AF_CUDA(cudaMemcpy(&sc, pl->scal, sizeof(AfScal), cudaMemcpyDeviceToHost));
    h[0] = sc.n_apod;
    h[1] = sc.fp64_solves;
    h[2] = sc.n_active;
    h[3] = pl->g.npair;
    return AF_OK;
}

}  // extern "C"
