// C ABI of the autofocus library (declared in include/af.h): argument
// validation, plan construction (device geometry and workspaces) and the call
// sequence of one iteration.  Everything numeric runs in the kernels of the
// sibling .cu files; this file only validates, allocates and launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <vector>

#include "af_internal.cuh"
#include "af_tc.cuh"

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

static std::atomic<uint32_t> g_wait_tries{tc::kWaitTries};

uint32_t af_wait_tries() { return g_wait_tries.load(std::memory_order_relaxed); }

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
    if (padded_grid_bytes(c) > kMaxGridSmemBytes) return fail(AF_ERR_UNSUPPORTED, "grid %d x %d does not fit in shared memory", c->nx, c->nz);
    if (!(c->dx > 0) || !(c->dz > 0) || !is_fin(c->x0) || !is_fin(c->z0)) return fail(AF_ERR_ARG, "bad grid spacing / origin");
    if (c->nseg < 1) return fail(AF_ERR_ARG, "nseg = %d < 1", c->nseg);
    if (c->nseg > AF_MAX_NSEG) return fail(AF_ERR_UNSUPPORTED, "nseg = %d > %d", c->nseg, AF_MAX_NSEG);
    if (c->n_samp < 2) return fail(AF_ERR_SHAPE, "n_samp = %d < 2", c->n_samp);
    if (!(c->fs > 0) || !is_fin(c->fs) || !is_fin(c->fd) || !is_fin(c->t0) || !is_fin(c->t_ttp))
        return fail(AF_ERR_ARG, "bad fs / fd / t0 / t_ttp");
    if (c->iq_dtype != AF_IQ_C64 && c->iq_dtype != AF_IQ_BF16 && c->iq_dtype != AF_IQ_F16)
        return fail(AF_ERR_DTYPE, "unknown iq_dtype %d", c->iq_dtype);
    if (c->lens_mode != AF_LENS_BENT_RAY && c->lens_mode != AF_LENS_NONE && c->lens_mode != AF_LENS_PLANAR)
        return fail(AF_ERR_ARG, "unknown lens_mode %d", c->lens_mode);
    if (c->apod_mode != AF_APOD_FNUMBER && c->apod_mode != AF_APOD_PRINTED) return fail(AF_ERR_ARG, "unknown apod_mode %d", c->apod_mode);
    if (!(c->fnum > 0) || !is_fin(c->fnum)) return fail(AF_ERR_ARG, "fnum must be > 0");
    if (!is_fin(c->rho_thresh)) return fail(AF_ERR_ARG, "rho_thresh not finite");
    const double regs[] = {c->w1, c->kx1, c->kz1, c->w2, c->kx2, c->kz2, c->lr};
    for (double r : regs)
        if (!(r >= 0) || !is_fin(r)) return fail(AF_ERR_ARG, "regulariser weights, thresholds and lr must be finite and >= 0");
    if (!(c->beta1 >= 0 && c->beta1 < 1) || !(c->beta2 >= 0 && c->beta2 < 1) || !(c->eps > 0) || !(c->c_unit > 0) || !is_fin(c->c_unit))
        return fail(AF_ERR_ARG, "bad Adam parameters");
    if (c->optimizer != AF_OPT_ADAM && c->optimizer != AF_OPT_GD)
        return fail(AF_ERR_ARG, "unknown optimizer %d", c->optimizer);
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
        if (c->lens_mode == AF_LENS_PLANAR && !(c->elem_z[a] < c->lens_z))
            return fail(AF_ERR_ARG, "element %d not above the lens line z = %.9g", a, c->lens_z);
    }
    if (c->lens_mode == AF_LENS_PLANAR && (!(c->c_lens > 0) || !is_fin(c->c_lens) || !is_fin(c->lens_z)))
        return fail(AF_ERR_ARG, "bad lens parameters");
    if (c->lens_mode == AF_LENS_BENT_RAY) {
        if (!(c->c_lens > 0) || !is_fin(c->c_lens) || !is_fin(c->arc_cx) || !is_fin(c->arc_cz))
            return fail(AF_ERR_ARG, "bad lens parameters");
        if (!(c->lens_radius >= remax * (1 - 1e-7)))
            return fail(AF_ERR_ARG, "lens_radius %.9g below the element radius %.9g", c->lens_radius, remax);
    }
    double pmin = emin, pmax = emax;
    double xlo = 1e300, xhi = -1e300;            // flat lens: extent of the exit points
    for (int a = 0; a < c->n_elem; ++a) {
        xlo = fmin(xlo, c->elem_x[a]);
        xhi = fmax(xhi, c->elem_x[a]);
    }
    for (long long p = 0; p < npix; ++p) {
        const double x = c->pix_x[p], z = c->pix_z[p];
        if (!is_fin(x) || !is_fin(z)) return fail(AF_ERR_ARG, "pixel %lld not finite", p);
        if (!inside(x, z)) return fail(AF_ERR_ARG, "pixel %lld outside the slowness grid", p);
        if (c->lens_mode == AF_LENS_PLANAR) {
            if (!(z > c->lens_z)) return fail(AF_ERR_ARG, "pixel %lld not below the lens line", p);
            xlo = fmin(xlo, x);
            xhi = fmax(xhi, x);
        }
        if (c->lens_mode == AF_LENS_BENT_RAY) {
            if (!(hypot(x - c->arc_cx, z - c->arc_cz) > c->lens_radius))
                return fail(AF_ERR_ARG, "pixel %lld inside the lens", p);
            const double th = atan2(x - c->arc_cx, z - c->arc_cz);
            pmin = fmin(pmin, th);
            pmax = fmax(pmax, th);
        }
    }
    if (c->lens_mode == AF_LENS_PLANAR && npix > 0) {
        // every exit point lies on the lens line between its element and its pixel
        if (!inside(xlo, c->lens_z) || !inside(xhi, c->lens_z))
            return fail(AF_ERR_ARG, "lens line over [%.6g, %.6g] outside the slowness grid", xlo, xhi);
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
    b += ne * (sizeof(float4) + sizeof(float2)) + npix * (2 * sizeof(float2) + sizeof(int2));
    b += ne * npix * (sizeof(float) + sizeof(float4) + sizeof(float));   // phi, D, gdel
    b += 2 * nb * npix * sizeof(float2);                                  // B, G
    b += (size_t)c->n_patch * npair * (sizeof(float2) + 1);               // z, mask
    b += (size_t)c->n_patch * (sizeof(double) + sizeof(int));
    b += (size_t)(c->nx + 5) * (c->nz + 4) * sizeof(long long);            // ray-adjoint integer grid
    b += sizeof(AfScal) + kStatBlocks * sizeof(StatPart);
    b += 4 * (size_t)AF_MLP_NPARAM * sizeof(float) + 2 * 128 * 128 * 2 + ne * npix;   // surrogate
    b += npix * 2 * sizeof(float2) + (size_t)c->n_patch * 5 * sizeof(double) + ng * sizeof(float);   // sweep
    *bytes = b;
    return AF_OK;
}

af_status af_destroy(af_plan_t pl)
{
    if (!pl) return AF_OK;
    jobs_release(pl);
    for (int k = 0; k < 2 * kTimingCap; ++k)
        if (pl->ev[k]) cudaEventDestroy(pl->ev[k]);
    void *ptrs[] = {pl->elem, pl->elem_pol, pl->pix, pl->pix_pol, pl->phi, pl->D, pl->nrange, pl->B, pl->G, pl->z,
                    pl->mask, pl->patch_sum, pl->patch_cnt, pl->gdel, pl->gpad, pl->scal, pl->stat_part,
                    pl->mlp_p, pl->mlp_m, pl->mlp_v, pl->mlp_g, pl->mlp_w2b, pl->mlp_w3b, pl->sur_fb};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *sweep_ptrs[] = {pl->pix_base, pl->pix_pol_base, pl->sweep_geo, pl->s_sweep};
    for (void *p : sweep_ptrs)
        if (p) cudaFree(p);
    delete[] pl->host_ex;
    delete[] pl->host_ez;
    delete[] pl->host_px;
    delete[] pl->host_pz;
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
    pl->cfg = *c;
    pl->host_ex = new double[c->n_elem];
    pl->host_ez = new double[c->n_elem];
    memcpy(pl->host_ex, c->elem_x, sizeof(double) * c->n_elem);
    memcpy(pl->host_ez, c->elem_z, sizeof(double) * c->n_elem);
    pl->cfg.elem_x = pl->host_ex;
    pl->cfg.elem_z = pl->host_ez;
    {
        const size_t np = (size_t)c->n_patch * c->patch_npix;
        pl->host_px = new double[np ? np : 1];
        pl->host_pz = new double[np ? np : 1];
        if (np) {
            memcpy(pl->host_px, c->pix_x, sizeof(double) * np);
            memcpy(pl->host_pz, c->pix_z, sizeof(double) * np);
        }
    }
    pl->cfg.pix_x = pl->cfg.pix_z = nullptr;
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
    g.lens_z = (float)c->lens_z;
    g.fnum_inv2 = (float)(1.0 / (2.0 * c->fnum));
    g.fnum_half = (float)(0.5 * c->fnum);
    g.x0 = (float)c->x0;
    g.z0 = (float)c->z0;
    g.inv_dx = (float)(1.0 / c->dx);
    g.inv_dz = (float)(1.0 / c->dz);
    const bool has_lens = c->lens_mode == AF_LENS_BENT_RAY || c->lens_mode == AF_LENS_PLANAR;
    g.inv_c_lens = has_lens ? (float)(1.0 / c->c_lens) : 0.0f;
    g.fs = (float)c->fs;
    g.wd = (float)(2.0 * 3.14159265358979323846 * c->fd);
    if (has_lens) split_ff(c->fs / c->c_lens, &g.fs_clens_hi, &g.fs_clens_lo);
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
        // window holds kRayFlushRays rays; one point's contribution stays below 2^20, so
        // the merged stencil of a work item (kRayGroup points) stays below 2^22
        const double diag = sqrt(c->dx * c->dx + c->dz * c->dz);
        const double lmax = sqrt(pow((c->nx - 1) * c->dx, 2) + pow((c->nz - 1) * c->dz, 2));
        const double per_ray = 5.0 * diag + lmax / (c->nseg + 1);
        const double window = kRayFlushRays * per_ray;
        const double s1 = ldexp(1.0, 30) / window;
        const double s2 = ldexp(1.0, 20) * (c->nseg + 1) / lmax;
        g.fix_scale = (float)fmin(s1, s2);
        g.ray_flush_budget = kRayFlushBudget;
    }
    g.c_unit = (float)c->c_unit;
    g.optimizer = c->optimizer;
    g.inv_c_unit = (float)(1.0 / c->c_unit);
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

    {
        // lens-surrogate sampling region and feature scales
        double re = 0, thlo = 1e300, thhi = -1e300, zmax = 0;
        for (int a = 0; a < ne; ++a) {
            re += elem_pol[a].y / ne;
            thlo = fmin(thlo, elem_pol[a].x);
            thhi = fmax(thhi, elem_pol[a].x);
        }
        for (int p = 0; p < npix; ++p) zmax = fmax(zmax, pix_pol[p].y - re);
        const double dl = fmax(c->lens_radius - re, 1e-5);
        MlpGeom &G = pl->mlp_geom;
        G.re = re;
        G.RL = c->lens_radius;
        G.inv_c_lens = c->lens_mode == AF_LENS_BENT_RAY ? 1.0 / c->c_lens : 0.0;
        G.th_lo = thlo - 0.01;
        G.th_hi = thhi + 0.01;
        G.z_lo = dl + 1e-3;
        G.z_hi = fmax(zmax, G.z_lo + 1e-3) + 10e-3;
        G.cone = 1.05 * (c->apod_mode == AF_APOD_PRINTED ? 0.5 * c->fnum : 1.0 / (2.0 * c->fnum));
        G.c_lo = 1400.0;
        G.c_hi = 1650.0;
        MlpNorm &n = pl->mlp_norm;
        n.th_c = (float)(0.5 * (G.th_lo + G.th_hi));
        n.th_s = (float)(2.0 / (G.th_hi - G.th_lo));
        const double rlo = re + G.z_lo, rhi = re + G.z_hi * sqrt(1.0 + G.cone * G.cone);
        n.r_c = (float)(0.5 * (rlo + rhi));
        n.r_s = (float)(2.0 / (rhi - rlo));
        n.dp_s = (float)(1.0 / 0.6);
        n.c_c = 1525.0f;
        n.c_s = 1.0f / 125.0f;
        n.y0_s = (float)(2.0 * dl / c->lens_radius);
        n.y1_c = (float)(dl * G.inv_c_lens);
        n.y1_s = (float)(0.5 * dl * G.inv_c_lens);
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
    AF_ALLOC(pl->nrange, npix * sizeof(int2));
    AF_ALLOC(pl->gdel, nep * sizeof(float));
    AF_ALLOC(pl->B, nbp * sizeof(float2));
    AF_ALLOC(pl->G, nbp * sizeof(float2));
    AF_ALLOC(pl->z, nzp * sizeof(float2));
    AF_ALLOC(pl->mask, nzp);
    AF_ALLOC(pl->patch_sum, g.n_patch * sizeof(double));
    AF_ALLOC(pl->patch_cnt, g.n_patch * sizeof(int));
    AF_ALLOC(pl->scal, sizeof(AfScal));
    AF_ALLOC(pl->stat_part, kStatBlocks * sizeof(StatPart));
    pl->smem_grid = padded_grid_bytes(c);
    pl->delay = delays_shape(pl->smem_grid, pl->sm_count);
    pl->rayadj = rayadj_shape(c->nx, c->nz, g.pitch, pl->sm_count);
    AF_ALLOC(pl->gpad, (pl->smem_grid / sizeof(float)) * sizeof(long long));
    AF_ALLOC(pl->mlp_p, AF_MLP_NPARAM * sizeof(float));
    AF_ALLOC(pl->mlp_m, AF_MLP_NPARAM * sizeof(float));
    AF_ALLOC(pl->mlp_v, AF_MLP_NPARAM * sizeof(float));
    AF_ALLOC(pl->mlp_g, AF_MLP_NPARAM * sizeof(float));
    AF_ALLOC(pl->mlp_w2b, 128 * 128 * 2);
    AF_ALLOC(pl->mlp_w3b, 128 * 128 * 2);
    AF_ALLOC(pl->sur_fb, nep);
    AF_ALLOC(pl->pix_base, npix * sizeof(float2));
    AF_ALLOC(pl->pix_pol_base, npix * sizeof(float2));
    AF_ALLOC(pl->sweep_geo, (size_t)g.n_patch * 5 * sizeof(double));
    AF_ALLOC(pl->s_sweep, (size_t)g.ng * sizeof(float));
#undef AF_ALLOC
    e = mlp_setup_attributes();
    if (e != cudaSuccess) return bail(cuda_fail(e, "MLP kernel attributes"));
    e = cudaMemcpy(pl->elem, elem.data(), ne * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->elem_pol, elem_pol.data(), ne * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && npix) e = cudaMemcpy(pl->pix, pix.data(), npix * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && npix) e = cudaMemcpy(pl->pix_pol, pix_pol.data(), npix * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(pl->scal, 0, sizeof(AfScal));
    if (e == cudaSuccess) e = cudaMemset(pl->gdel, 0, (nep ? nep : 1) * sizeof(float));
    // the gradient reduce returns every cell it reads to zero, so the ray adjoint
    // always starts from a zero grid
    if (e == cudaSuccess) e = cudaMemset(pl->gpad, 0, (pl->smem_grid / sizeof(float)) * sizeof(long long));
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
    if (pl->use_surrogate)
        AF_CUDA(staged(pl, 8, [&] { return mlp_infer(pl, 0.0f, pl->sur_fb, pl->phi, nullptr); }));
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
    AF_CUDA(staged(pl, 5, [&] { return launch_das_adjoint(pl); }));
    AF_CUDA(staged(pl, 6, [&] { return launch_ray_adjoint(pl, pl->slowness, grad); }));
    pl->have_adj = true;
    return AF_OK;
}

af_status af_step(af_plan_t pl, const float *grad, float *s, float *m, float *v, int step)
{
    g_err[0] = 0;
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!grad || !s) return fail(AF_ERR_ARG, "d_grad and d_slowness must be non-NULL");
    if (pl->g.optimizer == AF_OPT_ADAM && (!m || !v)) return fail(AF_ERR_ARG, "Adam needs d_adam_m and d_adam_v");
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

af_status af_set_pixels(af_plan_t pl, const double *px, const double *pz)
{
    g_err[0] = 0;
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    af_config c = pl->cfg;
    c.pix_x = px;
    c.pix_z = pz;
    af_status st = af_check_config(&c);
    if (st != AF_OK) return st;
    const int npix = pl->g.npix;
    std::vector<float2> pix((size_t)npix), pix_pol((size_t)npix);
    for (int p = 0; p < npix; ++p) {
        pix[p] = make_float2((float)px[p], (float)pz[p]);
        const double vx = px[p] - c.arc_cx, vz = pz[p] - c.arc_cz;
        pix_pol[p] = make_float2((float)atan2(vx, vz), (float)hypot(vx, vz));
    }
    AF_CUDA(cudaStreamSynchronize(pl->stream));
    if (npix) {
        AF_CUDA(cudaMemcpy(pl->pix, pix.data(), npix * sizeof(float2), cudaMemcpyHostToDevice));
        AF_CUDA(cudaMemcpy(pl->pix_pol, pix_pol.data(), npix * sizeof(float2), cudaMemcpyHostToDevice));
        memcpy(pl->host_px, px, sizeof(double) * npix);
        memcpy(pl->host_pz, pz, sizeof(double) * npix);
    }
    pl->have_phi = false;        // exit angles of the old pixels are no warm start
    pl->have_fwd = false;
    return AF_OK;
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

af_status af_cmpe_totals(af_plan_t pl, double *d_totals)
{
    if (!pl || !d_totals) return fail(AF_ERR_ARG, "af_cmpe_totals: NULL argument");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "no forward pass yet");
    AF_CUDA(launch_cmpe_totals(pl, d_totals));
    return AF_OK;
}

af_status af_set_cmpe_totals(af_plan_t pl, const double *d_totals, float *d_loss)
{
    if (!pl || !d_totals) return fail(AF_ERR_ARG, "af_set_cmpe_totals: NULL argument");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "no forward pass yet");
    AF_CUDA(launch_cmpe_set_totals(pl, d_totals, d_loss));
    return AF_OK;
}

af_status af_get_image_grad(af_plan_t pl, float *G)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_adj) return fail(AF_ERR_STATE, "no adjoint pass yet");
    const size_t n = (size_t)pl->g.nb * pl->g.npix;
    if (n == 0) return AF_OK;
    if (!G) return fail(AF_ERR_ARG, "d_G is NULL");
    // the adjoint forms dL/dB inside the DAS adjoint without storing it: form it here
    AF_CUDA(launch_cmpe_backward(pl));
    AF_CUDA(cudaMemcpyAsync(G, pl->G, n * sizeof(float2), cudaMemcpyDeviceToDevice, pl->stream));
    return AF_OK;
}

af_status af_get_bmode(af_plan_t pl, float *bmode, float *cmpe_image)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "no forward pass yet");
    if (pl->g.npix && !bmode && !cmpe_image) return fail(AF_ERR_ARG, "both outputs are NULL");
    AF_CUDA(launch_images(pl, bmode, cmpe_image));
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

af_status af_surrogate_train(af_plan_t pl, long long n_samples, int epochs, int tiles_per_step, float lr,
                             unsigned long long seed, double *h_report)
{
    g_err[0] = 0;
    if (!pl || !h_report) return fail(AF_ERR_ARG, "NULL argument");
    if (pl->g.lens_mode != AF_LENS_BENT_RAY) return fail(AF_ERR_UNSUPPORTED, "the surrogate models the lens (bent-ray mode only)");
    if (!pl->have_fwd) return fail(AF_ERR_STATE, "run af_forward once first (validation uses its apodization)");
    if (tiles_per_step < 1 || tiles_per_step > 1024 || epochs < 1 || !(lr > 0))
        return fail(AF_ERR_ARG, "bad epochs / tiles_per_step / lr");
    const long long per_step = (long long)tiles_per_step * 128;
    if (n_samples < per_step || n_samples > (1LL << 31)) return fail(AF_ERR_ARG, "n_samples out of range");
    const long long steps_per_epoch = n_samples / per_step;
    const long long n = steps_per_epoch * per_step;
    float4 *X = nullptr;
    float2 *Y = nullptr;
    float *gpart = nullptr, *lpart = nullptr, *tphi = nullptr, *ttl = nullptr;
    unsigned long long *stats = nullptr;
    const size_t nep = (size_t)pl->g.ne * pl->g.npix;
    auto cleanup = [&]() {
        void *ptrs[] = {X, Y, gpart, lpart, tphi, ttl, stats};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    };
#define SU_CUDA(call)                                                         \
    do {                                                                      \
        cudaError_t _e = (call);                                              \
        if (_e != cudaSuccess) { cleanup(); return cuda_fail(_e, #call); }    \
    } while (0)
    SU_CUDA(cudaMalloc(&X, n * sizeof(float4)));
    SU_CUDA(cudaMalloc(&Y, n * sizeof(float2)));
    SU_CUDA(cudaMalloc(&gpart, (size_t)tiles_per_step * AF_MLP_NPARAM * sizeof(float)));
    SU_CUDA(cudaMalloc(&lpart, tiles_per_step * sizeof(float)));
    SU_CUDA(cudaMalloc(&tphi, (nep ? nep : 1) * sizeof(float)));
    SU_CUDA(cudaMalloc(&ttl, (nep ? nep : 1) * sizeof(float)));
    SU_CUDA(cudaMalloc(&stats, 8 * sizeof(unsigned long long)));
    SU_CUDA(cudaMemsetAsync(&pl->scal->mlp_err, 0, sizeof(int), pl->stream));
    SU_CUDA(mlp_init_params(pl, seed));
    SU_CUDA(mlp_generate(pl, n, seed * 2654435761ull + 1, X, Y));
    const long long total_steps = steps_per_epoch * epochs;
    std::vector<float> hl(tiles_per_step);
    double last_loss = 0.0;
    long long step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (long long st = 0; st < steps_per_epoch; ++st, ++step) {
            // cosine decay to lr / 20
            const double frac = (double)step / (double)total_steps;
            const float lr_t = (float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + cos(3.14159265358979323846 * frac))));
            SU_CUDA(mlp_train_step(pl, X, Y, st * per_step, tiles_per_step, lr_t, (int)(step + 1), lpart, gpart));
        }
        SU_CUDA(cudaMemcpyAsync(hl.data(), lpart, tiles_per_step * sizeof(float), cudaMemcpyDeviceToHost, pl->stream));
        SU_CUDA(cudaStreamSynchronize(pl->stream));
        last_loss = 0.0;
        for (float v : hl) last_loss += v;
    }
    // validation on this plan's apodized pairs at several medium speeds
    const double tol = 1.0 / (50.0 * (double)pl->g.wd / (2.0 * 3.14159265358979323846));   // lambda / 50 in time
    SU_CUDA(cudaMemsetAsync(pl->sur_fb, 0, nep ? nep : 1, pl->stream));
    SU_CUDA(cudaMemsetAsync(stats, 0, 8 * sizeof(unsigned long long), pl->stream));
    const double speeds[] = {1400.0, 1450.0, 1500.0, 1550.0, 1600.0, 1650.0};
    for (double cv : speeds) {
        SU_CUDA(mlp_infer(pl, (float)cv, nullptr, tphi, ttl));
        SU_CUDA(mlp_validate(pl, cv, tphi, ttl, tol, pl->sur_fb, stats));
    }
    unsigned long long hs[8];
    long long nfb = 0;
    {
        std::vector<uint8_t> hfb(nep);
        SU_CUDA(cudaMemcpyAsync(hs, stats, sizeof hs, cudaMemcpyDeviceToHost, pl->stream));
        if (nep) SU_CUDA(cudaMemcpyAsync(hfb.data(), pl->sur_fb, nep, cudaMemcpyDeviceToHost, pl->stream));
        SU_CUDA(cudaStreamSynchronize(pl->stream));
        for (uint8_t v : hfb) nfb += v;
    }
    int merr = 0;
    SU_CUDA(cudaMemcpy(&merr, &pl->scal->mlp_err, sizeof(int), cudaMemcpyDeviceToHost));
    cleanup();
#undef SU_CUDA
    if (merr) return fail(AF_ERR_TIMEOUT, "a tensor-core completion wait timed out");
    const double count = hs[0] > 0 ? (double)hs[0] : 1.0;
    h_report[0] = last_loss;
    h_report[1] = sqrt((double)hs[4] * 1e-12 / count);      // rms exit-angle error (rad)
    h_report[2] = (double)hs[2] * 1e-12;                    // max delay error (s)
    h_report[3] = (double)hs[3] * 1e-12;                    // max lens-time error (s)
    h_report[4] = (double)nfb / (double)(hs[0] / 6 > 0 ? hs[0] / 6 : 1);   // fallback fraction of apodized pairs
    h_report[5] = (double)n;
    h_report[6] = tol;
    h_report[7] = (double)total_steps;
    pl->sur_trained = true;
    return AF_OK;
}

af_status af_surrogate_enable(af_plan_t pl, int enable)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (enable && !pl->sur_trained) return fail(AF_ERR_STATE, "surrogate not trained");
    pl->use_surrogate = enable != 0;
    return AF_OK;
}

af_status af_surrogate_eval(af_plan_t pl, float c, float *d_phi, float *d_tlens)
{
    if (!pl || !d_phi || !d_tlens) return fail(AF_ERR_ARG, "NULL argument");
    if (!(c > 0)) return fail(AF_ERR_ARG, "c must be > 0");
    AF_CUDA(mlp_infer(pl, c, nullptr, d_phi, d_tlens));
    return AF_OK;
}

af_status af_surrogate_params(af_plan_t pl, float *d_params, int set)
{
    if (!pl || !d_params) return fail(AF_ERR_ARG, "NULL argument");
    if (set) {
        AF_CUDA(cudaMemcpyAsync(pl->mlp_p, d_params, AF_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, pl->stream));
        AF_CUDA(mlp_refresh_bf16(pl));
    } else {
        AF_CUDA(cudaMemcpyAsync(d_params, pl->mlp_p, AF_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, pl->stream));
    }
    return AF_OK;
}

af_status af_surrogate_grad(af_plan_t pl, const float *d_X, const float *d_Y, int n, float *d_grad, float *h_loss)
{
    if (!pl || !d_X || !d_Y || !d_grad || !h_loss) return fail(AF_ERR_ARG, "NULL argument");
    if (n <= 0 || n % 128 || n / 128 > 1024) return fail(AF_ERR_SHAPE, "n must be a positive multiple of 128 (<= 131072)");
    const int tiles = n / 128;
    float *gpart = nullptr, *lpart = nullptr;
    AF_CUDA(cudaMalloc(&gpart, (size_t)tiles * AF_MLP_NPARAM * sizeof(float)));
    cudaError_t e = cudaMalloc(&lpart, tiles * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(&pl->scal->mlp_err, 0, sizeof(int), pl->stream);
    if (e == cudaSuccess)
        e = mlp_train_step(pl, reinterpret_cast<const float4 *>(d_X), reinterpret_cast<const float2 *>(d_Y), 0, tiles,
                           0.0f, 1, lpart, gpart);
    std::vector<float> hl(tiles);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_grad, pl->mlp_g, AF_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, pl->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hl.data(), lpart, tiles * sizeof(float), cudaMemcpyDeviceToHost, pl->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
    int merr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&merr, &pl->scal->mlp_err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(gpart);
    cudaFree(lpart);
    if (e != cudaSuccess) return cuda_fail(e, "af_surrogate_grad");
    if (merr) return fail(AF_ERR_TIMEOUT, "a tensor-core completion wait timed out");
    double l = 0.0;
    for (float v : hl) l += v;
    *h_loss = (float)l;
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

af_status af_set_ray_flush_budget(af_plan_t pl, double rays)
{
    if (!pl) return fail(AF_ERR_ARG, "plan is NULL");
    if (!(rays >= 0.0)) return fail(AF_ERR_ARG, "rays must be >= 0");
    pl->g.ray_flush_budget = rays < (double)kRayFlushBudget ? (float)rays : kRayFlushBudget;
    return AF_OK;
}

af_status af_set_wait_limit(int tries)
{
    g_wait_tries.store(tries >= 0 ? (uint32_t)tries : tc::kWaitTries, std::memory_order_relaxed);
    return AF_OK;
}

}  // extern "C"
