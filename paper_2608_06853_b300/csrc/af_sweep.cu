// Global-speed sweep (Sec. II-C, Sec. III-A; Fig. 3): L_CMPE of uniform maps
// at a list of speeds, one forward pass each, with no host round trip between
// speeds.
//
// Dynamic grid: at speed c0 every patch keeps its direction from the
// reference surface's centre, its depth below that surface scales by
// k = c0 / c_ref, and its pixels' offsets from the patch centre scale by k, so
// that each patch's pixels and kernel spacing follow the echoes they observe
// (time of flight fixed: apparent depth proportional to c0).  The reference
// surface is the lens surface: the arc of radius lens_radius about
// (arc_cx, arc_cz), or the line z = lens_z for a flat lens.  The patch centre
// is the mean of the patch's pixels.
//
// The moved pixels are computed in float64 on the host (validation) and on the
// device (the pixels used), by the same operations in the same order, then
// rounded to float.
#include <math.h>

#include <vector>

#include "af_internal.cuh"

void sweep_patch_geometry(const af_config *c, const double *px, const double *pz, double *geo)
{
    const int n = c->patch_npix;
    for (int P = 0; P < c->n_patch; ++P) {
        double sx = 0.0, sz = 0.0;
        for (int q = 0; q < n; ++q) {
            sx += px[(size_t)P * n + q];
            sz += pz[(size_t)P * n + q];
        }
        const double ccx = sx / n, ccz = sz / n;
        double ux, uz, d;
        if (c->lens_mode == AF_LENS_PLANAR) {
            ux = 0.0;
            uz = 1.0;
            d = ccz - c->lens_z;                       // depth below the lens line
        } else {
            const double vx = ccx - c->arc_cx, vz = ccz - c->arc_cz;
            const double rho = sqrt(vx * vx + vz * vz);
            ux = vx / rho;
            uz = vz / rho;
            d = rho - c->lens_radius;                  // depth below the lens arc
        }
        double *gp = geo + (size_t)P * 5;
        gp[0] = ccx;
        gp[1] = ccz;
        gp[2] = ux;
        gp[3] = uz;
        gp[4] = d;
    }
}

// moved position of one pixel (float64), the same expression on host and device
__host__ __device__ __forceinline__ void moved_pixel(double ccx, double ccz, double ux, double uz, double d,
                                                     double sx, double sz, double k, double &x, double &z)
{
    const double dk = d * k;
    // new centre = foot of the old centre on the reference surface + scaled depth
    const double ncx = (ccx - d * ux) + dk * ux, ncz = (ccz - d * uz) + dk * uz;
    x = ncx + k * (sx - ccx);
    z = ncz + k * (sz - ccz);
}

void sweep_moved_pixels(const af_config *c, const double *px, const double *pz, const double *geo, double k,
                        double *out_x, double *out_z)
{
    const int n = c->patch_npix;
    for (int P = 0; P < c->n_patch; ++P) {
        const double *gp = geo + (size_t)P * 5;
        for (int q = 0; q < n; ++q) {
            const size_t p = (size_t)P * n + q;
            double x, z;
            moved_pixel(gp[0], gp[1], gp[2], gp[3], gp[4], px[p], pz[p], k, x, z);
            out_x[p] = (double)(float)x;
            out_z[p] = (double)(float)z;
        }
    }
}

namespace {

__global__ void sweep_pixels_kernel(int npix, int patch_npix, double arc_cx, double arc_cz, double k,
                                    const float2 *__restrict__ base, const double *__restrict__ geo,
                                    float2 *__restrict__ pix, float2 *__restrict__ pix_pol)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const double *gp = geo + (size_t)(p / patch_npix) * 5;
    double x, z;
    moved_pixel(gp[0], gp[1], gp[2], gp[3], gp[4], (double)base[p].x, (double)base[p].y, k, x, z);
    const float2 q = make_float2((float)x, (float)z);
    pix[p] = q;
    const double vx = (double)q.x - arc_cx, vz = (double)q.y - arc_cz;
    pix_pol[p] = make_float2((float)atan2(vx, vz), (float)hypot(vx, vz));
}

__global__ void fill_kernel(float *__restrict__ s, int n, float v)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) s[k] = v;
}

__global__ void sweep_record_kernel(const AfScal *__restrict__ scal, float *__restrict__ cmpe,
                                    int *__restrict__ active)
{
    *cmpe = scal->lcmpe;
    if (active) *active = scal->n_active;
}

}  // namespace

extern "C" af_status af_sweep(af_plan_t pl, const void *d_iq, const float *d_iq_scale, const double *h_speeds,
                              int n_speeds, double c_ref, int dynamic, float *d_cmpe, int *d_active)
{
    if (!pl || !d_iq || !h_speeds || !d_cmpe) return af_set_error(AF_ERR_ARG, "af_sweep: NULL argument");
    if (n_speeds < 1 || !(c_ref > 0) || !isfinite(c_ref)) return af_set_error(AF_ERR_ARG, "af_sweep: bad n_speeds / c_ref");
    if (pl->iq_dtype != AF_IQ_C64 && !d_iq_scale) return af_set_error(AF_ERR_DTYPE, "16-bit channel data needs d_iq_scale");
    for (int k = 0; k < n_speeds; ++k)
        if (!(h_speeds[k] > 0) || !isfinite(h_speeds[k])) return af_set_error(AF_ERR_ARG, "af_sweep: bad speed %d", k);
    const af_config &c = pl->cfg;
    const int npix = pl->g.npix;
    const bool dyn = dynamic != 0 && npix > 0;
    if (dyn && c.lens_mode != AF_LENS_PLANAR && !(c.lens_radius > 0))
        return af_set_error(AF_ERR_ARG, "af_sweep: the dynamic grid needs a lens surface (lens_radius > 0)");
    std::vector<double> geo(dyn ? (size_t)c.n_patch * 5 : 1), mx(dyn ? npix : 1), mz(dyn ? npix : 1);
    // every moved pixel set must pass the plan's validation (grid box, lens)
    auto validate = [&](int k) -> af_status {
        sweep_moved_pixels(&c, pl->host_px, pl->host_pz, geo.data(), h_speeds[k] / c_ref, mx.data(), mz.data());
        af_config m = c;
        m.pix_x = mx.data();
        m.pix_z = mz.data();
        return af_check_config(&m);
    };
    if (dyn) {
        sweep_patch_geometry(&c, pl->host_px, pl->host_pz, geo.data());
        // the extreme speeds first, so that a sweep leaving the grid box fails before any work
        af_status v = validate(0);
        if (v == AF_OK && n_speeds > 1) v = validate(n_speeds - 1);
        if (v != AF_OK) return v;
    }
    cudaStream_t st = pl->stream;
#define SW_CUDA(call)                                                                                    \
    do {                                                                                                 \
        const cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_sweep: %s", cudaGetErrorString(e_)); \
    } while (0)
    if (dyn) {
        SW_CUDA(cudaMemcpyAsync(pl->pix_base, pl->pix, npix * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        SW_CUDA(cudaMemcpyAsync(pl->pix_pol_base, pl->pix_pol, npix * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        // synchronous copy: the host vector is released at return
        SW_CUDA(cudaStreamSynchronize(st));
        SW_CUDA(cudaMemcpy(pl->sweep_geo, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    pl->iq = d_iq;
    pl->iq_scale = d_iq_scale;
    pl->slowness = pl->s_sweep;
    const int ng = pl->g.ng;
    for (int k = 0; k < n_speeds; ++k) {
        // the speeds in between are validated while the device runs the earlier ones
        if (dyn && k > 0 && k < n_speeds - 1) {
            const af_status v = validate(k);
            if (v != AF_OK) {
                // put the plan's pixels back before reporting
                cudaMemcpyAsync(pl->pix, pl->pix_base, npix * sizeof(float2), cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(pl->pix_pol, pl->pix_pol_base, npix * sizeof(float2), cudaMemcpyDeviceToDevice, st);
                pl->have_phi = false;
                pl->have_fwd = pl->have_adj = false;
                return v;
            }
        }
        if (dyn) {
            sweep_pixels_kernel<<<(npix + 255) / 256, 256, 0, st>>>(npix, c.patch_npix, c.arc_cx, c.arc_cz,
                                                                    h_speeds[k] / c_ref, pl->pix_base,
                                                                    pl->sweep_geo, pl->pix, pl->pix_pol);
            SW_CUDA(cudaGetLastError());
            // the previous speed's exit angles start the (bracketed) exit solve: the
            // pixels moved little, and any start inside the bracket converges
            pl->have_phi = pl->have_phi && k > 0;
        }
        fill_kernel<<<(ng + 255) / 256, 256, 0, st>>>(pl->s_sweep, ng, (float)(1.0 / h_speeds[k]));
        SW_CUDA(cudaGetLastError());
        SW_CUDA(launch_grid_stats(pl, pl->s_sweep));
        if (pl->use_surrogate) SW_CUDA(mlp_infer(pl, 0.0f, pl->sur_fb, pl->phi, nullptr));
        SW_CUDA(launch_delays(pl, pl->s_sweep));
        SW_CUDA(launch_das_forward(pl));
        SW_CUDA(launch_cmpe_forward(pl, nullptr));
        sweep_record_kernel<<<1, 1, 0, st>>>(pl->scal, d_cmpe + k, d_active ? d_active + k : nullptr);
        SW_CUDA(cudaGetLastError());
    }
    if (dyn) {
        SW_CUDA(cudaMemcpyAsync(pl->pix, pl->pix_base, npix * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        SW_CUDA(cudaMemcpyAsync(pl->pix_pol, pl->pix_pol_base, npix * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        pl->have_phi = false;
    }
    pl->have_fwd = false;                        // the last pass was of the sweep's map
    pl->have_adj = false;
#undef SW_CUDA
    return af_set_error(AF_OK, "");
}
