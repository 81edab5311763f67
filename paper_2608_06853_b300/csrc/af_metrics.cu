// Image-quality metrics of one forward pass (Sec. III-F, Model Evaluation) and
// the sound-speed MAE.  Definitions (the paper gives MAE and cites the rest):
//  - receive images S_j(p) = sum_i B_ij(p); coherence factor over receive
//    subapertures CF(p) = |sum_j S_j|^2 / (n_sub sum_j |S_j|^2);
//  - lag-one coherence over a region: mean over j of
//    Re sum_p S_j conj(S_{j+1}) / sqrt(sum_p |S_j|^2 sum_p |S_{j+1}|^2);
//  - common-midpoint correlation: mean over patches and common-midpoint pairs of
//    the CMPE correlation coefficient rho;
//  - contrast (dB), CNR and generalized CNR of the envelope |sum_ij B_ij| between
//    a target region (roi 1) and a background region (roi 2);
//  - MAE: mean over the pixels of |1 / bicubic(s) - c_true|.
// Sums are formed in double in a fixed order (one CTA per column), histogram
// counts with integer atomics, so the results do not depend on scheduling.
#include <math.h>
#include <string.h>

#include <vector>

#include "af_internal.cuh"

namespace {

// columns of the per-pixel table (each times its region indicator)
enum { kColCf = 0, kColBg, kColEnvIn, kColEnv2In, kColIn, kColEnvBg, kColEnv2Bg, kColLag0 };
// lag-one products follow at kColLag0 + j (j < nsub - 1), channel energies at
// kColLag0 + (nsub - 1) + j (j < nsub)
__host__ __device__ inline int metric_columns(int nsub) { return kColLag0 + (nsub - 1) + nsub; }

__global__ void __launch_bounds__(256) metrics_pixel_kernel(AfGeom g, const float2 *__restrict__ B,
                                                            const uint8_t *__restrict__ roi,
                                                            float *__restrict__ cols, float *__restrict__ env)
{
    const int n = g.nsub;
    const long np = g.npix;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long)gridDim.x * blockDim.x) {
        const int r = roi[p];
        const float bg = r == 2 ? 1.0f : 0.0f, in = r == 1 ? 1.0f : 0.0f;
        float tr = 0.f, ti = 0.f, energy = 0.f, pr = 0.f, pi = 0.f;
        for (int j = 0; j < n; ++j) {
            float sr = 0.f, si = 0.f;
            for (int i = 0; i < n; ++i) {
                const float2 v = B[(long)(i * n + j) * np + p];
                sr += v.x;
                si += v.y;
            }
            const float e = sr * sr + si * si;
            if (j > 0) cols[(long)(kColLag0 + j - 1) * np + p] = bg * (pr * sr + pi * si);   // Re S_{j-1} conj S_j
            cols[(long)(kColLag0 + (n - 1) + j) * np + p] = bg * e;
            tr += sr;
            ti += si;
            energy += e;
            pr = sr;
            pi = si;
        }
        const float t2 = tr * tr + ti * ti, a = sqrtf(t2);
        const float cf = energy > 0.0f ? t2 / (n * energy) : 0.0f;
        env[p] = a;
        cols[(long)kColCf * np + p] = bg * cf;
        cols[(long)kColBg * np + p] = bg;
        cols[(long)kColEnvIn * np + p] = in * a;
        cols[(long)kColEnv2In * np + p] = in * a * a;
        cols[(long)kColIn * np + p] = in;
        cols[(long)kColEnvBg * np + p] = bg * a;
        cols[(long)kColEnv2Bg * np + p] = bg * a * a;
    }
}

// out[c] = sum_p cols[c][p] in double, fixed order: one CTA per column
__global__ void __launch_bounds__(256) column_sum_kernel(const float *__restrict__ cols, long np,
                                                         double *__restrict__ out)
{
    __shared__ double red[256];
    const float *col = cols + (long)blockIdx.x * np;
    double acc = 0.0;
    for (long p = threadIdx.x; p < np; p += 256) acc += (double)col[p];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// min / max of the envelope over the two regions (one CTA)
__global__ void __launch_bounds__(256) env_range_kernel(const float *__restrict__ env,
                                                        const uint8_t *__restrict__ roi, long np,
                                                        float *__restrict__ range)
{
    __shared__ float lo[256], hi[256];
    float a = INFINITY, b = -INFINITY;
    for (long p = threadIdx.x; p < np; p += 256)
        if (roi[p] == 1 || roi[p] == 2) {
            a = fminf(a, env[p]);
            b = fmaxf(b, env[p]);
        }
    lo[threadIdx.x] = a;
    hi[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            lo[threadIdx.x] = fminf(lo[threadIdx.x], lo[threadIdx.x + o]);
            hi[threadIdx.x] = fmaxf(hi[threadIdx.x], hi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        range[0] = lo[0];
        range[1] = hi[0];
    }
}

// hist[r - 1][b] += 1 for every pixel of region r in {1, 2}, b its envelope bin
__global__ void __launch_bounds__(256) env_hist_kernel(const float *__restrict__ env,
                                                       const uint8_t *__restrict__ roi, long np,
                                                       const float *__restrict__ range, int nbins,
                                                       int *__restrict__ hist)
{
    const float lo = range[0], span = range[1] > range[0] ? range[1] - range[0] : 1.0f;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long)gridDim.x * blockDim.x) {
        const int r = roi[p];
        if (r != 1 && r != 2) continue;
        const int b = min((int)((env[p] - lo) / span * (float)nbins), nbins - 1);
        atomicAdd(&hist[(r - 1) * nbins + b], 1);
    }
}

// per patch: sum over common-midpoint pairs of rho (one CTA per patch, warp per pair)
__global__ void __launch_bounds__(256) patch_rho_kernel(AfGeom g, const float2 *__restrict__ B,
                                                        double *__restrict__ patch_rho)
{
    __shared__ double s_sum[8];
    const int P = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31, n = g.nsub;
    const int base = P * g.patch_npix;
    double lsum = 0.0;
    for (int k = w; k < g.npair; k += 8) {
        const int i = k / (n - 2), jj = k - i * (n - 2);
        const int j = jj < i ? jj + 1 : jj + 2;
        const float2 *B1 = B + (long)(i * n + j) * g.npix + base;
        const float2 *B2 = B + (long)((i + 1) * n + (j - 1)) * g.npix + base;
        float zr = 0.f, zi = 0.f, e1 = 0.f, e2 = 0.f;
        for (int q = lane; q < g.patch_npix; q += 32) {
            const float2 a = B1[q], c = B2[q];
            zr = fmaf(a.x, c.x, fmaf(a.y, c.y, zr));
            zi = fmaf(a.y, c.x, fmaf(-a.x, c.y, zi));
            e1 = fmaf(a.x, a.x, fmaf(a.y, a.y, e1));
            e2 = fmaf(c.x, c.x, fmaf(c.y, c.y, e2));
        }
        for (int o = 16; o > 0; o >>= 1) {
            zr += __shfl_xor_sync(0xffffffffu, zr, o);
            zi += __shfl_xor_sync(0xffffffffu, zi, o);
            e1 += __shfl_xor_sync(0xffffffffu, e1, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        }
        if (lane == 0) {
            const float den = sqrtf(e1) * sqrtf(e2);
            lsum += den > 0.0f ? (double)(hypotf(zr, zi) / den) : 0.0;
        }
    }
    if (lane == 0) s_sum[w] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < 8; ++k) a += s_sum[k];
        patch_rho[P] = a;
    }
}

// |1 / bicubic(s, r_p) - c_true[p]| (Keys a = -1/2, clamp to edge), one column
__global__ void __launch_bounds__(256) speed_err_kernel(AfGeom g, const float *__restrict__ s,
                                                        const float2 *__restrict__ pix,
                                                        const float *__restrict__ c_true,
                                                        float *__restrict__ err)
{
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < g.npix; p += (long)gridDim.x * blockDim.x) {
        const float2 r = pix[p];
        const float gx = (r.x - g.x0) * g.inv_dx, gz = (r.y - g.z0) * g.inv_dz;
        const float fx = floorf(gx), fz = floorf(gz);
        const int i0 = (int)fx, j0 = (int)fz;
        float wx[4], wz[4];
        keys_weights(gx - fx, wx);
        keys_weights(gz - fz, wz);
        float v = 0.0f;
        for (int b = 0; b < 4; ++b) {
            const int j = min(max(j0 - 1 + b, 0), g.nz - 1);
            float h = 0.0f;
            for (int a = 0; a < 4; ++a) h = fmaf(wx[a], s[j * g.nx + min(max(i0 - 1 + a, 0), g.nx - 1)], h);
            v = fmaf(wz[b], h, v);
        }
        err[p] = fabsf(1.0f / v - c_true[p]);
    }
}

}  // namespace

namespace {

// device scratch owned by one call of the metric entry points
struct DevScratch {
    void *p = nullptr;
    ~DevScratch()
    {
        if (p) cudaFree(p);
    }
};

af_status cuda_fail(const char *what, cudaError_t e)
{
    return af_set_error(AF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

#define MT_CHECK(call)                                         \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(#call, e_);    \
    } while (0)

extern "C" af_status af_image_metrics(af_plan_t pl, const uint8_t *d_roi, int nbins, af_metrics *out)
{
    if (!pl || !d_roi || !out) return af_set_error(AF_ERR_ARG, "af_image_metrics: NULL argument");
    if (nbins < 2 || nbins > 65536)
        return af_set_error(AF_ERR_ARG, "af_image_metrics: nbins %d outside [2, 65536]", nbins);
    if (!pl->have_fwd) return af_set_error(AF_ERR_STATE, "af_image_metrics: no forward pass yet");
    const AfGeom &g = pl->g;
    const long np = g.npix;
    const int C = metric_columns(g.nsub);
    memset(out, 0, sizeof(*out));
    if (np == 0) return af_set_error(AF_OK, "");
    cudaStream_t st = pl->stream;
    DevScratch cols, env, sums, range, hist, prho;
    MT_CHECK(cudaMalloc(&cols.p, (size_t)C * np * sizeof(float)));
    MT_CHECK(cudaMalloc(&env.p, (size_t)np * sizeof(float)));
    MT_CHECK(cudaMalloc(&sums.p, (size_t)C * sizeof(double)));
    MT_CHECK(cudaMalloc(&range.p, 2 * sizeof(float)));
    MT_CHECK(cudaMalloc(&hist.p, (size_t)2 * nbins * sizeof(int)));
    MT_CHECK(cudaMalloc(&prho.p, (size_t)(g.n_patch > 0 ? g.n_patch : 1) * sizeof(double)));
    MT_CHECK(cudaMemsetAsync(hist.p, 0, (size_t)2 * nbins * sizeof(int), st));
    const int blocks = (int)((np + 255) / 256 < 4096 ? (np + 255) / 256 : 4096);
    metrics_pixel_kernel<<<blocks, 256, 0, st>>>(g, pl->B, d_roi, (float *)cols.p, (float *)env.p);
    MT_CHECK(cudaGetLastError());
    column_sum_kernel<<<C, 256, 0, st>>>((const float *)cols.p, np, (double *)sums.p);
    MT_CHECK(cudaGetLastError());
    env_range_kernel<<<1, 256, 0, st>>>((const float *)env.p, d_roi, np, (float *)range.p);
    MT_CHECK(cudaGetLastError());
    env_hist_kernel<<<blocks, 256, 0, st>>>((const float *)env.p, d_roi, np, (const float *)range.p, nbins,
                                            (int *)hist.p);
    MT_CHECK(cudaGetLastError());
    if (g.n_patch > 0 && g.npair > 0) {
        patch_rho_kernel<<<g.n_patch, 256, 0, st>>>(g, pl->B, (double *)prho.p);
        MT_CHECK(cudaGetLastError());
    }
    std::vector<double> h_sums(C), h_prho(g.n_patch > 0 ? g.n_patch : 1, 0.0);
    std::vector<int> h_hist(2 * (size_t)nbins);
    MT_CHECK(cudaMemcpyAsync(h_sums.data(), sums.p, C * sizeof(double), cudaMemcpyDeviceToHost, st));
    MT_CHECK(cudaMemcpyAsync(h_hist.data(), hist.p, 2 * (size_t)nbins * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (g.n_patch > 0 && g.npair > 0)
        MT_CHECK(cudaMemcpyAsync(h_prho.data(), prho.p, g.n_patch * sizeof(double), cudaMemcpyDeviceToHost, st));
    MT_CHECK(cudaStreamSynchronize(st));

    const int n = g.nsub;
    const double n_bg = h_sums[kColBg], n_in = h_sums[kColIn];
    out->n_in = (long long)llround(n_in);
    out->n_out = (long long)llround(n_bg);
    out->cf_mean = n_bg > 0 ? h_sums[kColCf] / n_bg : NAN;
    double loc = 0.0;
    for (int j = 0; j + 1 < n; ++j) {
        const double e1 = h_sums[kColLag0 + (n - 1) + j], e2 = h_sums[kColLag0 + (n - 1) + j + 1];
        loc += e1 > 0 && e2 > 0 ? h_sums[kColLag0 + j] / sqrt(e1 * e2) : 0.0;
    }
    out->loc = n > 1 ? loc / (n - 1) : 0.0;
    double rho = 0.0;
    for (int P = 0; P < g.n_patch && g.npair > 0; ++P) rho += h_prho[P];
    out->cmcc = g.n_patch > 0 && g.npair > 0 ? rho / ((double)g.n_patch * g.npair) : 0.0;
    if (n_in > 0 && n_bg > 0) {
        const double mi = h_sums[kColEnvIn] / n_in, mo = h_sums[kColEnvBg] / n_bg;
        const double vi = fmax(h_sums[kColEnv2In] / n_in - mi * mi, 0.0);
        const double vo = fmax(h_sums[kColEnv2Bg] / n_bg - mo * mo, 0.0);
        out->mean_in = mi;
        out->mean_out = mo;
        out->contrast_db = 20.0 * log10(mi / mo);
        out->cnr = fabs(mi - mo) / sqrt(vi + vo);
        double overlap = 0.0;
        for (int b = 0; b < nbins; ++b) overlap += fmin(h_hist[b] / n_in, h_hist[nbins + b] / n_bg);
        out->gcnr = 1.0 - overlap;
    } else {
        out->mean_in = out->mean_out = out->contrast_db = out->cnr = out->gcnr = NAN;
    }
    return af_set_error(AF_OK, "");
}

extern "C" af_status af_speed_mae(af_plan_t pl, const float *d_s, const float *d_c_true, double *h_mae)
{
    if (!pl || !d_s || !d_c_true || !h_mae) return af_set_error(AF_ERR_ARG, "af_speed_mae: NULL argument");
    const AfGeom &g = pl->g;
    const long np = g.npix;
    *h_mae = 0.0;
    if (np == 0) return af_set_error(AF_OK, "");
    cudaStream_t st = pl->stream;
    DevScratch err, sum;
    MT_CHECK(cudaMalloc(&err.p, (size_t)np * sizeof(float)));
    MT_CHECK(cudaMalloc(&sum.p, sizeof(double)));
    const int blocks = (int)((np + 255) / 256 < 4096 ? (np + 255) / 256 : 4096);
    speed_err_kernel<<<blocks, 256, 0, st>>>(g, d_s, pl->pix, d_c_true, (float *)err.p);
    MT_CHECK(cudaGetLastError());
    column_sum_kernel<<<1, 256, 0, st>>>((const float *)err.p, np, (double *)sum.p);
    MT_CHECK(cudaGetLastError());
    double h = 0.0;
    MT_CHECK(cudaMemcpyAsync(&h, sum.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    MT_CHECK(cudaStreamSynchronize(st));
    *h_mae = h / (double)np;
    return af_set_error(AF_OK, "");
}
