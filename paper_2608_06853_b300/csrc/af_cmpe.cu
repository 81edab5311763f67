// Common-midpoint phase error (Sec. II-D; the focusing loss of Simson et al.
// that the paper keeps unchanged).  Reading used by this library: per patch
// and per pair of common-midpoint subaperture images (i, j) ~ (i+1, j-1),
// with the reciprocal pair j = i + 1 skipped,
//   z   = sum_p B_ij(p) conj(B_i+1,j-1(p)),
//   rho = |z| / sqrt(sum |B_ij|^2 sum |B_i+1,j-1|^2),  m = [rho >= rho_thresh],
//   L_CMPE = sum m |arg z| / max(1, sum m),
// with m held constant in the adjoint.  Total loss of Eq. 12 adds w1 R_TV +
// w2 R_SV from the grid-statistics kernel.
#include <math.h>

#include "af_cmpe.cuh"
#include "af_internal.cuh"

namespace {

using cmpe::pair_ij;
// index of the pair whose first image is (i, j), or -1
using cmpe::pair_index;

// one CTA of kCmpeWarps warps per patch; warp w takes the kPairsPerWarp pairs from
// w kPairsPerWarp on, then those kCmpeWarps kPairsPerWarp further, ...
// (16 warps per patch: 29.5 us, 32: 44.8 us, 8: 37.2 us on the 128-element
// workload, where 16-warp CTAs of all 400 patches are resident at once)
constexpr int kCmpeWarps = 16;

// fixed-order sums over patches (256 strided partial sums, then a halving tree);
// loss = {L, L_CMPE, R_TV, R_SV}.  Called by every thread of a block of at least
// 256 threads; the partials are read from L2, where other CTAs wrote them.
__device__ void cmpe_fold(const AfGeom &g, const double *patch_sum, const int *patch_cnt, AfScal *scal,
                          float *loss)
{
    __shared__ double s_a[256];
    __shared__ int s_c[256];
    const int t = threadIdx.x;
    if (t < 256) {
        double a = 0.0;
        int c = 0;
        for (int P = t; P < g.n_patch; P += 256) { a += __ldcg(patch_sum + P); c += __ldcg(patch_cnt + P); }
        s_a[t] = a;
        s_c[t] = c;
    }
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) { s_a[t] += s_a[t + o]; s_c[t] += s_c[t + o]; }
        __syncthreads();
    }
    if (t == 0) {
        const int M = s_c[0];
        const double lc = s_a[0] / (M > 1 ? M : 1);
        scal->cmpe_sum = s_a[0];
        scal->lcmpe = (float)lc;
        scal->n_active = M;
        scal->inv_m = (float)(1.0 / (M > 1 ? M : 1));
        scal->cmpe_done = 0;
        scal->gmax_bits = 0;           // max|dL/dT|, taken by the next DAS adjoint
        if (loss) {
            loss[0] = (float)(lc + (double)g.w1 * scal->rtv + (double)g.w2 * scal->rsv);
            loss[1] = (float)lc;
            loss[2] = scal->rtv;
            loss[3] = scal->rsv;
        }
    }
}

// The CTA that finishes last (counted in scal->cmpe_done, which it sets back to
// zero) folds all patches' sums, so the loss needs no second launch.
__global__ void __launch_bounds__(32 * kCmpeWarps) cmpe_forward_kernel(AfGeom g, const float2 *__restrict__ B,
                                                           float2 *__restrict__ z,
                                                           uint8_t *__restrict__ mask,
                                                           double *__restrict__ patch_sum,
                                                           int *__restrict__ patch_cnt, AfScal *scal,
                                                           float *__restrict__ loss)
{
    __shared__ double s_sum[kCmpeWarps];
    __shared__ int s_cnt[kCmpeWarps];
    __shared__ int s_last;
    pdl_wait();
    const int P = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int base = P * g.patch_npix;
    double lsum = 0.0;
    int cnt = 0;
    const int slot = lane / cmpe::kPairLanes, sub = lane % cmpe::kPairLanes;
    for (int k0 = w * cmpe::kPairsPerWarp; k0 < g.npair; k0 += kCmpeWarps * cmpe::kPairsPerWarp) {
        const int k = k0 + slot;
        const cmpe::PairTerms t = cmpe::pair_terms(B, g.nsub, g.npix, base, g.patch_npix, k, sub, k < g.npair);
        if (sub == 0 && k < g.npair) {
            const int m = t.rho >= g.rho_thresh;
            const long o = (long)P * g.npair + k;
            z[o] = make_float2(t.zr, t.zi);
            mask[o] = (uint8_t)m;
            if (m) {
                lsum += (double)fabsf(atan2f(t.zi, t.zr));
                ++cnt;
            }
        }
    }
    lsum = cmpe::group_leaders_sum(lsum);
    cnt = cmpe::group_leaders_sum(cnt);
    if (lane == 0) { s_sum[w] = lsum; s_cnt[w] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        int c = 0;
        for (int k = 0; k < kCmpeWarps; ++k) { a += s_sum[k]; c += s_cnt[k]; }
        patch_sum[P] = a;
        patch_cnt[P] = c;
        __threadfence();                               // the sums are visible before the count
        s_last = atomicAdd(&scal->cmpe_done, 1u) == gridDim.x - 1;
        __threadfence();
    }
    __syncthreads();
    if (s_last) cmpe_fold(g, patch_sum, patch_cnt, scal, loss);
}

// the fold alone, for plans without CMPE terms (L_CMPE = 0)
__global__ void __launch_bounds__(256) cmpe_finalize_kernel(AfGeom g, const double *__restrict__ patch_sum,
                                                            const int *__restrict__ patch_cnt,
                                                            AfScal *scal, float *__restrict__ loss)
{
    pdl_wait();
    cmpe_fold(g, patch_sum, patch_cnt, scal, loss);
}

// {sum m |arg z|, M} of the last forward, for callers that add them over plans
__global__ void cmpe_totals_kernel(const AfScal *__restrict__ scal, double *__restrict__ out)
{
    out[0] = scal->cmpe_sum;
    out[1] = (double)scal->n_active;
}

// Replaces the plan's CMPE normalisation by totals added over several plans (a
// patch-sharded run): L_CMPE = sum / max(1, M) of the whole problem, which the
// adjoint then differentiates; the loss vector is rewritten the way the patch
// fold writes it (the regularisers are this plan's own).
__global__ void cmpe_set_totals_kernel(AfGeom g, const double *__restrict__ in, AfScal *scal,
                                       float *__restrict__ loss)
{
    const double sum = in[0];
    const int M = (int)llrint(in[1]);
    const double lc = sum / (M > 1 ? M : 1);
    scal->cmpe_sum = sum;
    scal->n_active = M;
    scal->lcmpe = (float)lc;
    scal->inv_m = (float)(1.0 / (M > 1 ? M : 1));
    if (loss) {
        loss[0] = (float)(lc + (double)g.w1 * scal->rtv + (double)g.w2 * scal->rsv);
        loss[1] = (float)lc;
        loss[2] = scal->rtv;
        loss[3] = scal->rsv;
    }
}

// G[b][p] = dL_CMPE/dB_b(p): an image is the first member of at most one pair
// ((i,j) ~ (i+1,j-1)) and the second member of at most one ((i-1,j+1) ~ (i,j)).
//   first:  w j z B2 / |z|^2     second: -w j conj(z) B1 / |z|^2,  w = sgn(arg z) / max(1, M)
// Grid: (pixel blocks, image b); the image's two pairs are the same for the block.
__global__ void __launch_bounds__(256) cmpe_backward_kernel(AfGeom g, const float2 *__restrict__ B,
                                                            const float2 *__restrict__ z,
                                                            const uint8_t *__restrict__ mask,
                                                            const AfScal *__restrict__ scal,
                                                            float2 *__restrict__ G)
{
    const int n = g.nsub, b = blockIdx.y, i = b / n, j = b - i * n;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npix) return;
    G[(long)b * g.npix + p] = cmpe::image_grad(B, z, mask, scal->inv_m, n, g.npix, g.npair, p / g.patch_npix, i, j, p);
}

// Full-aperture image |sum_ij B_ij(p)| (Figs. 2, 4) and the integrated CMPE
// image: per pixel, the sum over the common-midpoint pairs of
// |arg(B_ij(p) conj(B_i+1,j-1(p)))| (Sec. IV).
__global__ void __launch_bounds__(256) image_kernel(AfGeom g, const float2 *__restrict__ B,
                                                    float *__restrict__ bmode, float *__restrict__ cimg)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npix) return;
    if (bmode) {
        float re = 0.f, im = 0.f;
        for (int b = 0; b < g.nb; ++b) {
            const float2 v = B[(long)b * g.npix + p];
            re += v.x;
            im += v.y;
        }
        bmode[p] = sqrtf(re * re + im * im);
    }
    if (cimg) {
        float acc = 0.f;
        for (int k = 0; k < g.npair; ++k) {
            int i, j;
            pair_ij(k, g.nsub, i, j);
            const float2 a = B[(long)(i * g.nsub + j) * g.npix + p];
            const float2 c = B[(long)((i + 1) * g.nsub + (j - 1)) * g.npix + p];
            acc += fabsf(atan2f(fmaf(a.y, c.x, -a.x * c.y), fmaf(a.x, c.x, a.y * c.y)));
        }
        cimg[p] = acc;
    }
}

}  // namespace

cudaError_t launch_images(af_plan_t pl, float *bmode, float *cimg)
{
    if (pl->g.npix == 0) return cudaSuccess;
    image_kernel<<<(pl->g.npix + 255) / 256, 256, 0, pl->stream>>>(pl->g, pl->B, bmode, cimg);
    return cudaGetLastError();
}

cudaError_t launch_cmpe_forward(af_plan_t pl, float *loss)
{
    if (pl->g.n_patch > 0 && pl->g.npair > 0) {
        return launch_dependent(cmpe_forward_kernel, dim3(pl->g.n_patch), dim3(32 * kCmpeWarps), 0, pl->stream, pl->g,
                                pl->B, pl->z, pl->mask, pl->patch_sum, pl->patch_cnt, pl->scal, loss);
    }
    AfGeom g = pl->g;
    g.n_patch = 0;                       // no terms: L_CMPE = 0
    return launch_dependent(cmpe_finalize_kernel, dim3(1), dim3(256), 0, pl->stream, g, pl->patch_sum, pl->patch_cnt,
                            pl->scal, loss);
}

cudaError_t launch_cmpe_totals(af_plan_t pl, double *out)
{
    cmpe_totals_kernel<<<1, 1, 0, pl->stream>>>(pl->scal, out);
    return cudaGetLastError();
}

cudaError_t launch_cmpe_set_totals(af_plan_t pl, const double *in, float *loss)
{
    cmpe_set_totals_kernel<<<1, 1, 0, pl->stream>>>(pl->g, in, pl->scal, loss);
    return cudaGetLastError();
}

cudaError_t launch_cmpe_backward(af_plan_t pl)
{
    const long total = (long)pl->g.nb * pl->g.npix;
    if (total == 0) return cudaSuccess;
    if (pl->g.npair == 0) {
        return cudaMemsetAsync(pl->G, 0, total * sizeof(float2), pl->stream);
    }
    const dim3 blocks((pl->g.npix + 255) / 256, pl->g.nb);
    cmpe_backward_kernel<<<blocks, 256, 0, pl->stream>>>(pl->g, pl->B, pl->z, pl->mask, pl->scal, pl->G);
    return cudaGetLastError();
}
