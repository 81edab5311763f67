// Adjoint of the discretised ray sum (Eq. 1, Sec. III-A) and of the
// regularisers (Eq. 10-11), then the Eq. 9 update as Adam.
//
// dL/ds_node = sum_{e,p} dL/dT[e][p] |q - r_p| / (N + 1) sum_k W_node(x_k)
//            + w1 dR_TV/ds + w2 dR_SV/ds.
// Each persistent CTA scatters its rays' bicubic weights into a private,
// padded copy of the grid in shared memory (shared-memory atomics only), folds
// the padding back onto the edge nodes and writes one partial grid; a second
// kernel sums the partials in a fixed order and adds the regulariser gradient.
// The padded row pitch is odd, so consecutive grid rows start in different
// shared-memory banks.
#include <math.h>

#include "af_internal.cuh"

namespace {

// Warp-cooperative scatter.  A warp takes 32 consecutive rays (element e,
// pixels p..p+31), compacts the ones with a non-zero dL/dT into a per-warp
// table, then walks their (N+1) points with lane = consecutive point index, so
// the 16 taps of one atomic instruction land on 32 different stencils along a
// ray (distinct addresses; the odd row pitch spreads them over the banks).
//
// Accumulation is int32 fixed point (shared-memory integer atomics are several
// times faster than float ones and their sums do not depend on order): value
// = round(c w S) with S = fix_scale / max|dL/dT|.  One ray adds at most
// max|dL/dT| (5 cell diagonals + L/(N+1)) to a node, and fix_scale is set on
// the host so that kRoundsPerFlush rounds of 256 rays stay below 2^30; after
// that many rounds the integer grid is flushed into the CTA's float
// accumulator in global memory and cleared.
constexpr int kRayWarps = 8;
constexpr int kRoundsPerFlush = 8;

__device__ __forceinline__ int round_to_int(float v)     // |v| < 2^22
{
    return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

__global__ void __launch_bounds__(256) ray_adjoint_kernel(AfGeom g, const float4 *__restrict__ elem,
                                                          const float2 *__restrict__ pix,
                                                          const float *__restrict__ phi,
                                                          const float *__restrict__ gdel,
                                                          const AfScal *__restrict__ scal,
                                                          float *__restrict__ gpad,
                                                          float *__restrict__ gpart)
{
    extern __shared__ int acci[];
    __shared__ float4 rays[kRayWarps][32];      // (gx0, gz0, gdx, gdz)
    __shared__ float rayc[kRayWarps][32];       // dL/dT |q - r| / (N + 1), scaled
    const int P = g.pitch, rows = g.nz + 4, npad = P * rows;
    for (int k = threadIdx.x; k < npad; k += blockDim.x) acci[k] = 0;
    float *mypad = gpad + (long)blockIdx.x * npad;
    for (int k = threadIdx.x; k < npad; k += blockDim.x) mypad[k] = 0.0f;
    const float gmax = __int_as_float(scal->gmax_bits);
    const float S = gmax > 0.0f ? g.fix_scale / gmax : 0.0f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npts = g.nseg + 1;
    const long total = (long)g.ne * g.npix;
    const long nchunks = (total + 31) / 32;
    // chunks of this CTA: blockIdx.x * 8 + warp + round * gridDim.x * 8
    const long per_round = (long)gridDim.x * kRayWarps;
    const long first = (long)blockIdx.x * kRayWarps;
    const long nrounds = first < nchunks ? (nchunks - first + per_round - 1) / per_round : 0;
    for (long round = 0; round < nrounds && S > 0.0f; ++round) {
        const long chunk = first + round * per_round + warp;
        const long idx = chunk * 32 + lane;
        float c = 0.0f;
        float4 rp = make_float4(0.f, 0.f, 0.f, 0.f);
        if (chunk < nchunks && idx < total) {
            const float gv = gdel[idx];
            if (gv != 0.0f) {
                const int e = (int)(idx / g.npix), p = (int)(idx - (long)e * g.npix);
                const float2 px = pix[p];
                float qx, qz;
                if (g.lens_mode == AF_LENS_BENT_RAY) {
                    float sn, cs;
                    sincosf(phi[idx], &sn, &cs);
                    qx = fmaf(g.RL, sn, g.arc_cx);
                    qz = fmaf(g.RL, cs, g.arc_cz);
                } else {
                    const float4 el = elem[e];
                    qx = el.x;
                    qz = el.y;
                }
                const float lx = px.x - qx, lz = px.y - qz;
                c = gv * S * sqrtf(lx * lx + lz * lz) * g.inv_nseg1;
                rp = make_float4((qx - g.x0) * g.inv_dx, (qz - g.z0) * g.inv_dz,
                                 lx * g.inv_dx * g.inv_nseg, lz * g.inv_dz * g.inv_nseg);
            }
        }
        const unsigned live = __ballot_sync(0xffffffffu, c != 0.0f);
        const int nlive = __popc(live);
        if (c != 0.0f) {
            const int slot = __popc(live & ((1u << lane) - 1u));
            rays[warp][slot] = rp;
            rayc[warp][slot] = c;
        }
        __syncwarp();
        const int npt_total = nlive * npts;
        for (int q = lane; q < npt_total; q += 32) {
            const int r = q / npts, k = q - r * npts;
            const float4 ry = rays[warp][r];
            const float cr = rayc[warp][r];
            const float gx = fmaf((float)k, ry.z, ry.x), gz = fmaf((float)k, ry.w, ry.y);
            const float fx = floorf(gx), fz = floorf(gz);
            const int i0 = min(max((int)fx, -1), g.nx - 1), j0 = min(max((int)fz, -1), g.nz - 1);
            float wx[4], wz[4];
            keys_weights(gx - fx, wx);
            keys_weights(gz - fz, wz);
            int *row = acci + (j0 + 1) * P + (i0 + 1);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float cb = cr * wz[b];
#pragma unroll
                for (int a = 0; a < 4; ++a) atomicAdd(row + b * P + a, round_to_int(cb * wx[a]));
            }
        }
        __syncwarp();
        if ((round + 1) % kRoundsPerFlush == 0 || round + 1 == nrounds) {
            __syncthreads();
            const float inv = 1.0f / S;
            for (int k = threadIdx.x; k < npad; k += blockDim.x) {
                const int v = acci[k];
                if (v != 0) {
                    mypad[k] += (float)v * inv;
                    acci[k] = 0;
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // fold the padding onto the clamped edge nodes and write this CTA's partial grid
    float *out = gpart + (long)blockIdx.x * g.ng;
    for (int k = threadIdx.x; k < g.ng; k += blockDim.x) {
        const int j = k / g.nx, i = k - j * g.nx;
        const int ilo = i == 0 ? 0 : i + 2, ihi = i == g.nx - 1 ? g.nx + 3 : i + 2;
        const int jlo = j == 0 ? 0 : j + 2, jhi = j == g.nz - 1 ? g.nz + 3 : j + 2;
        float v = 0.0f;
        for (int jj = jlo; jj <= jhi; ++jj)
            for (int ii = ilo; ii <= ihi; ++ii) v += mypad[jj * P + ii];
        out[k] = v;
    }
}

__device__ __forceinline__ float dz_sign(float x, float k)      // D_k'(x)
{
    return fabsf(x) <= k ? 0.0f : (x > 0.0f ? 1.0f : -1.0f);
}

// grad[k] = sum_c gpart[c][k] + d(w1 R_TV + w2 R_SV)/ds_k  (gather form on c = 1/s)
__global__ void __launch_bounds__(256) reduce_grad_kernel(AfGeom g, const float *__restrict__ s,
                                                          const float *__restrict__ gpart, int nparts,
                                                          float *__restrict__ grad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ng) return;
    float acc = 0.0f;
    for (int c = 0; c < nparts; ++c) acc += gpart[(long)c * g.ng + k];
    const int j = k / g.nx, i = k - j * g.nx, nx = g.nx, nz = g.nz;
    auto C = [&](int ii, int jj) { return 1.0f / s[jj * nx + ii]; };
    const float hx = g.hx_mm, hz = g.hz_mm, hx2 = hx * hx, hz2 = hz * hz;
    float dc = 0.0f;   // dR/dc_k
    // Eq. 10: forward differences touching node k
    float a = 0.0f;
    if (i >= 1) a += dz_sign((C(i, j) - C(i - 1, j)) / hx, g.kx1) / hx;
    if (i + 1 < nx) a -= dz_sign((C(i + 1, j) - C(i, j)) / hx, g.kx1) / hx;
    if (j >= 1) a += dz_sign((C(i, j) - C(i, j - 1)) / hz, g.kz1) / hz;
    if (j + 1 < nz) a -= dz_sign((C(i, j + 1) - C(i, j)) / hz, g.kz1) / hz;
    dc += g.w1 * g.na_inv * a;
    // Eq. 11: central second differences whose stencil contains node k
    float b = 0.0f;
    for (int m = i - 1; m <= i + 1; ++m) {
        if (m < 1 || m > nx - 2) continue;
        const float d = dz_sign((C(m + 1, j) - 2.0f * C(m, j) + C(m - 1, j)) / hx2, g.kx2) / hx2;
        b += m == i ? -2.0f * d : d;
    }
    for (int m = j - 1; m <= j + 1; ++m) {
        if (m < 1 || m > nz - 2) continue;
        const float d = dz_sign((C(i, m + 1) - 2.0f * C(i, m) + C(i, m - 1)) / hz2, g.kz2) / hz2;
        b += m == j ? -2.0f * d : d;
    }
    dc += g.w2 * g.nb_inv * b;
    const float c0 = C(i, j);
    grad[k] = acc - dc * c0 * c0;     // dc/ds = -c^2
}

// Adam on u = s * c_ref (Eq. 9 with Adam moments)
__global__ void __launch_bounds__(256) adam_kernel(AfGeom g, const float *__restrict__ grad,
                                                   float *__restrict__ s, float *__restrict__ m,
                                                   float *__restrict__ v, float bc1, float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ng) return;
    const float gu = grad[k] / g.c_ref;
    const float mk = fmaf(g.beta1, m[k], g.omb1 * gu);
    const float vk = fmaf(g.beta2, v[k], g.omb2 * gu * gu);
    m[k] = mk;
    v[k] = vk;
    const float u = s[k] * g.c_ref - g.lr * (mk / bc1) / (sqrtf(vk / bc2) + g.eps);
    s[k] = u / g.c_ref;
}

}  // namespace

int rayadj_blocks_per_sm(size_t smem)
{
    int n = 0;
    // the attribute is per function, shared by every plan: set it to the largest
    // grid any plan may use, the occupancy query uses this plan's size
    cudaFuncSetAttribute(ray_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxGridSmemBytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ray_adjoint_kernel, 256, smem);
    return n > 0 ? n : 1;
}

cudaError_t launch_ray_adjoint(af_plan_t pl, const float *s, float *grad)
{
    int nparts = 0;
    if ((long)pl->g.ne * pl->g.npix > 0) {
        ray_adjoint_kernel<<<pl->rayadj_blocks, 256, pl->smem_grid, pl->stream>>>(
            pl->g, pl->elem, pl->pix, pl->phi, pl->gdel, pl->scal, pl->gpad, pl->gpart);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        nparts = pl->rayadj_blocks;
    }
    reduce_grad_kernel<<<(pl->g.ng + 255) / 256, 256, 0, pl->stream>>>(pl->g, s, pl->gpart, nparts, grad);
    return cudaGetLastError();
}

cudaError_t launch_adam(af_plan_t pl, const float *grad, float *s, float *m, float *v, int step)
{
    const double bc1 = 1.0 - pow((double)pl->g.beta1, step);
    const double bc2 = 1.0 - pow((double)pl->g.beta2, step);
    adam_kernel<<<(pl->g.ng + 255) / 256, 256, 0, pl->stream>>>(pl->g, grad, s, m, v, (float)bc1, (float)bc2);
    return cudaGetLastError();
}
