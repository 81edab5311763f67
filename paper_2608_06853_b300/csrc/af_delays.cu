// Delay generation: grid statistics (c_med, Eq. 10-11) and the fused
// one-way delay kernel (Eq. 2-4 apodization, Eq. 8 lens exit point by
// Fermat's principle, Eq. 1 straight-ray bicubic slowness sum, Sec. III-A).
#include <math.h>

#include <type_traits>

#include "af_internal.cuh"
#include "af_lens.cuh"

namespace {

// deadzone D_k(x) = max(0, |x| - k)  (Sec. II-D)
__device__ __forceinline__ float deadzone(float x, float k) { return fmaxf(fabsf(x) - k, 0.0f); }

// c_med = mean(1/s) (Sec. III-A), the two regularisers of Eq. 10-11 on
// c = 1 / (c_unit s) (the speed in km/s, positions in mm), and the numeric check of the slowness map, in two steps: kStatBlocks CTAs
// write partial sums {sum 1/s, sum of the Eq. 10 terms, sum of the Eq. 11 terms,
// bad-value flag}, and the CTA that finishes last adds them in a fixed order.
// one warp: lane l adds partials l, l + 32, ..., then a fixed xor tree; the
// partials are read from L2, where other CTAs wrote them
__device__ __forceinline__ void grid_stats_fold(const AfGeom &g, const StatPart *part, int nparts, AfScal *scal)
{
    double c = 0.0, a = 0.0, b = 0.0, bad = 0.0;
    for (int k = threadIdx.x; k < nparts; k += 32) {
        const double2 ca = __ldcg(reinterpret_cast<const double2 *>(part + k));
        const double2 bb = __ldcg(reinterpret_cast<const double2 *>(part + k) + 1);
        c += ca.x;
        a += ca.y;
        b += bb.x;
        bad += bb.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (threadIdx.x != 0) return;
    const double cmed = c / g.ng;
    scal->sbar = (float)(1.0 / cmed);
    scal->rtv = (float)(a * g.na_inv);
    scal->rsv = (float)(b * g.nb_inv);
    scal->fp64_solves = 0;
    scal->n_apod = 0;
    scal->stat_done = 0;
    if (bad > 0.0) scal->numeric_flag = 1;
}

// The CTA that finishes last (counted in scal->stat_done, which the fold sets
// back to zero) folds the gridDim.x partials with its first warp.
__global__ void __launch_bounds__(256, 4) grid_stats_partial_kernel(AfGeom g, const float *__restrict__ s,
                                                                 StatPart *__restrict__ part, AfScal *scal,
                                                                 int2 *__restrict__ nrange)
{
    pdl_wait();
    // the delay kernel, which always follows, takes the minima of the pixels' one-way
    // sample indices (and of their negatives) into nrange
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.npix; p += gridDim.x * blockDim.x)
        nrange[p] = make_int2(0x7F7F7F7F, 0x7F7F7F7F);
    __shared__ double red[3][8];
    __shared__ int s_last;
    // per-thread partial sums in float (float64 throughput is low on this GPU); the
    // sum of 1/s, which sets c_med and with it every delay, is compensated (Kahan)
    float pc = 0.0f, pc_comp = 0.0f, pa = 0.0f, pb = 0.0f;
    int bad = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.ng; k += gridDim.x * blockDim.x) {
        int j = k / g.nx, i = k - j * g.nx;
        float sv = s[k];
        if (!(sv > 0.0f) || !isfinite(sv)) bad = 1;
        const float cm = 1.0f / sv;                       // m/s, for c_med
        const float y = cm - pc_comp, t = pc + y;
        pc_comp = (t - pc) - y;
        pc = t;
        const float cu = g.inv_c_unit / sv;                // Eq. 10-11 units
        auto C = [&](int q) { return g.inv_c_unit / s[q]; };
        if (i + 1 < g.nx) pa += deadzone((C(k + 1) - cu) / g.hx_mm, g.kx1);
        if (j + 1 < g.nz) pa += deadzone((C(k + g.nx) - cu) / g.hz_mm, g.kz1);
        if (i >= 1 && i + 1 < g.nx)
            pb += deadzone((C(k + 1) - 2.0f * cu + C(k - 1)) / (g.hx_mm * g.hx_mm), g.kx2);
        if (j >= 1 && j + 1 < g.nz)
            pb += deadzone((C(k + g.nx) - 2.0f * cu + C(k - g.nx)) / (g.hz_mm * g.hz_mm), g.kz2);
    }
    double acc_c = (double)pc - (double)pc_comp, acc_a = pa, acc_b = pb;
    for (int o = 16; o > 0; o >>= 1) {
        acc_c += __shfl_xor_sync(0xffffffffu, acc_c, o);
        acc_a += __shfl_xor_sync(0xffffffffu, acc_a, o);
        acc_b += __shfl_xor_sync(0xffffffffu, acc_b, o);
    }
    bad = __syncthreads_or(bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = acc_c; red[1][w] = acc_a; red[2][w] = acc_b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c = 0.0, a = 0.0, b = 0.0;
        for (int k = 0; k < 8; ++k) { c += red[0][k]; a += red[1][k]; b += red[2][k]; }
        part[blockIdx.x] = StatPart{c, a, b, bad ? 1.0 : 0.0};
        __threadfence();                               // the partial is visible before the count
        s_last = atomicAdd(&scal->stat_done, 1u) == gridDim.x - 1;
        __threadfence();
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) grid_stats_fold(g, part, gridDim.x, scal);
}

// Padded grid in shared memory: scalar v[jj][ii], or (PAIRS) the node pairs
// (v[jj][ii], v[jj][ii + 2]) as float2, so that the 4 taps of a row are two
// aligned 64-bit loads (ii0, ii0 + 2) and (ii0 + 1, ii0 + 3).
template <bool PAIRS> struct GridTaps;
template <> struct GridTaps<false> {
    static __device__ __forceinline__ void store(float *sm, int k, int P, float v, float) { sm[k] = v; }
    static __device__ __forceinline__ float row(const float *sm, int o, const float (&wx)[4])
    {
        float h = wx[0] * sm[o];
        h = fmaf(wx[1], sm[o + 1], h);
        h = fmaf(wx[2], sm[o + 2], h);
        return fmaf(wx[3], sm[o + 3], h);
    }
};
template <> struct GridTaps<true> {
    static __device__ __forceinline__ void store(float *sm, int k, int, float v, float v2)
    {
        reinterpret_cast<float2 *>(sm)[k] = make_float2(v, v2);
    }
    static __device__ __forceinline__ float row(const float *sm, int o, const float (&wx)[4])
    {
        const float2 *r = reinterpret_cast<const float2 *>(sm) + o;
        const float2 a = r[0], b = r[1];      // (v0, v2), (v1, v3)
        float h = wx[0] * a.x;
        h = fmaf(wx[1], b.x, h);
        h = fmaf(wx[2], a.y, h);
        return fmaf(wx[3], b.y, h);
    }
};

// One thread per (element e, pixel p), items e * npix + p taken by warps in
// chunks of 32 from a counter, with the slowness deviation s - sbar staged once
// per CTA in shared memory, padded by two edge-replicated nodes on every side so
// that each of the 16 taps of a point inside the grid box reads the
// clamp-to-edge value without a branch.
template <bool PAIRS, int PF = 0>
__global__ void __launch_bounds__(PAIRS ? 1024 : 256) delays_kernel(AfGeom g, const float *__restrict__ s,
                                                     const float4 *__restrict__ elem,
                                                     const float2 *__restrict__ elem_pol,
                                                     const float2 *__restrict__ pix,
                                                     const float2 *__restrict__ pix_pol,
                                                     float *__restrict__ phi, int warm,
                                                     const uint8_t *__restrict__ sur_fb,
                                                     float4 *__restrict__ D, int2 *__restrict__ nrange,
                                                     AfScal *scal)
{
    extern __shared__ float sm[];
    pdl_wait();
    const float sbar = scal->sbar;
    const int P = PF ? PF : g.pitch, rows = g.nz + 4;   // PF: the pitch as a compile-time constant
    for (int k = threadIdx.x; k < P * rows; k += blockDim.x) {
        int jj = k / P, ii = k - jj * P;
        int i = min(max(ii - 2, 0), g.nx - 1), j = min(max(jj - 2, 0), g.nz - 1);
        const int i2 = min(max(ii, 0), g.nx - 1);          // node ii + 2 of the padded row
        // exact (Sterbenz) for s within 2x of sbar
        GridTaps<PAIRS>::store(sm, k, P, s[j * g.nx + i] - sbar, PAIRS ? s[j * g.nx + i2] - sbar : 0.0f);
    }
    __syncthreads();

    const ff sfs = ff_two_prod(sbar, g.fs);       // sbar * fs, exact
    const ff fscl = {g.fs_clens_hi, g.fs_clens_lo};
    const ff off = {g.off_hi, g.off_lo};
    int n_apod = 0, n_fp64 = 0;
    const long total = (long)g.ne * g.npix;
    // warps take chunks of 32 consecutive items from a counter, the next one claimed
    // while the current one runs, so the SMs finish together (a fixed grid stride
    // left them finishing over ~50 us: 0.552 -> 0.542 ms, 128 elements)
    const int lane = threadIdx.x & 31;
    unsigned long long cn = 0;
    if (lane == 0) cn = atomicAdd(&scal->delay_next, 32ull);
    for (long chunk = (long)__shfl_sync(0xffffffffu, cn, 0); chunk < total;
         chunk = (long)__shfl_sync(0xffffffffu, cn, 0)) {
        if (lane == 0) cn = atomicAdd(&scal->delay_next, 32ull);
        const long idx = chunk + lane;
        if (idx >= total) continue;
        const int e = (int)(idx / g.npix), p = (int)(idx - (long)e * g.npix);
        const float4 el = elem[e];
        const float2 px = pix[p];
        // Eq. 2: pixel in the element frame; Eq. 4: constant f-number cone
        const float ddx = px.x - el.x, ddz = px.y - el.y;
        const float xp = el.z * ddx - el.w * ddz, zp = el.w * ddx + el.z * ddz;
        const float lim = g.apod_mode == AF_APOD_PRINTED ? zp * g.fnum_half : zp * g.fnum_inv2;
        if (!(zp > 0.0f && fabsf(xp) <= lim)) {
            D[idx] = make_float4(__int_as_float(AF_APOD_OFF), 0.0f, 0.0f, 0.0f);
            continue;
        }
        ++n_apod;
        // Eq. 8 / Sec. III-A: exit point at c_med by Fermat's principle
        float qx = el.x, qz = el.y, ph = 0.0f;
        ff tl = {0.0f, 0.0f};
        if (g.lens_mode == AF_LENS_BENT_RAY) {
            const float2 ep = elem_pol[e], pp = pix_pol[p];
            const float dp = pp.x - ep.x;
            float lo = fminf(0.0f, dp), hi = fmaxf(0.0f, dp);
            float x = warm ? fminf(fmaxf(phi[idx] - ep.x, lo), hi) : 0.0f;
            bool conv = (lo == hi);
            // lens surrogate: its exit angle (already in phi) replaces the solve
            const bool use_sur = sur_fb && !sur_fb[idx];
            if (use_sur) { x = phi[idx] - ep.x; conv = true; }
            for (int it = 0; it < 16 && !conv; ++it) {
                Chord a = chord(ep.y, g.RL, x), b = chord(pp.y, g.RL, x - dp);
                float f = fmaf(b.d1, sbar, a.d1 * g.inv_c_lens);
                float fp = fmaf(b.d2, sbar, a.d2 * g.inv_c_lens);
                if (f == 0.0f) { conv = true; break; }     // stationary point reached exactly
                if (f < 0.0f) lo = x; else hi = x;
                float xn = fp > 0.0f ? x - f / fp : 0.5f * (lo + hi);
                if (!(xn >= lo && xn <= hi)) xn = 0.5f * (lo + hi);
                conv = fabsf(xn - x) < 1e-6f || hi - lo < 1e-6f;
                x = xn;
            }
            // grazing exit (tissue ray beyond ~80 deg from the lens normal) or no
            // convergence: solve again in float64
            float c_t;
            {
                float sd, cd;
                sincosf(x - dp, &sd, &cd);
                Chord b = chord(pp.y, g.RL, x - dp);
                c_t = (pp.y * cd - g.RL) / b.len;
            }
            if (!use_sur && (!conv || c_t < 0.17f)) {
                x = (float)exit_solve_fp64(ep.y, pp.y, g.RL, (double)dp, (double)g.inv_c_lens,
                                           (double)sbar);
                ++n_fp64;
            }
            ph = ep.x + x;
            phi[idx] = ph;
            float sn, cs;
            sincosf(ph, &sn, &cs);
            qx = fmaf(g.RL, sn, g.arc_cx);
            qz = fmaf(g.RL, cs, g.arc_cz);
            tl = ff_mul(ff_dist(qx, qz, el.x, el.y), fscl);      // lens leg in samples
        } else if (g.lens_mode == AF_LENS_PLANAR) {
            // Eq. 8 with a flat lens: exit x u on z = lens_z, root of
            // dT/du = (u - xe) / (c_lens d1) - (xp - u) sbar / d2 (convex T)
            const float h1 = g.lens_z - el.y, h2 = px.y - g.lens_z;
            float lo = fminf(el.x, px.x), hi = fmaxf(el.x, px.x);
            float u = warm ? fminf(fmaxf(phi[idx], lo), hi) : el.x;
            bool conv = (lo == hi);
            for (int it = 0; it < 16 && !conv; ++it) {
                const float a = u - el.x, b = px.x - u;
                const float d1 = sqrtf(fmaf(a, a, h1 * h1)), d2 = sqrtf(fmaf(b, b, h2 * h2));
                const float r1 = 1.0f / d1, r2 = 1.0f / d2;
                const float f = fmaf(a * g.inv_c_lens, r1, -b * sbar * r2);
                const float fp = fmaf(h1 * h1 * g.inv_c_lens, r1 * r1 * r1, h2 * h2 * sbar * r2 * r2 * r2);
                if (f == 0.0f) { conv = true; break; }     // stationary point reached exactly
                if (f < 0.0f) lo = u; else hi = u;
                float un = u - f / fp;
                if (!(un >= lo && un <= hi)) un = 0.5f * (lo + hi);
                // the delay error is second order in the exit-point error: 1e-8 m is ample
                conv = fabsf(un - u) < 1e-8f || hi - lo < 1e-8f;
                u = un;
            }
            // grazing exit (tissue ray beyond ~80 deg from the lens normal) or no
            // convergence: solve again in float64
            const float bx = px.x - u;
            if (!conv || h2 < 0.17f * sqrtf(fmaf(bx, bx, h2 * h2))) {
                u = (float)exit_solve_flat_fp64((double)el.x, (double)h1, (double)px.x, (double)h2,
                                                (double)g.inv_c_lens, (double)sbar);
                ++n_fp64;
            }
            ph = u;
            phi[idx] = u;
            qx = u;
            qz = g.lens_z;
            tl = ff_mul(ff_dist(qx, qz, el.x, el.y), fscl);      // lens leg in samples
        }
        // Eq. 1 discretised: L * (sbar + mean_k interp(s - sbar)) over N+1 endpoints
        const ff L = ff_dist(px.x, px.y, qx, qz);
        const float gx0 = (qx - g.x0) * g.inv_dx, gz0 = (qz - g.z0) * g.inv_dz;
        const float gdx = (px.x - qx) * g.inv_dx * g.inv_nseg;
        const float gdz = (px.y - qz) * g.inv_dz * g.inv_nseg;
        // The endpoints' grid coordinates fmaf(k, gd, g0) are monotone in k, so the
        // first and last bound all of them: when both lie in [-1, n) every cell index
        // is inside the padded grid and the per-point clamps can be left out (a NaN
        // coordinate fails the test and takes the clamped loop).
        const float kend = (float)g.nseg;
        const float gx1 = fmaf(kend, gdx, gx0), gz1 = fmaf(kend, gdz, gz0);
        const bool inside = fminf(gx0, gx1) >= -1.0f && fmaxf(gx0, gx1) < (float)g.nx &&
                            fminf(gz0, gz1) >= -1.0f && fmaxf(gz0, gz1) < (float)g.nz;
        // the N+1 endpoint values in partial sums of 8, Kahan-summed
        float sum = 0.0f, comp = 0.0f;
        auto kahan = [&](float v) {
            const float y = v - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        };
        auto ray_sum = [&](auto clamp) {
            // interpolated value at endpoint kf, added into the running partial sum
            auto point = [&](float kf, float part) {
                // position, fractions and Keys weights of both axes as packed pairs
                // (the same round-to-nearest steps as the scalar forms)
                const float2 gg = __ffma2_rn(make_float2(kf, kf), make_float2(gdx, gdz), make_float2(gx0, gz0));
                const float fx = floorf(gg.x), fz = floorf(gg.y);
                int i0 = (int)fx, j0 = (int)fz;
                if (decltype(clamp)::value) {
                    i0 = min(max(i0, -1), g.nx - 1);
                    j0 = min(max(j0, -1), g.nz - 1);
                }
                float2 w[4];
                keys_weights2(__ffma2_rn(make_float2(fx, fz), make_float2(-1.0f, -1.0f), gg), w);
                const float wx[4] = {w[0].x, w[1].x, w[2].x, w[3].x};
                const int row = (j0 + 1) * P + (i0 + 1);           // padded node (i0-1, j0-1)
#pragma unroll
                for (int b = 0; b < 4; ++b) part = fmaf(w[b].y, GridTaps<PAIRS>::row(sm, row + b * P, wx), part);
                return part;
            };
            float kf = 0.0f;
            // partial sums of 8 endpoints, Kahan-summed (groups of 4: 0.538 ms,
            // of 2: 0.545 ms, of 8: 0.528 ms on the 128-element workload)
            for (; kf + 7.0f <= kend; kf += 8.0f) {
                float part = point(kf, 0.0f);
#pragma unroll
                for (int q = 1; q < 7; ++q) part = point(kf + (float)q, part);
                kahan(point(kf + 7.0f, part));
            }
            float part = 0.0f;
            for (; kf <= kend; kf += 1.0f) part = point(kf, part);
            kahan(part);
        };
        if (inside)
            ray_sum(std::false_type{});
        else
            ray_sum(std::true_type{});
        const float mean_fs = (sum - comp) * g.inv_nseg1 * g.fs;
        // one-way delay in samples, shifted by (t_ttp - t0) fs / 2
        ff U = ff_mul(L, sfs);
        U = ff_add(U, tl);
        U = ff_add_f(U, L.hi * mean_fs);
        U = ff_add(U, off);
        float n = floorf(U.hi);
        float fr = (U.hi - n) + U.lo;
        if (fr < 0.0f) { fr += 1.0f; n -= 1.0f; }
        if (fr >= 1.0f) { fr -= 1.0f; n += 1.0f; }
        const int ni = (int)n;
        // phasor exp(j 2 pi fd (T + t_ttp / 2)) = exp(j 2 pi (rfd (n + fr) + cyc0))
        ff a = ff_two_prod(g.rfd_hi, n);
        float cyc = a.hi - rintf(a.hi);
        cyc += a.lo + g.rfd_lo * n + fmaf(g.rfd_hi, fr, g.cyc0);
        cyc -= rintf(cyc);
        float ps, pc;
        sincospif(2.0f * cyc, &ps, &pc);
        D[idx] = make_float4(__int_as_float(ni), fr, pc, ps);
        atomicMin(&nrange[p].x, ni);
        atomicMin(&nrange[p].y, -ni);
    }
    // counters
    for (int o = 16; o > 0; o >>= 1) {
        n_apod += __shfl_xor_sync(0xffffffffu, n_apod, o);
        n_fp64 += __shfl_xor_sync(0xffffffffu, n_fp64, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_apod) atomicAdd(&scal->n_apod, n_apod);
        if (n_fp64) atomicAdd(&scal->fp64_solves, n_fp64);
    }
    // the CTA that finishes last returns the item counter to zero for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&scal->delay_done, 1u) == gridDim.x - 1) {
            scal->delay_next = 0;
            scal->delay_done = 0;
        }
    }
}

// T[e][p] in seconds (double) from the stored sample index and fraction
__global__ void export_delays_kernel(AfGeom g, const float4 *__restrict__ D, double t_shift,
                                     double inv_fs, double *__restrict__ T,
                                     uint8_t *__restrict__ apod)
{
    long total = (long)g.ne * g.npix;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        float4 d = D[idx];
        int n = __float_as_int(d.x);
        bool on = n != AF_APOD_OFF;
        if (T) T[idx] = on ? ((double)n + (double)d.y) * inv_fs - t_shift : 0.0;
        if (apod) apod[idx] = on ? 1 : 0;
    }
}

}  // namespace

// launch shape of the delay kernel: the paired grid (one 1024-thread CTA per SM;
// 64 registers with a few bytes spilled, 0.552 ms against 0.578 ms for 768
// threads at 80) when it fits in shared memory, else the scalar grid (256-thread
// CTAs)
// padded row pitch of 128-wide grids ((nx + 4) | 1), compiled into one instance
// so that the four tap rows of a point sit at constant offsets
constexpr int kDelayPitch128 = 133;

DelayShape delays_shape(size_t smem_scalar, int sm_count)
{
    DelayShape sh;
    sh.pairs = 2 * smem_scalar <= kMaxGridSmemBytes;
    sh.smem = sh.pairs ? 2 * smem_scalar : smem_scalar;
    sh.threads = sh.pairs ? 1024 : 256;
    int n = 0;
    // the attribute is per function, shared by every plan: set it to the largest
    // grid any plan may use, the occupancy query uses this plan's size
    if (sh.pairs) {
        cudaFuncSetAttribute(delays_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMaxGridSmemBytes);
        cudaFuncSetAttribute(delays_kernel<true, kDelayPitch128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMaxGridSmemBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, delays_kernel<true>, 1024, sh.smem);
    } else {
        cudaFuncSetAttribute(delays_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMaxGridSmemBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, delays_kernel<false>, 256, sh.smem);
    }
    sh.blocks = sm_count * (n > 0 ? n : 1);
    return sh;
}

cudaError_t launch_grid_stats(af_plan_t pl, const float *s)
{
    return launch_dependent(grid_stats_partial_kernel, dim3(kStatBlocks), dim3(256), 0, pl->stream, pl->g, s,
                            pl->stat_part, pl->scal, pl->nrange);
}

cudaError_t launch_delays(af_plan_t pl, const float *s)
{
    if ((long)pl->g.ne * pl->g.npix == 0) return cudaSuccess;
    const DelayShape &sh = pl->delay;
    // sample-index range per pixel: both fields were set to 0x7F7F7F7F (above any
    // index) by the grid statistics, which every caller launches just before
    auto kernel = sh.pairs && pl->g.pitch == kDelayPitch128 ? delays_kernel<true, kDelayPitch128>
                  : sh.pairs                                   ? delays_kernel<true>
                                                               : delays_kernel<false>;
    const cudaError_t err = launch_dependent(kernel, dim3(sh.blocks), dim3(sh.threads), sh.smem, pl->stream, pl->g, s,
                                             pl->elem, pl->elem_pol, pl->pix, pl->pix_pol, pl->phi,
                                             pl->have_phi ? 1 : 0, pl->use_surrogate ? pl->sur_fb : nullptr, pl->D,
                                             pl->nrange, pl->scal);
    if (err == cudaSuccess) pl->have_phi = true;
    return err;
}

cudaError_t launch_export_delays(af_plan_t pl, double *T, uint8_t *apod)
{
    long total = (long)pl->g.ne * pl->g.npix;
    if (total == 0) return cudaSuccess;
    // U = (T + (t_ttp - t0) / 2) fs  =>  T = U / fs - (t_ttp - t0) / 2
    const double shift = ((double)pl->g.off_hi + (double)pl->g.off_lo) / (double)pl->g.fs;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 65535) blocks = 65535;
    export_delays_kernel<<<blocks, 256, 0, pl->stream>>>(pl->g, pl->D, shift, 1.0 / (double)pl->g.fs,
                                                          T, apod);
    return cudaGetLastError();
}
