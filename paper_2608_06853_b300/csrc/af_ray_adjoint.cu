// Adjoint of the discretised ray sum (Eq. 1, Sec. III-A) and of the
// regularisers (Eq. 10-11), then the Eq. 9 update as Adam.
//
// dL/ds_node = sum_{e,p} dL/dT[e][p] |q - r_p| / (N + 1) sum_k W_node(x_k)
//            + w1 dR_TV/ds + w2 dR_SV/ds.
// Each persistent CTA scatters its rays' bicubic weights into a private,
// padded copy of the grid in shared memory (shared-memory atomics only) and
// adds it, block by block, into one padded integer grid in global memory; a
// second kernel folds the padding back onto the edge nodes, clears the grid for
// the next launch and adds the regulariser gradient.  The padded row pitch is odd, so consecutive grid rows
// start in different shared-memory banks.
#include <math.h>

#include "af_internal.cuh"

namespace {

// Scatter of the ray points.  A work item is one element and kRayGroup
// consecutive pixels (for a 9 x 9 patch, a third of one patch row); their
// rays run side by side, so at one step k their points usually fall in the
// same grid cell.  A CTA takes blocks of one item per thread from a device
// counter (blocks differ in work because of the apodization; a block's inputs
// are loaded while the block before it is scattered; the last round of blocks
// is cut into quarter blocks), compacts the
// items with a non-zero dL/dT into a table, and spreads the flattened
// (item, step) list over all its threads (lane = consecutive step along a
// ray).  A thread sums, in registers, the 4 x 4 stencils of the item's points
// that share the cell of its middle ray and adds them with one set of 16
// shared-memory atomics.  A point in another cell goes to a per-warp queue,
// which is processed 32 points at a time (one point per lane), so that these
// points do not run as a divergent branch.
//
// Bank layout.  Along one ray the visited cells form a monotone path; with a
// row pitch of 1 (mod 32) the bank of cell (i, j) is i + j (mod 32), so for a
// ray going right-down (or left-up) the banks of 32 consecutive points differ
// by their Manhattan distance and do not collide; rays going left-down use a
// second copy of the grid with a row pitch of 31 (mod 32), bank i - j.  When
// both copies do not fit in shared memory one copy with an odd pitch is used.
//
// Accumulation is fixed point: value = round(c w S), S = fix_scale /
// max|dL/dT|.  Shared memory holds int32 (integer atomics are several times
// faster than float ones).  A ray with dL/dT = g adds at most |g| (5 cell
// diagonals + L/(N+1)) to a node, and fix_scale is set on the host so that
// kRayFlushRays rays with |g| = max|dL/dT| stay below 2^30.  Each block sums
// |g| / max|dL/dT| over its rays; before a block is scattered whose sum would
// take the total since the last flush past that budget, the integer grids are
// added into the int64 padded grid in global memory, by integer atomic adds no
// thread waits for, and cleared (and once more at the end).  Most rays carry far
// less than the largest |dL/dT|, so a CTA flushes rarely (flushing after every
// block of 768 items cost 0.730 against 0.700 ms).  All sums are integer sums up
// to the final conversion, so the result depends neither on which CTA took which
// block nor on the order of the adds.  Rounding adds 1.5 * 2^23 in the last FMA
// of a value (|value| < 2^22), so each partial sum is rounded to an integer.
struct RayGrid {
    int width, rows;        // padded grid: nx + 4 columns, nz + 4 rows
    int pa, pb, base_b;     // row pitch of copy A (and B), offset of copy B
};

constexpr float kRound = 12582912.0f;   // 1.5 * 2^23
constexpr int kRoundBits = 0x4B400000;
constexpr int kLeadRay = kRayGroup / 2; // the middle ray of an item

// padded cell of point k of a ray (gx0, gz0, gdx, gdz), the floors of its grid
// coordinates and its Keys weights
__device__ __forceinline__ void ray_stencil(const AfGeom &g, float k, float4 ry, int &ic, int &jc, float &fx,
                                            float &fz, float wx[4], float wz[4])
{
    const float gx = fmaf(k, ry.z, ry.x), gz = fmaf(k, ry.w, ry.y);
    fx = floorf(gx);
    fz = floorf(gz);
    ic = min(max((int)fx, -1), g.nx - 1) + 1;
    jc = min(max((int)fz, -1), g.nz - 1) + 1;
    keys_weights(gx - fx, wx);
    keys_weights(gz - fz, wz);
}

// t in [0, 1) (as bits: +0 up to the largest float below 1)
__device__ __forceinline__ bool unit_fraction(float t) { return __float_as_uint(t) < 0x3F800000u; }

// 16 atomics of one stencil whose values carry the rounding constant
__device__ __forceinline__ void add_stencil(int *row, int pitch, const float (&W)[16])
{
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) atomicAdd(row + b * pitch + a, __float_as_int(W[b * 4 + a]) - kRoundBits);
}

// grid copy of an item (rayb = 1: copy B) as (base, row pitch)
template <bool DUAL>
__device__ __forceinline__ int2 copy_of(const RayGrid &rg, int b)
{
    return DUAL && b ? make_int2(rg.base_b, rg.pb) : make_int2(0, rg.pa);
}

// one queued point: entry = (item << 18) | (step << 2) | ray
template <bool DUAL>
__device__ __forceinline__ void run_queued(const AfGeom &g, const RayGrid &rg, int ent, int *acci,
                                           const float4 *rays, int T, const float *rayc, const int *rayb)
{
    const int r = ent >> 18, k = (ent >> 2) & 0xFFFF, m = ent & 3;
    const int2 gb = copy_of<DUAL>(rg, rayb[r]);
    const float cm = rayc[m * T + r];
    float wx[4], wz[4], W[16], fx, fz;
    int i1, j1;
    ray_stencil(g, (float)k, rays[m * T + r], i1, j1, fx, fz, wx, wz);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float cb = cm * wz[b];
#pragma unroll
        for (int a = 0; a < 4; ++a) W[b * 4 + a] = fmaf(cb, wx[a], kRound);
    }
    add_stencil(acci + gb.x + j1 * gb.y + i1, gb.y, W);
}

template <int WARPS, bool DUAL>
__global__ void __launch_bounds__(WARPS * 32) ray_adjoint_kernel(AfGeom g, RayGrid rg,
                                                                 const float4 *__restrict__ elem,
                                                                 const float2 *__restrict__ pix,
                                                                 const float *__restrict__ phi,
                                                                 const float *__restrict__ gdel,
                                                                 AfScal *__restrict__ scal,
                                                                 long long *__restrict__ gpad)
{
    constexpr int T = WARPS * 32;                    // threads = items per block
    constexpr int kQueue = 96;                       // < 32 carried + 2 x 32 new
    extern __shared__ int acci[];
    __shared__ float4 rays[kRayGroup * T];           // (gx0, gz0, gdx, gdz), ray m of item r at m * T + r
    __shared__ float rayc[kRayGroup * T];            // dL/dT |q - r| / (N + 1), scaled, ray m at m * T + r
    __shared__ int rayb[T];                          // grid copy of the item (1: copy B)
    __shared__ int fq[WARPS][kQueue];                // queued points
    __shared__ int wcount[WARPS];
    __shared__ float wbound[WARPS];
    __shared__ long s_blk;
    const int P = g.pitch;
    const int nacc = DUAL ? rg.base_b + rg.pb * rg.rows : rg.pa * rg.rows;
    for (int k = threadIdx.x; k < nacc; k += T) acci[k] = 0;      // shared memory only: before the wait
    pdl_wait();
    const float gmax = __int_as_float(scal->gmax_bits);
    const float S = gmax > 0.0f ? g.fix_scale / gmax : 0.0f;
    const float inv_gmax = gmax > 0.0f ? 1.0f / gmax : 0.0f;
    // adds the integer grids into the global one (integer adds no thread waits for,
    // exact in any order) and clears them; called by every thread of the CTA
    auto flush_grid = [&]() {
        for (int q = threadIdx.x; q < rg.width * rg.rows; q += T) {
            const int j = q / rg.width, i = q - j * rg.width;
            int v = acci[j * rg.pa + i];
            acci[j * rg.pa + i] = 0;
            if (DUAL) {
                v += acci[rg.base_b + j * rg.pb + i];
                acci[rg.base_b + j * rg.pb + i] = 0;
            }
            if (v != 0) atomicAdd(reinterpret_cast<unsigned long long *>(gpad + j * P + i),
                                  (unsigned long long)(long long)v);
        }
        __syncthreads();
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npts = g.nseg + 1;
    const int ngroups = (g.npix + kRayGroup - 1) / kRayGroup;
    const long nitems = (long)g.ne * ngroups;
    // blocks of T items, then quarter blocks for the last gridDim.x * T items, so
    // that the CTAs run out of work within a quarter block of each other (whole
    // blocks of ~50 us left SMs idle for up to one block: 0.750 -> 0.734 ms;
    // eighth blocks 0.738, quarter blocks over two rounds 0.741)
    constexpr int TQ = T / 4;
    static_assert(T * kRayGroup * (1.0f + kRayRoundShare) <= kRayFlushBudget,
                  "a single block must fit in the flush budget");
    long nfull = (nitems - (long)gridDim.x * T) / T;
    if (nfull < 0) nfull = 0;
    const long nblk = S > 0.0f ? nfull + (nitems - nfull * T + TQ - 1) / TQ : 0;
    auto bstart = [&](long b) { return b < nfull ? b * T : nfull * T + (b - nfull) * TQ; };
    auto bsize = [&](long b) { return b < nfull ? T : TQ; };
    if (threadIdx.x == 0) s_blk = atomicAdd(&scal->ray_next, 1);
    __syncthreads();
    long blk = s_blk;
    float since_bound = 0.0f;                        // magnitude bound of the rays since the last flush
    // the inputs of this thread's item (dL/dT, exit angle or exit x, pixel), loaded
    // one block ahead: the next block's are in flight while this one is scattered
    float in_gv[kRayGroup], in_ph[kRayGroup];
    float2 in_px[kRayGroup];
    auto load_inputs = [&](long b) {
        const long it = bstart(b) + threadIdx.x;
        const bool ok = b < nblk && threadIdx.x < bsize(b) && it < nitems;
        const int e = ok ? (int)(it / ngroups) : 0, grp = ok ? (int)(it - (long)e * ngroups) : 0;
#pragma unroll
        for (int m = 0; m < kRayGroup; ++m) {
            const int p = grp * kRayGroup + m;
            const bool on = ok && p < g.npix;
            const long idx = (long)e * g.npix + p;
            in_gv[m] = on ? gdel[idx] : 0.0f;
            in_ph[m] = on && g.lens_mode != AF_LENS_NONE ? phi[idx] : 0.0f;
            in_px[m] = on ? pix[p] : make_float2(0.0f, 0.0f);
        }
    };
    load_inputs(blk);
    while (blk < nblk) {
        // the next block's index, claimed now and needed only after the table fill
        long nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(&scal->ray_next, 1);
        const long item = bstart(blk) + threadIdx.x;
        const int cur_size = bsize(blk);
        float c[kRayGroup];
        float4 rp[kRayGroup];
        bool any = false;
        float ub = 0.0f;                             // this thread's rays, in rays of the largest |dL/dT|
#pragma unroll
        for (int m = 0; m < kRayGroup; ++m) {
            c[m] = 0.0f;
            rp[m] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (threadIdx.x < cur_size && item < nitems) {
            const int e = (int)(item / ngroups);
#pragma unroll
            for (int m = 0; m < kRayGroup; ++m) {
                const float gv = in_gv[m];
                if (gv == 0.0f) continue;
                const float2 px = in_px[m];
                float qx, qz;
                if (g.lens_mode == AF_LENS_BENT_RAY) {
                    float sn, cs;
                    sincosf(in_ph[m], &sn, &cs);
                    qx = fmaf(g.RL, sn, g.arc_cx);
                    qz = fmaf(g.RL, cs, g.arc_cz);
                } else if (g.lens_mode == AF_LENS_PLANAR) {
                    qx = in_ph[m];          // exit x on the lens line
                    qz = g.lens_z;
                } else {
                    const float4 el = elem[e];
                    qx = el.x;
                    qz = el.y;
                }
                const float lx = px.x - qx, lz = px.y - qz;
                c[m] = gv * S * sqrtf(lx * lx + lz * lz) * g.inv_nseg1;
                rp[m] = make_float4((qx - g.x0) * g.inv_dx, (qz - g.z0) * g.inv_dz,
                                    lx * g.inv_dx * g.inv_nseg, lz * g.inv_dz * g.inv_nseg);
                any = any || c[m] != 0.0f;
                if (c[m] != 0.0f) ub += fabsf(gv) * inv_gmax + kRayRoundShare;
            }
        }
        // CTA-wide compaction of the live items
        const unsigned live = __ballot_sync(0xffffffffu, any);
        for (int o = 16; o > 0; o >>= 1) ub += __shfl_xor_sync(0xffffffffu, ub, o);
        if (lane == 0) {
            wcount[warp] = __popc(live);
            wbound[warp] = ub;
        }
        __syncthreads();
        int base = 0, nlive = 0;
        float bb = 0.0f;                             // the block's bound, the same in every thread
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const int n = wcount[w];
            base += w < warp ? n : 0;
            nlive += n;
            bb += wbound[w];
        }
        if (any) {
            const int slot = base + __popc(live & ((1u << lane) - 1u));
            // path of the lead: the middle ray if live, else the first live one
            float4 rl = rp[kLeadRay];
            if (c[kLeadRay] == 0.0f) {
#pragma unroll
                for (int m = kRayGroup - 1; m >= 0; --m)
                    if (c[m] != 0.0f) rl = rp[m];
            }
            // dead rays take the lead's path (weight 0), so they always merge
#pragma unroll
            for (int m = 0; m < kRayGroup; ++m) rays[m * T + slot] = c[m] != 0.0f ? rp[m] : rl;
#pragma unroll
            for (int m = 0; m < kRayGroup; ++m) rayc[m * T + slot] = c[m];
            const bool right_down = rl.z * rl.w >= 0.0f;
            rayb[slot] = DUAL && !right_down ? 1 : 0;
        }
        if (threadIdx.x == 0) s_blk = nxt;
        __syncthreads();
        load_inputs(s_blk);                          // the next block's, in flight during the scatter
        if (since_bound + bb > g.ray_flush_budget) { // this block could overflow the integer grids
            flush_grid();
            since_bound = 0.0f;
        }
        since_bound += bb;
        const int npt_total = nlive * npts;
        int nq = 0;                                  // queued points of this warp (warp-uniform)
        // flat index q = r * npts + k of this lane, advanced by T per pass without division
        int r = (warp * 32 + lane) / npts, k = (warp * 32 + lane) - r * npts;
        const int dr = T / npts, dk = T - dr * npts;
        for (int q0 = warp * 32; q0 < npt_total; q0 += T) {
            bool apart[kRayGroup];
#pragma unroll
            for (int m = 0; m < kRayGroup; ++m) apart[m] = false;
            if (q0 + lane < npt_total) {
                const float kf = (float)k;
                const int2 gb = copy_of<DUAL>(rg, rayb[r]);
                float W[16], fx0, fz0;
                int i0, j0;
                {
                    float wx[4], wz[4];
                    ray_stencil(g, kf, rays[kLeadRay * T + r], i0, j0, fx0, fz0, wx, wz);
                    // rank-1 stencil rows on the packed FP32 pipe: one paired FMA is two
                    // round-to-nearest FMAs, so W is the same as with scalar fmaf
                    const float cl = rayc[kLeadRay * T + r];
                    const float2 x01 = make_float2(wx[0], wx[1]), x23 = make_float2(wx[2], wx[3]);
                    const float2 kR = make_float2(kRound, kRound);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float cb = cl * wz[b];
                        const float2 c2 = make_float2(cb, cb);
                        const float2 lo = __ffma2_rn(c2, x01, kR), hi = __ffma2_rn(c2, x23, kR);
                        W[b * 4 + 0] = lo.x; W[b * 4 + 1] = lo.y; W[b * 4 + 2] = hi.x; W[b * 4 + 3] = hi.y;
                    }
                }
#pragma unroll
                for (int m = 0; m < kRayGroup; ++m) {
                    if (m == kLeadRay) continue;
                    // the point shares the lead's cell when its coordinates have the
                    // lead's floors; its fractions are then exactly its own
                    const float4 rm = rays[m * T + r];
                    const float tx = fmaf(kf, rm.z, rm.x) - fx0, tz = fmaf(kf, rm.w, rm.y) - fz0;
                    float wx[4], wz[4];
                    keys_weights(tx, wx);
                    keys_weights(tz, wz);
                    const float cm = rayc[m * T + r];
                    const bool away = !(unit_fraction(tx) && unit_fraction(tz));
                    const float cmerge = away ? 0.0f : cm;
                    const float2 x01 = make_float2(wx[0], wx[1]), x23 = make_float2(wx[2], wx[3]);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float cb = cmerge * wz[b];
                        const float2 c2 = make_float2(cb, cb);
                        const float2 lo = __ffma2_rn(c2, x01, make_float2(W[b * 4 + 0], W[b * 4 + 1]));
                        const float2 hi = __ffma2_rn(c2, x23, make_float2(W[b * 4 + 2], W[b * 4 + 3]));
                        W[b * 4 + 0] = lo.x; W[b * 4 + 1] = lo.y; W[b * 4 + 2] = hi.x; W[b * 4 + 3] = hi.y;
                    }
                    apart[m] = away && cm != 0.0f;
                }
                add_stencil(acci + gb.x + j0 * gb.y + i0, gb.y, W);
            }
            // queue the points that left the lead's cell; run full batches of 32
#pragma unroll
            for (int m = 0; m < kRayGroup; ++m) {
                if (m == kLeadRay) continue;
                const unsigned am = __ballot_sync(0xffffffffu, apart[m]);
                if (apart[m]) fq[warp][nq + __popc(am & ((1u << lane) - 1u))] = (r << 18) | (k << 2) | m;
                nq += __popc(am);
            }
            __syncwarp();
            while (nq >= 32) {
                nq -= 32;
                const int ent = fq[warp][nq + lane];
                __syncwarp();
                run_queued<DUAL>(g, rg, ent, acci, rays, T, rayc, rayb);
            }
            r += dr;
            k += dk;
            if (k >= npts) { k -= npts; ++r; }
        }
        if (lane < nq) run_queued<DUAL>(g, rg, fq[warp][lane], acci, rays, T, rayc, rayb);   // last partial batch
        blk = s_blk;
        __syncthreads();                             // table and queue free for the next block
        if (blk >= nblk) flush_grid();
    }
}

__device__ __forceinline__ float dz_sign(float x, float k)      // D_k'(x)
{
    return fabsf(x) <= k ? 0.0f : (x > 0.0f ? 1.0f : -1.0f);
}

// grad[k] = (folded integer grid)[k] / S + d(w1 R_TV + w2 R_SV)/ds_k  (gather form on
// c = 1 / (c_unit s), the speed in the units of Eq. 10-11);
// also returns the ray adjoint's block counter to zero for its next launch
__global__ void __launch_bounds__(256) reduce_grad_kernel(AfGeom g, const float *__restrict__ s,
                                                          long long *__restrict__ gpad, int have_rays,
                                                          AfScal *scal, float *__restrict__ grad)
{
    pdl_wait();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) scal->ray_next = 0;
    if (k >= g.ng) return;
    const int j = k / g.nx, i = k - j * g.nx, nx = g.nx, nz = g.nz;
    // fold the padding of the integer grid onto the clamped edge nodes; every padded
    // cell belongs to exactly one node, whose thread also returns it to zero for the
    // next launch of the ray adjoint
    long long tot = 0;
    if (have_rays) {
        const int P = g.pitch;
        const int ilo = i == 0 ? 0 : i + 2, ihi = i == nx - 1 ? nx + 3 : i + 2;
        const int jlo = j == 0 ? 0 : j + 2, jhi = j == nz - 1 ? nz + 3 : j + 2;
        for (int jj = jlo; jj <= jhi; ++jj)
            for (int ii = ilo; ii <= ihi; ++ii) {
                tot += gpad[jj * P + ii];
                gpad[jj * P + ii] = 0;
            }
    }
    const float gmax = __int_as_float(scal->gmax_bits);
    const float acc = gmax > 0.0f ? (float)((double)tot * ((double)gmax / (double)g.fix_scale)) : 0.0f;
    auto C = [&](int ii, int jj) { return g.inv_c_unit / s[jj * nx + ii]; };
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
    grad[k] = acc - dc * (c0 * c0 * g.c_unit);     // dc/ds = -c_unit c^2
}

// Eq. 9 on the sound speed c = 1 / (c_unit s) (km/s): the plain gradient step as
// printed (AF_OPT_GD) or with Adam moments; dL/dc = dL/ds ds/dc, ds/dc = -c_unit s^2
__global__ void __launch_bounds__(256) adam_kernel(AfGeom g, const float *__restrict__ grad,
                                                   float *__restrict__ s, float *__restrict__ m,
                                                   float *__restrict__ v, float bc1, float bc2)
{
    pdl_wait();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ng) return;
    const float sk = s[k];
    const float gc = -grad[k] * (g.c_unit * sk * sk);
    if (g.optimizer == AF_OPT_GD) {
        s[k] = g.inv_c_unit / (g.inv_c_unit / sk - g.lr * gc);
        return;
    }
    const float mk = fmaf(g.beta1, m[k], g.omb1 * gc);
    const float vk = fmaf(g.beta2, v[k], g.omb2 * gc * gc);
    m[k] = mk;
    v[k] = vk;
    const float c = g.inv_c_unit / sk - g.lr * (mk / bc1) / (sqrtf(vk / bc2) + g.eps);
    s[k] = g.inv_c_unit / c;
}

}  // namespace

// copy A pitch = 1 (mod 32), copy B pitch = 31 (mod 32), both >= nx + 4
static RayGrid ray_grid_layout(int nx, int nz, bool dual, int pitch)
{
    RayGrid rg;
    rg.width = nx + 4;
    rg.rows = nz + 4;
    if (dual) {
        rg.pa = ((rg.width - 1 + 31) / 32) * 32 + 1;
        rg.pb = ((rg.width + 1 + 31) / 32) * 32 - 1;
        rg.base_b = rg.pa * rg.rows;
    } else {
        rg.pa = rg.pb = pitch;
        rg.base_b = 0;
    }
    return rg;
}

static size_t ray_grid_bytes(const RayGrid &rg, bool dual)
{
    return (size_t)(dual ? rg.base_b + rg.pb * rg.rows : rg.pa * rg.rows) * sizeof(int);
}

// ray-adjoint launch shape of a plan: the two-copy layout when it fits in
// shared memory, one CTA per SM, with 24 warps when the CTA's item tables fit
// beside the two copies (more warps hide the shared-memory atomics: 0.80 ms
// against 0.83 ms with 16 warps on a 128 x 128 grid), else 16 warps; otherwise
// one odd-pitch copy (8 warps)
RayAdjShape rayadj_shape(int nx, int nz, int pitch, int sm_count)
{
    RayAdjShape sh;
    const RayGrid dual = ray_grid_layout(nx, nz, true, pitch);
    sh.dual = ray_grid_bytes(dual, true) <= kRayDualMaxBytes;
    const RayGrid rg = ray_grid_layout(nx, nz, sh.dual, pitch);
    sh.smem = ray_grid_bytes(rg, sh.dual);
    sh.threads = sh.dual ? 512 : 256;
    int n = 0;
    if (sh.dual) {
        int dev = 0, optin = 0;
        cudaFuncAttributes a24{};
        const bool known = cudaGetDevice(&dev) == cudaSuccess &&
                           cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) ==
                               cudaSuccess &&
                           cudaFuncGetAttributes(&a24, ray_adjoint_kernel<24, true>) == cudaSuccess;
        // 1 KB kept free for the per-CTA reservation
        if (known && a24.sharedSizeBytes + sh.smem + 1024 <= (size_t)optin &&
            cudaFuncSetAttribute(ray_adjoint_kernel<24, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)a24.sharedSizeBytes - 1024) == cudaSuccess) {
            sh.threads = 768;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ray_adjoint_kernel<24, true>, 768, sh.smem);
        } else {
            cudaGetLastError();
            cudaFuncSetAttribute(ray_adjoint_kernel<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRayDualMaxBytes);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ray_adjoint_kernel<16, true>, 512, sh.smem);
        }
    } else {
        // the attribute is per function, shared by every plan: set it to the largest
        // grid any plan may use, the occupancy query uses this plan's size
        cudaFuncSetAttribute(ray_adjoint_kernel<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMaxGridSmemBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ray_adjoint_kernel<8, false>, 256, sh.smem);
    }
    sh.blocks = sm_count * (n > 0 ? n : 1);
    return sh;
}

cudaError_t launch_ray_adjoint(af_plan_t pl, const float *s, float *grad)
{
    int have_rays = 0;
    if ((long)pl->g.ne * pl->g.npix > 0) {
        const RayAdjShape &sh = pl->rayadj;
        const RayGrid rg = ray_grid_layout(pl->g.nx, pl->g.nz, sh.dual, pl->g.pitch);
        auto kernel = sh.dual && sh.threads == 768 ? ray_adjoint_kernel<24, true>
                      : sh.dual                    ? ray_adjoint_kernel<16, true>
                                                   : ray_adjoint_kernel<8, false>;
        const int threads = sh.dual && sh.threads == 768 ? 768 : sh.dual ? 512 : 256;
        const cudaError_t e = launch_dependent(kernel, dim3(sh.blocks), dim3(threads), sh.smem, pl->stream, pl->g, rg,
                                               pl->elem, pl->pix, pl->phi, pl->gdel, pl->scal, pl->gpad);
        if (e != cudaSuccess) return e;
        have_rays = 1;
    }
    return launch_dependent(reduce_grad_kernel, dim3((pl->g.ng + 255) / 256), dim3(256), 0, pl->stream, pl->g, s,
                            pl->gpad, have_rays, pl->scal, grad);
}

cudaError_t launch_adam(af_plan_t pl, const float *grad, float *s, float *m, float *v, int step)
{
    const double bc1 = 1.0 - pow((double)pl->g.beta1, step);
    const double bc2 = 1.0 - pow((double)pl->g.beta2, step);
    return launch_dependent(adam_kernel, dim3((pl->g.ng + 255) / 256), dim3(256), 0, pl->stream, pl->g, grad, s, m, v,
                            (float)bc1, (float)bc2);
}
