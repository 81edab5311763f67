// Subaperture delay-and-sum (Eq. 5) and its adjoint with respect to the
// one-way delays (Fig. 1g).  Delays are generated inside the gather from the
// one-way tables (tau = T_t + T_r + t_ttp, never materialised per pair).
//
// A lane owns a pixel and one receive block j; the receive-side delays and
// phasors of block j live in registers, the transmit side is re-read per
// transmit.  Phase rotation is separable:
//   exp(j 2 pi fd tau) = P_t P_r,  P_e = exp(j 2 pi fd (T_e + t_ttp / 2)).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "af_cmpe.cuh"
#include "af_internal.cuh"

namespace {

template <int DT> struct Sample;
template <> struct Sample<AF_IQ_C64> {
    using T = float2;
    static __device__ __forceinline__ float2 load(const T *p) { return __ldg(p); }
};
template <> struct Sample<AF_IQ_BF16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ float2 load(const T *p) { return __bfloat1622float2(__ldg(p)); }
};
template <> struct Sample<AF_IQ_F16> {
    using T = __half2;
    static __device__ __forceinline__ float2 load(const T *p) { return __half22float2(__ldg(p)); }
};

// The adjoint's CTAs hold 4 warps: a warp whose transmit blocks all have a zero
// image gradient finishes at once, and a small CTA hands its slot on sooner
// (0.30 ms against 0.33 ms with 8-warp CTAs, 128 elements).  Five CTAs per SM
// (96 registers, no spill) against four (128 registers): 0.397 against 0.400 ms
// for complex64, 0.378 against 0.410 for bf16, 0.364 against 0.406 for f16;
// six or eight per SM spill and run slower (0.415, 0.421 ms for complex64).
constexpr int kAdjWarps = 4;
constexpr int kAdjMinBlocks = 5;
// Unroll of the adjoint's transmit loop: 4 for complex64 (0.361 -> 0.346 ms), 2 for
// 16-bit samples (4 measured bf16 0.361 -> 0.370, f16 0.347 -> 0.354; a full unroll
// of 8 was slower for all three), same registers (96) and no spill.
template <int DT> struct AdjUnroll { static constexpr int k = DT == AF_IQ_C64 ? 4 : 2; };

// Forward launch: warps per CTA, CTAs per SM and transmit-loop unroll, the same
// for every sample type.  Measured on the 128-element workload (forward ms):
//   complex64: 8-warp CTAs, 2 per SM, unroll 2: 0.64; 4 per SM, none: 0.61;
//              4-warp CTAs, 8 per SM, none: 0.59; 7 per SM: 0.98; 6 per SM: 0.66
//   bf16:      4-warp CTAs, 6 per SM, none: 0.61; 7 per SM: 0.80; 8 per SM: 0.54
//   f16:       4-warp CTAs, 4 per SM, unroll 2: 0.55; 8 per SM, unroll 2: 0.90;
//              8 per SM, none: 0.51
// At 8 CTAs per SM (64 registers) the compiler spills a few bytes; every
// shape that fits without spilling runs slower.  With the transmit pieces
// below, 8-warp CTAs (4 per SM) measured 0.544 ms against 0.523, and an unroll
// of 2 or 4 0.80-0.86 ms for all three sample types.
template <int DT> struct FwdLaunch { static constexpr int kWarps = 4, kMinBlocks = 8, kUnroll = 1; };

// Each (pixel tile, receive block) is split into pieces of consecutive transmit
// blocks, one CTA per piece; grid.y = piece * nsub + j, so all CTAs of one piece
// are issued before the next piece's.  Whole tiles made CTAs of ~150 us that ran
// in 3.4 waves of 1184 resident CTAs; the last wave left SMs part-empty for
// ~150 us.  Shorter CTAs shorten that tail, and more CTAs cost more issue
// overhead (128 elements, ms): forward 0.590 whole, 0.534 in 2 pieces, 0.523 in
// 4, 0.538 in 8; adjoint 0.395, 0.367, 0.386, 0.441.  Pieces are independent:
// each writes its own B_ij, and the adjoint adds into dL/dT atomically anyway.
constexpr int kFwdSplit = 4, kAdjSplit = 2;

// Gather of one transmit for the W receivers held by a lane: all 2W loads are
// issued before any is used, so a warp keeps 2W loads in flight.  CHECK: the
// indices are clamped into the trace and out-of-range samples get weight 0;
// without CHECK the caller has shown that every sample n, n + 1 of the W
// receivers lies in the trace.
template <int W, typename S, bool CHECK>
__device__ __forceinline__ void gather_w(const typename S::T *__restrict__ base, int ns, int nt,
                                         float ft, const int (&nr)[W], const float (&fr)[W],
                                         float2 (&a)[W], float2 (&b)[W], float (&f)[W], float (&on)[W])
{
    const int lim = ns - 1;
    int idx[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
        int n = nt + nr[k];
        float fk = ft + fr[k];
        if (fk >= 1.0f) { fk -= 1.0f; ++n; }
        f[k] = fk;
        if (CHECK) {
            const bool valid = (unsigned)n < (unsigned)lim;
            idx[k] = k * ns + (valid ? n : 0);
            on[k] = valid ? 1.0f : 0.0f;
        } else {
            idx[k] = k * ns + n;
            on[k] = 1.0f;
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
        a[k] = S::load(base + idx[k]);
        b[k] = S::load(base + idx[k] + 1);
    }
}

// Receive side of a lane (block j, pixel p) in registers.  A receiver outside
// the aperture gets phasor 0 and the sample index of a live receiver of the
// block, so it adds exactly nothing and its samples lie where the live ones
// do.  Returns the mask of live receivers (bit k: receiver j W + k), 0 when
// the whole block is outside the aperture.
template <int W>
__device__ __forceinline__ unsigned receive_side(const float4 *__restrict__ D, int npix, int j, int p,
                                                 int (&nr)[W], float (&fr)[W], float2 (&pr)[W])
{
    int live = 0;
    unsigned mask = 0u;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const float4 d = D[(long)(j * W + k) * npix + p];
        nr[k] = __float_as_int(d.x);
        fr[k] = d.y;
        pr[k] = make_float2(d.z, d.w);
        if (nr[k] != AF_APOD_OFF) { live = nr[k]; mask |= 1u << k; }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
        if (nr[k] == AF_APOD_OFF) {
            nr[k] = live;
            fr[k] = 0.0f;
            pr[k] = make_float2(0.0f, 0.0f);
        }
    }
    return mask;
}

// Every gather of pixel p reads samples n and n + 1 with n = n_t + n_r + carry
// <= 2 max n + 1, n >= 2 min n, where r = {min n, -max n} over the pixel's live
// one-way indices (written by the delay kernel).  True when all of them lie in
// [0, ns - 1], so that the gathers need no range check.
__device__ __forceinline__ bool pixel_in_trace(int2 r, int ns)
{
    return r.x >= 0 && 2LL * -(long long)r.y <= (long long)ns - 3;
}

template <int W, typename S, bool CHECK>
__device__ __forceinline__ float2 das_transmit(const typename S::T *__restrict__ base, int ns, int nt, float ft,
                                               const int (&nr)[W], const float (&fr)[W], const float2 (&pr)[W])
{
    float2 a[W], b[W];
    float f[W], on[W];
    gather_w<W, S, CHECK>(base, ns, nt, ft, nr, fr, a, b, f, on);
    float sr = 0.0f, si = 0.0f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        float vr = fmaf(f[k], b[k].x - a[k].x, a[k].x);
        float vi = fmaf(f[k], b[k].y - a[k].y, a[k].y);
        if (CHECK) { vr *= on[k]; vi *= on[k]; }
        sr = fmaf(pr[k].x, vr, fmaf(-pr[k].y, vi, sr));
        si = fmaf(pr[k].x, vi, fmaf(pr[k].y, vr, si));
    }
    return make_float2(sr, si);
}

// B_ij(p) for the transmit blocks i0 <= i < i1 of one lane (receive block j)
template <int W, int DT, bool CHECK>
__device__ __forceinline__ void das_forward_blocks(const AfGeom &g, const typename Sample<DT>::T *__restrict__ psi,
                                                   const float *__restrict__ scale, const float4 *__restrict__ D,
                                                   float2 *__restrict__ B, int j, int p, const int (&nr)[W],
                                                   const float (&fr)[W], const float2 (&pr)[W], int i0, int i1)
{
    using S = Sample<DT>;
    float4 dnext = D[(long)i0 * W * g.npix + p];
    for (int i = i0; i < i1; ++i) {
        float ar = 0.0f, ai = 0.0f;
#pragma unroll(FwdLaunch<DT>::kUnroll)
        for (int tt = 0; tt < W; ++tt) {
            const int t = i * W + tt;
            const float4 dt = dnext;
            if (t + 1 < g.ne) dnext = D[(long)(t + 1) * g.npix + p];
            const int nt = __float_as_int(dt.x);
            if (nt == AF_APOD_OFF) continue;
            const typename S::T *base = psi + ((long)t * g.ne + j * W) * g.ns;
            const float2 sv = das_transmit<W, S, CHECK>(base, g.ns, nt, dt.y, nr, fr, pr);
            float cr = dt.z, ci = dt.w;
            if (DT != AF_IQ_C64) { const float sc = scale[t]; cr *= sc; ci *= sc; }
            ar = fmaf(cr, sv.x, fmaf(-ci, sv.y, ar));
            ai = fmaf(cr, sv.y, fmaf(ci, sv.x, ai));
        }
        B[(long)(i * g.nsub + j) * g.npix + p] = make_float2(ar, ai);
    }
}

// Forward: CTA = 4 warps on as many neighbouring tiles of 32 pixels (128
// consecutive pixels, one or two laterally adjacent patches), all with the same
// receive block j and the same piece of transmit blocks (blockIdx.y).  The warps
// walk the transmits in the same order, so the trace windows one warp pulls into
// L1 serve the others.
// The gathers are latency bound; the CTA size, the CTAs per SM and the unroll
// of the transmit loop are chosen per sample type (FwdLaunch).
// A warp whose receive block is outside the aperture for all its pixels only
// writes zeros; a warp whose pixels' samples all lie in the trace runs the
// gathers without range checks.
template <int W, int DT>
__global__ void __launch_bounds__(32 * FwdLaunch<DT>::kWarps, FwdLaunch<DT>::kMinBlocks)
    das_forward_kernel(AfGeom g, const void *__restrict__ iq,
                                                             const float *__restrict__ scale,
                                                             const float4 *__restrict__ D,
                                                             const int2 *__restrict__ nrange,
                                                             float2 *__restrict__ B)
{
    pdl_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = (blockIdx.x * FwdLaunch<DT>::kWarps + warp) * 32 + lane;
    const int j = blockIdx.y % g.nsub, piece = blockIdx.y / g.nsub;
    const int i0 = piece * g.nsub / kFwdSplit, i1 = (piece + 1) * g.nsub / kFwdSplit;   // transmit blocks
    if (p >= g.npix) return;
    const typename Sample<DT>::T *psi = reinterpret_cast<const typename Sample<DT>::T *>(iq);
    int nr[W];
    float fr[W];
    float2 pr[W];
    const bool live = receive_side<W>(D, g.npix, j, p, nr, fr, pr) != 0u;
    const unsigned act = __activemask();
    if (!__any_sync(act, live)) {
        for (int i = i0; i < i1; ++i) B[(long)(i * g.nsub + j) * g.npix + p] = make_float2(0.0f, 0.0f);
        return;
    }
    if (__all_sync(act, pixel_in_trace(nrange[p], g.ns)))
        das_forward_blocks<W, DT, false>(g, psi, scale, D, B, j, p, nr, fr, pr, i0, i1);
    else
        das_forward_blocks<W, DT, true>(g, psi, scale, D, B, j, p, nr, fr, pr, i0, i1);
}

// Adjoint: CTAs of kAdjWarps neighbouring pixel tiles with one receive block j
// and one piece of transmit blocks (blockIdx.y).  For one gather dL/dtau =
// Re(conj(G) exp(j 2 pi fd tau) (fs dPsi/du + j 2 pi fd Psi(u))); it is added to
// dL/dT_t and dL/dT_r.  A lane sums the transmit role over its block's W
// receivers and the receive role over the piece's transmits, then adds both into
// the zeroed dL/dT table with coalesced atomic adds (one per transmit and one per
// live receiver of the block).
template <int W, typename S, bool CHECK>
__device__ __forceinline__ float adj_transmit(const AfGeom &g, const typename S::T *__restrict__ base, int nt,
                                              float ft, float xr, float xi, const int (&nr)[W],
                                              const float (&fr)[W], const float2 (&pr)[W], float (&gr)[W])
{
    float2 a[W], b[W];
    float f[W], on[W];
    gather_w<W, S, CHECK>(base, g.ns, nt, ft, nr, fr, a, b, f, on);
    float gt = 0.0f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const float sx = b[k].x - a[k].x, sy = b[k].y - a[k].y;
        const float vr = fmaf(f[k], sx, a[k].x), vi = fmaf(f[k], sy, a[k].y);
        float yr = fmaf(xr, pr[k].x, -xi * pr[k].y);
        float yi = fmaf(xr, pr[k].y, xi * pr[k].x);
        if (CHECK) { yr *= on[k]; yi *= on[k]; }
        const float dr = fmaf(g.fs, sx, -g.wd * vi);
        const float di = fmaf(g.fs, sy, g.wd * vr);
        const float q = fmaf(yr, dr, -yi * di);
        gt += q;
        gr[k] += q;
    }
    return gt;
}

template <int W, int DT, bool CHECK>
__device__ __forceinline__ void das_adjoint_blocks(const AfGeom &g, const typename Sample<DT>::T *__restrict__ psi,
                                                   const float *__restrict__ scale, const float4 *__restrict__ D,
                                                   const float2 *__restrict__ B, const float2 *__restrict__ z,
                                                   const uint8_t *__restrict__ mask, float inv_m,
                                                   float *__restrict__ gdel, int j,
                                                   int p, bool live, const int (&nr)[W], const float (&fr)[W],
                                                   const float2 (&pr)[W], float (&gr)[W], int i0, int i1)
{
    using S = Sample<DT>;
    float4 dnext = D[(long)i0 * W * g.npix + p];
    for (int i = i0; i < i1; ++i) {
        // dL/dB_ij(p), formed here from the images and the CMPE terms (never stored)
        const float2 Gv = cmpe::image_grad(B, z, mask, inv_m, g.nsub, g.npix, g.npair, p / g.patch_npix, i, j, p);
        // every term of transmit block i is weighted by conj(G_ij(p)): where the CMPE
        // mask leaves G_ij(p) = 0 the block adds exactly nothing, so it is skipped
        // (by the whole warp when no lane has a gradient, else lane by lane)
        const bool gzero = (Gv.x == 0.0f && Gv.y == 0.0f) || !live;
        if (__all_sync(__activemask(), gzero)) {
            if ((i + 1) * W < g.ne) dnext = D[(long)(i + 1) * W * g.npix + p];
            continue;
        }
#pragma unroll(AdjUnroll<DT>::k)
        for (int tt = 0; tt < W; ++tt) {
            const int t = i * W + tt;
            const float4 dt = dnext;
            if (t + 1 < g.ne) dnext = D[(long)(t + 1) * g.npix + p];
            const int nt = __float_as_int(dt.x);
            if (nt == AF_APOD_OFF || gzero) continue;
            float sc = 1.0f;
            if (DT != AF_IQ_C64) sc = scale[t];
            // X = conj(G) P_t (scaled)
            const float xr = sc * fmaf(Gv.x, dt.z, Gv.y * dt.w);
            const float xi = sc * fmaf(Gv.x, dt.w, -Gv.y * dt.z);
            const typename S::T *base = psi + ((long)t * g.ne + j * W) * g.ns;
            const float gt = adj_transmit<W, S, CHECK>(g, base, nt, dt.y, xr, xi, nr, fr, pr, gr);
            atomicAdd(&gdel[(long)t * g.npix + p], gt);
        }
    }
}

template <int W, int DT>
__global__ void __launch_bounds__(32 * kAdjWarps, kAdjMinBlocks) das_adjoint_kernel(AfGeom g, const void *__restrict__ iq,
                                                             const float *__restrict__ scale,
                                                             const float4 *__restrict__ D,
                                                             const int2 *__restrict__ nrange,
                                                             const float2 *__restrict__ B,
                                                             const float2 *__restrict__ z,
                                                             const uint8_t *__restrict__ mask,
                                                             const AfScal *__restrict__ scal,
                                                             float *__restrict__ gdel)
{
    pdl_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = (blockIdx.x * kAdjWarps + warp) * 32 + lane;
    const int j = blockIdx.y % g.nsub, piece = blockIdx.y / g.nsub;
    const int i0 = piece * g.nsub / kAdjSplit, i1 = (piece + 1) * g.nsub / kAdjSplit;   // transmit blocks
    if (p >= g.npix) return;
    const typename Sample<DT>::T *psi = reinterpret_cast<const typename Sample<DT>::T *>(iq);
    int nr[W];
    float fr[W];
    float2 pr[W];
    float gr[W];
    const unsigned rmask = receive_side<W>(D, g.npix, j, p, nr, fr, pr);
    const bool live = rmask != 0u;
    const unsigned act = __activemask();
    if (!__any_sync(act, live)) return;        // adds nothing
    const float inv_m = scal->inv_m;
#pragma unroll
    for (int k = 0; k < W; ++k) gr[k] = 0.0f;
    if (__all_sync(act, pixel_in_trace(nrange[p], g.ns)))
        das_adjoint_blocks<W, DT, false>(g, psi, scale, D, B, z, mask, inv_m, gdel, j, p, live, nr, fr, pr, gr, i0, i1);
    else
        das_adjoint_blocks<W, DT, true>(g, psi, scale, D, B, z, mask, inv_m, gdel, j, p, live, nr, fr, pr, gr, i0, i1);
#pragma unroll
    for (int k = 0; k < W; ++k)
        if (rmask >> k & 1u) atomicAdd(&gdel[(long)(j * W + k) * g.npix + p], gr[k]);
}

// zeroes x[0, n) with float4 stores (x is a device allocation, so 16-byte aligned);
// a kernel rather than a memset node, so that the launches before and after it
// stay programmatic (1.5 us per step less than cudaMemsetAsync, 128 elements)
__global__ void __launch_bounds__(256) zero_kernel(float *__restrict__ x, long n)
{
    pdl_wait();
    const long n4 = n >> 2, stride = (long)gridDim.x * blockDim.x, first = (long)blockIdx.x * blockDim.x + threadIdx.x;
    float4 *__restrict__ x4 = reinterpret_cast<float4 *>(x);
    for (long k = first; k < n4; k += stride) x4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long k = (n4 << 2) + first; k < n; k += stride) x[k] = 0.0f;
}

// max |dL/dT| for the fixed-point scale of the ray adjoint (non-negative floats
// order like their bit patterns)
__global__ void __launch_bounds__(256) gdel_max_kernel(const float *__restrict__ gdel, long n,
                                                       int *__restrict__ gmax_bits)
{
    // float4 loads (the table is a device allocation, so 16-byte aligned), then the
    // tail; a maximum does not depend on the order
    pdl_wait();
    float amax = 0.0f;
    const long n4 = n >> 2, stride = (long)gridDim.x * blockDim.x, first = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const float4 *__restrict__ g4 = reinterpret_cast<const float4 *>(gdel);
#pragma unroll 4
    for (long k = first; k < n4; k += stride) {
        const float4 v = g4[k];
        amax = fmaxf(fmaxf(amax, fabsf(v.x)), fmaxf(fmaxf(fabsf(v.y), fabsf(v.z)), fabsf(v.w)));
    }
    for (long k = (n4 << 2) + first; k < n; k += stride) amax = fmaxf(amax, fabsf(gdel[k]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0 && amax > 0.0f) atomicMax(gmax_bits, __float_as_int(amax));
}

template <int W, int DT>
cudaError_t launch_fwd_t(af_plan_t pl)
{
    constexpr int kW = FwdLaunch<DT>::kWarps;
    const dim3 blocks((pl->g.npix + 32 * kW - 1) / (32 * kW), pl->g.nsub * kFwdSplit);
    return launch_dependent(das_forward_kernel<W, DT>, blocks, dim3(32 * kW), 0, pl->stream, pl->g, pl->iq,
                            pl->iq_scale, pl->D, pl->nrange, pl->B);
}

template <int W, int DT>
cudaError_t launch_adj_t(af_plan_t pl)
{
    const long n = (long)pl->g.ne * pl->g.npix;
    // (max|dL/dT| starts from zero: the CMPE forward's fold resets it)
    cudaError_t e = launch_dependent(zero_kernel, dim3(pl->sm_count * 4), dim3(256), 0, pl->stream, pl->gdel, n);
    if (e != cudaSuccess) return e;
    const dim3 blocks((pl->g.npix + 32 * kAdjWarps - 1) / (32 * kAdjWarps), pl->g.nsub * kAdjSplit);
    e = launch_dependent(das_adjoint_kernel<W, DT>, blocks, dim3(32 * kAdjWarps), 0, pl->stream, pl->g, pl->iq,
                         pl->iq_scale, pl->D, pl->nrange, pl->B, pl->z, pl->mask, pl->scal, pl->gdel);
    if (e != cudaSuccess) return e;
    return launch_dependent(gdel_max_kernel, dim3(pl->sm_count * 4), dim3(256), 0, pl->stream, pl->gdel, n,
                            &pl->scal->gmax_bits);
}

template <int DT>
cudaError_t dispatch_w(af_plan_t pl, bool adj)
{
    switch (pl->g.W) {
    case 1: return adj ? launch_adj_t<1, DT>(pl) : launch_fwd_t<1, DT>(pl);
    case 2: return adj ? launch_adj_t<2, DT>(pl) : launch_fwd_t<2, DT>(pl);
    case 4: return adj ? launch_adj_t<4, DT>(pl) : launch_fwd_t<4, DT>(pl);
    case 8: return adj ? launch_adj_t<8, DT>(pl) : launch_fwd_t<8, DT>(pl);
    case 16: return adj ? launch_adj_t<16, DT>(pl) : launch_fwd_t<16, DT>(pl);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch(af_plan_t pl, bool adj)
{
    if (pl->g.npix == 0) return cudaSuccess;
    switch (pl->iq_dtype) {
    case AF_IQ_C64: return dispatch_w<AF_IQ_C64>(pl, adj);
    case AF_IQ_BF16: return dispatch_w<AF_IQ_BF16>(pl, adj);
    case AF_IQ_F16: return dispatch_w<AF_IQ_F16>(pl, adj);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_das_forward(af_plan_t pl) { return dispatch(pl, false); }
cudaError_t launch_das_adjoint(af_plan_t pl) { return dispatch(pl, true); }
