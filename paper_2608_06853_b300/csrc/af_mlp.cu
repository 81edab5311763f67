// Lens-surrogate MLP: a learned stand-in for the Fermat exit-point solve of
// Eq. 8 (Sec. III-A).  Inputs: element angle, pixel radius and pixel angle
// relative to the element (all about the arc centre), and the medium speed
// c_med.  Outputs: the exit-angle offset from the element and the lens transit
// time.  4 layers, 4 -> 128 -> 128 -> 128 -> 2, tanh.
//
// The two 128 x 128 layers run on the tensor cores (tcgen05, bf16 operands,
// f32 accumulation in tensor memory), forward and backward; the 4-wide input
// layer and 2-wide output layer run on the FP32 pipes.  Training samples are
// labelled by the float64 exact solver.  In the delay kernel the surrogate's
// exit angle replaces the Newton solve and both path lengths are still
// computed exactly, so a small angle error changes the delay only at second
// order (Fermat stationarity).  Pairs whose validated delay error exceeds the
// tolerance fall back to the exact solver.
//
// Shared-memory operand tiles are 128 x 128 bf16 in the no-swizzle K-major
// core-matrix layout of af_tc.cuh; the same bytes read as an MN-major tile are
// the transpose, which gives the dW = dZ^T H and dH = dZ W products without
// any data movement.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <random>
#include <vector>

#include "af_internal.cuh"
#include "af_lens.cuh"
#include "af_tc.cuh"

namespace {

constexpr int HID = 128;              // hidden width
constexpr int TILE = 128;             // samples per CTA tile
constexpr int TB = TILE * HID * 2;    // bytes of one bf16 tile
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * 4, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID, OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + 2 * HID;
static_assert(OFF_B4 + 2 == AF_MLP_NPARAM, "parameter layout");

__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x rounded to the nearest bfloat16 (ties to even), on the integer pipes instead
// of a conversion instruction (finite x: the activations are tanh outputs)
__device__ __forceinline__ float round_bf16(float x)
{
    uint32_t u = __float_as_uint(x);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return __uint_as_float(u & 0xFFFF0000u);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ float ld_bf16(const uint8_t *tile, int row, int k)
{
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(tile + tc::kmajor_offset(row, k, HID)));
}

// normalised input features
__device__ __forceinline__ void features(const MlpNorm &n, float th_e, float rho, float th_p, float c, float x[4])
{
    x[0] = (th_e - n.th_c) * n.th_s;
    x[1] = (rho - n.r_c) * n.r_s;
    x[2] = (th_p - th_e) * n.dp_s;
    x[3] = (c - n.c_c) * n.c_s;
}

// copy a row-major bf16 [128][128] weight (out x in) to a K-major tile (rows = out)
__device__ __forceinline__ void stage_weight(uint8_t *dst, const __nv_bfloat16 *W)
{
    for (int u = threadIdx.x; u < HID * HID / 8; u += blockDim.x) {
        const int r = u / (HID / 8), kc = (u % (HID / 8)) * 8;
        *reinterpret_cast<uint4 *>(dst + tc::kmajor_offset(r, kc, HID)) =
            *reinterpret_cast<const uint4 *>(W + r * HID + kc);
    }
}

// D (tensor memory, 128 columns) = A B^T with K = 128; a_mn / b_mn choose the
// K-major (LBO 128, SBO 2048) or MN-major (LBO 2048, SBO 128) view of a tile.
// Issued by one thread; completion is signalled on mbar.
__device__ __forceinline__ void mma_tile(uint32_t tmem, const uint8_t *A, int a_mn, const uint8_t *B, int b_mn,
                                         uint64_t *mbar)
{
    const uint32_t idesc = tc::idesc_bf16_f32(TILE, HID, a_mn, b_mn);
    const uint32_t la = a_mn ? TILE * 16 : 128, sa = a_mn ? 128 : HID * 16;
    const uint32_t lb = b_mn ? TILE * 16 : 128, sb = b_mn ? 128 : HID * 16;
    tc::fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < HID / 16; ++kk) {
        const uint64_t da = tc::smem_desc(tc::smem_addr(A) + kk * 2 * la, la, sa);
        const uint64_t db = tc::smem_desc(tc::smem_addr(B) + kk * 2 * lb, lb, sb);
        tc::mma_bf16(tmem, da, db, idesc, kk > 0 ? 1 : 0);
    }
    tc::mma_commit(mbar);
}

// all threads: make shared writes visible to the tensor core, run one product, wait
__device__ __forceinline__ bool run_mma(uint32_t tmem, const uint8_t *A, int a_mn, const uint8_t *B, int b_mn,
                                        uint64_t *mbar, uint32_t &phase, uint32_t wait_tries)
{
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) mma_tile(tmem, A, a_mn, B, b_mn, mbar);
    const bool ok = tc::mma_wait(mbar, phase, wait_tries);
    phase ^= 1u;
    tc::fence_after_sync();
    return ok;
}

// this thread's 32 columns [c, c + 32) of its tensor-memory row (row = 32 * warp + lane)
__device__ __forceinline__ void row_chunk(uint32_t tmem, int c, float (&v)[32])
{
    const int warp = threadIdx.x >> 5;
    tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
}

// bf16 row write of 32 values at columns [c, c+32) of a K-major tile
__device__ __forceinline__ void store_row32(uint8_t *tile, int row, int c, const float (&v)[32])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 w;
        w.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
        w.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
        w.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
        w.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
        *reinterpret_cast<uint4 *>(tile + tc::kmajor_offset(row, c + 8 * q, HID)) = w;
    }
}

// ---------------------------------------------------------------- training
// One CTA of 128 threads per tile of 128 samples (thread = sample row).
// Writes this CTA's gradient partial of every parameter to gpart[blockIdx.x].
__global__ void __launch_bounds__(128, 1) mlp_train_kernel(const float4 *__restrict__ X, const float2 *__restrict__ Y,
                                                           long first, float inv_batch,
                                                           const float *__restrict__ P,
                                                           const __nv_bfloat16 *__restrict__ W2b,
                                                           const __nv_bfloat16 *__restrict__ W3b,
                                                           float *__restrict__ gpart, float *__restrict__ lpart,
                                                           int *__restrict__ err, uint32_t wait_tries)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sW2 = smem, *sW3 = smem + TB, *sH1 = smem + 2 * TB, *sH2 = smem + 3 * TB, *sH3 = smem + 4 * TB;
    uint8_t *sG = smem + 5 * TB;
    float *sF = reinterpret_cast<float *>(sH2);            // [128][129] f32 over sH2..sG, used last
    __shared__ float sx[TILE][4], sdy[TILE][2], sW4[2 * HID], sloss[4];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int b = threadIdx.x, warp = b >> 5, lane = b & 31;
    float *gp = gpart + (long)blockIdx.x * AF_MLP_NPARAM;

    if (warp == 0) tc::tmem_alloc(&tslot, HID);
    if (b == 0) { tc::mbar_init(&mbar, 1); tc::fence_mbar_init(); }
    stage_weight(sW2, W2b);
    stage_weight(sW3, W3b);
    for (int k = b; k < 2 * HID; k += blockDim.x) sW4[k] = P[OFF_W4 + k];
    const long sample = first + (long)blockIdx.x * TILE + b;
    const float4 xs = X[sample];
    const float2 ys = Y[sample];
    sx[b][0] = xs.x; sx[b][1] = xs.y; sx[b][2] = xs.z; sx[b][3] = xs.w;
    // layer 1 on the FP32 pipes: H1 = tanh(W1 x + b1)
    for (int c = 0; c < HID; c += 32) {
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float *w = P + OFF_W1 + (c + k) * 4;
            v[k] = tanh_fast(fmaf(w[0], xs.x, fmaf(w[1], xs.y, fmaf(w[2], xs.z, fmaf(w[3], xs.w, P[OFF_B1 + c + k])))));
        }
        store_row32(sH1, b, c, v);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    uint32_t phase = 0;
    bool ok = true;
    const int row = 32 * warp + lane;                      // == b

    // layer 2: Z2 = H1 W2^T
    ok = run_mma(tmem, sH1, 0, sW2, 0, &mbar, phase, wait_tries) && ok;
    for (int c = 0; c < HID; c += 32) {
        float v[32];
        row_chunk(tmem, c, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = tanh_fast(v[k] + P[OFF_B2 + c + k]);
        store_row32(sH2, row, c, v);
    }
    // layer 3: Z3 = H2 W3^T; layer 4 in the epilogue
    ok = run_mma(tmem, sH2, 0, sW3, 0, &mbar, phase, wait_tries) && ok;
    float y0 = P[OFF_B4], y1 = P[OFF_B4 + 1];
    for (int c = 0; c < HID; c += 32) {
        float v[32];
        row_chunk(tmem, c, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = __bfloat162float(__float2bfloat16_rn(tanh_fast(v[k] + P[OFF_B3 + c + k])));
        store_row32(sH3, row, c, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            y0 = fmaf(sW4[c + k], v[k], y0);
            y1 = fmaf(sW4[HID + c + k], v[k], y1);
        }
    }
    // loss = mean over the batch of (y - y*)^2 (both outputs); dy = dL/dy
    const float e0 = y0 - ys.x, e1 = y1 - ys.y;
    sdy[row][0] = 2.0f * e0 * inv_batch;
    sdy[row][1] = 2.0f * e1 * inv_batch;
    float l = (e0 * e0 + e1 * e1) * inv_batch;
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) sloss[warp] = l;
    // dZ3 = (dy W4) * (1 - H3^2), bf16 into sG
    {
        const float d0 = sdy[row][0], d1 = sdy[row][1];
        for (int c = 0; c < HID; c += 32) {
            float v[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float h = ld_bf16(sH3, row, c + k);
                v[k] = fmaf(d0, sW4[c + k], d1 * sW4[HID + c + k]) * (1.0f - h * h);
            }
            store_row32(sG, row, c, v);
        }
    }
    __syncthreads();
    // column reductions over the tile (thread j = feature): dW4, db3; db4, loss
    {
        const int j = b;
        float a0 = 0.f, a1 = 0.f, g3 = 0.f;
        for (int r = 0; r < TILE; ++r) {
            const float h = ld_bf16(sH3, r, j);
            a0 = fmaf(sdy[r][0], h, a0);
            a1 = fmaf(sdy[r][1], h, a1);
            g3 += ld_bf16(sG, r, j);
        }
        gp[OFF_W4 + j] = a0;
        gp[OFF_W4 + HID + j] = a1;
        gp[OFF_B3 + j] = g3;
        if (j < 2) {
            float s = 0.f;
            for (int r = 0; r < TILE; ++r) s += sdy[r][j];
            gp[OFF_B4 + j] = s;
        }
        if (j == 0) lpart[blockIdx.x] = sloss[0] + sloss[1] + sloss[2] + sloss[3];
    }
    // dW3 = dZ3^T H2  (A = sG as MN-major, B = sH2 as MN-major); rows of D = output feature
    ok = run_mma(tmem, sG, 1, sH2, 1, &mbar, phase, wait_tries) && ok;
    for (int c = 0; c < HID; c += 32) {
        float v[32];
        row_chunk(tmem, c, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) gp[OFF_W3 + row * HID + c + k] = v[k];
    }
    // dH2 = dZ3 W3 (A = sG K-major, B = sW3 as MN-major) -> dZ2 into sG
    ok = run_mma(tmem, sG, 0, sW3, 1, &mbar, phase, wait_tries) && ok;
    __syncthreads();                                        // every read of dZ3 is done
    for (int c = 0; c < HID; c += 32) {
        float v[32];
        row_chunk(tmem, c, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float h = ld_bf16(sH2, row, c + k);
            v[k] *= 1.0f - h * h;
        }
        store_row32(sG, row, c, v);
    }
    __syncthreads();
    {
        const int j = b;
        float g2 = 0.f;
        for (int r = 0; r < TILE; ++r) g2 += ld_bf16(sG, r, j);
        gp[OFF_B2 + j] = g2;
    }
    // dW2 = dZ2^T H1
    ok = run_mma(tmem, sG, 1, sH1, 1, &mbar, phase, wait_tries) && ok;
    for (int c = 0; c < HID; c += 32) {
        float v[32];
        row_chunk(tmem, c, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) gp[OFF_W2 + row * HID + c + k] = v[k];
    }
    // dH1 = dZ2 W2 -> dZ1 (f32) into sF
    ok = run_mma(tmem, sG, 0, sW2, 1, &mbar, phase, wait_tries) && ok;
    __syncthreads();                                        // sH2 / sH3 / sG are free now
    for (int c = 0; c < HID; c += 32) {
        float v[32];
        row_chunk(tmem, c, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float h = ld_bf16(sH1, row, c + k);
            sF[row * (HID + 1) + c + k] = v[k] * (1.0f - h * h);
        }
    }
    __syncthreads();
    {
        const int j = b;
        float g1 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f;
        for (int r = 0; r < TILE; ++r) {
            const float d = sF[r * (HID + 1) + j];
            g1 += d;
            w0 = fmaf(d, sx[r][0], w0);
            w1 = fmaf(d, sx[r][1], w1);
            w2 = fmaf(d, sx[r][2], w2);
            w3 = fmaf(d, sx[r][3], w3);
        }
        gp[OFF_B1 + j] = g1;
        gp[OFF_W1 + j * 4 + 0] = w0;
        gp[OFF_W1 + j * 4 + 1] = w1;
        gp[OFF_W1 + j * 4 + 2] = w2;
        gp[OFF_W1 + j * 4 + 3] = w3;
    }
    if (!ok) atomicExch(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::tmem_dealloc(tmem, HID);
        tc::tmem_relinquish();
    }
}

// Adam over the summed per-CTA partials; refreshes the bf16 copies of W2, W3
__global__ void mlp_adam_kernel(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                                const float *__restrict__ gpart, int nparts, float lr, float bc1, float bc2,
                                __nv_bfloat16 *__restrict__ W2b, __nv_bfloat16 *__restrict__ W3b,
                                float *__restrict__ G)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= AF_MLP_NPARAM) return;
    float g = 0.f;
    for (int c = 0; c < nparts; ++c) g += gpart[(long)c * AF_MLP_NPARAM + k];
    if (G) G[k] = g;
    if (lr > 0.f) {
        const float m = 0.9f * M[k] + 0.1f * g;
        const float v = 0.999f * V[k] + 0.001f * g * g;
        M[k] = m;
        V[k] = v;
        P[k] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
    }
    if (k >= OFF_W2 && k < OFF_W2 + HID * HID) W2b[k - OFF_W2] = __float2bfloat16_rn(P[k]);
    if (k >= OFF_W3 && k < OFF_W3 + HID * HID) W3b[k - OFF_W3] = __float2bfloat16_rn(P[k]);
}

// ---------------------------------------------------------------- samples
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double unif(uint64_t key, int k)
{
    return (double)(splitmix64(key * 8 + k) >> 11) * (1.0 / 9007199254740992.0);
}

// exact label (float64 Fermat solve) of one configuration
__device__ void exact_exit(const MlpGeom &G, double th_e, double rho, double th_p, double c, double *delta,
                           double *tl)
{
    const double dp = th_p - th_e;
    const double x = exit_solve_fp64(G.re, rho, G.RL, dp, G.inv_c_lens, 1.0 / c);
    *delta = x;
    *tl = chord_d(G.re, G.RL, x).len * G.inv_c_lens;
}

// samples inside the constant f-number cone of an element on the arc, c in [c_lo, c_hi]
__global__ void mlp_gen_kernel(MlpGeom G, MlpNorm n, long count, uint64_t seed, float4 *__restrict__ X,
                               float2 *__restrict__ Y)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        const uint64_t key = splitmix64(seed ^ (uint64_t)i);
        const double th_e = G.th_lo + (G.th_hi - G.th_lo) * unif(key, 0);
        const double zp = G.z_lo + (G.z_hi - G.z_lo) * unif(key, 1);
        const double xp = (2.0 * unif(key, 2) - 1.0) * zp * G.cone;
        const double c = G.c_lo + (G.c_hi - G.c_lo) * unif(key, 3);
        // element on the arc, normal = radial direction
        const double ex = G.re * sin(th_e), ez = G.re * cos(th_e);
        const double px = ex + zp * sin(th_e) + xp * cos(th_e), pz = ez + zp * cos(th_e) - xp * sin(th_e);
        const double rho = sqrt(px * px + pz * pz), th_p = atan2(px, pz);
        double dl, tl;
        exact_exit(G, th_e, rho, th_p, c, &dl, &tl);
        float x[4];
        features(n, (float)th_e, (float)rho, (float)th_p, (float)c, x);
        X[i] = make_float4(x[0], x[1], x[2], x[3]);
        Y[i] = make_float2((float)(dl / n.y0_s), (float)((tl - n.y1_c) / n.y1_s));
    }
}

// ---------------------------------------------------------------- inference
// Persistent: each CTA keeps W2, W3 in shared memory (and the small parameters
// W1, b1..b4, W4) and runs tiles of 128 (element, pixel) pairs.  256 threads:
// warp w reads tensor-memory lanes 32 (w mod 4).. (its rows) and handles hidden
// columns 64 (w / 4)..+63 of them, so two warps share a row's epilogue; two CTAs
// per SM let one CTA's epilogue overlap the other's MMA.  Writes the exit angle
// (phi) and the predicted lens time for every pair whose fallback bit is clear
// (all pairs if fb is NULL).
constexpr int kInferThreads = 256;
constexpr int kHalf = HID / 2;

__global__ void __launch_bounds__(kInferThreads) mlp_infer_kernel(AfGeom g, MlpNorm n, const float *__restrict__ P,
                                                                  const __nv_bfloat16 *__restrict__ W2b,
                                                                  const __nv_bfloat16 *__restrict__ W3b,
                                                                  const float2 *__restrict__ elem_pol,
                                                                  const float2 *__restrict__ pix_pol,
                                                                  const AfScal *__restrict__ scal, float c_fixed,
                                                                  const uint8_t *__restrict__ fb,
                                                                  float *__restrict__ phi_out,
                                                                  float *__restrict__ tl_out, int *__restrict__ err,
                                                                  uint32_t wait_tries)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sW2 = smem, *sW3 = smem + TB, *sH = smem + 2 * TB;
    __shared__ __align__(16) float sW1[HID * 4], sB1[HID], sB2[HID], sB3[HID], sW4[2 * HID];
    __shared__ float2 sY[TILE];                 // the second half's partial outputs
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int b = threadIdx.x, warp = b >> 5, lane = b & 31;
    const int quad = warp & 3, half = warp >> 2, row = 32 * quad + lane, c0 = half * kHalf;
    if (warp == 0) {
        tc::tmem_alloc(&tslot, HID);
        tc::tmem_relinquish();       // no further allocation: let the SM's other CTA allocate
    }
    if (b == 0) { tc::mbar_init(&mbar, 1); tc::fence_mbar_init(); }
    stage_weight(sW2, W2b);
    stage_weight(sW3, W3b);
    for (int k = b; k < HID * 4; k += kInferThreads) sW1[k] = P[OFF_W1 + k];
    for (int k = b; k < HID; k += kInferThreads) {
        sB1[k] = P[OFF_B1 + k];
        sB2[k] = P[OFF_B2 + k];
        sB3[k] = P[OFF_B3 + k];
    }
    for (int k = b; k < 2 * HID; k += kInferThreads) sW4[k] = P[OFF_W4 + k];
    const float b40 = P[OFF_B4], b41 = P[OFF_B4 + 1];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
    const float c = c_fixed > 0.f ? c_fixed : 1.0f / scal->sbar;
    uint32_t phase = 0;
    bool ok = true;
    const long total = (long)g.ne * g.npix;
    const long ntiles = (total + TILE - 1) / TILE;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long idx = t * TILE + row;
        const bool live = idx < total;
        const int e = live ? (int)(idx / g.npix) : 0, p = live ? (int)(idx - (long)e * g.npix) : 0;
        const float2 ep = elem_pol[e], pp = pix_pol[p];
        float x[4];
        features(n, ep.x, pp.y, pp.x, c, x);
        // layer 1 (4 -> 128, FP32): this thread's 64 columns of its row
#pragma unroll
        for (int cc = 0; cc < kHalf; cc += 32) {
            float v[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float4 w = *reinterpret_cast<const float4 *>(sW1 + (c0 + cc + k) * 4);
                v[k] = tanh_fast(fmaf(w.x, x[0], fmaf(w.y, x[1], fmaf(w.z, x[2], fmaf(w.w, x[3], sB1[c0 + cc + k])))));
            }
            store_row32(sH, row, c0 + cc, v);
        }
        ok = run_mma(tmem, sH, 0, sW2, 0, &mbar, phase, wait_tries) && ok;
        __syncthreads();                                   // the MMA has consumed H1
#pragma unroll
        for (int cc = 0; cc < kHalf; cc += 32) {
            float v[32];
            tc::tmem_ld32(trow + c0 + cc, v);
#pragma unroll
            for (int k = 0; k < 32; ++k) v[k] = tanh_fast(v[k] + sB2[c0 + cc + k]);
            store_row32(sH, row, c0 + cc, v);
        }
        ok = run_mma(tmem, sH, 0, sW3, 0, &mbar, phase, wait_tries) && ok;
        float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
        for (int cc = 0; cc < kHalf; cc += 32) {
            float v[32];
            tc::tmem_ld32(trow + c0 + cc, v);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const float h = round_bf16(tanh_fast(v[k] + sB3[c0 + cc + k]));
                y0 = fmaf(sW4[c0 + cc + k], h, y0);
                y1 = fmaf(sW4[HID + c0 + cc + k], h, y1);
            }
        }
        if (half == 1) sY[row] = make_float2(y0, y1);
        __syncthreads();                                   // sY ready; sH free for the next tile
        if (half == 0 && live && (!fb || !fb[idx])) {
            const float2 q = sY[row];
            phi_out[idx] = ep.x + (b40 + y0 + q.x) * n.y0_s;
            if (tl_out) tl_out[idx] = n.y1_c + (b41 + y1 + q.y) * n.y1_s;
        }
    }
    if (!ok) atomicExch(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, HID);
}

// Validation at one medium speed: delay error of the surrogate's exit angle
// (exact path lengths) and error of its lens-time output, per apodized pair;
// sets fallback bits above tol and accumulates statistics.
__global__ void mlp_validate_kernel(AfGeom g, MlpGeom G, const float2 *__restrict__ elem_pol,
                                    const float2 *__restrict__ pix_pol, const float4 *__restrict__ D, double c,
                                    const float *__restrict__ phi_s, const float *__restrict__ tl_s, double tol,
                                    uint8_t *__restrict__ fb, unsigned long long *__restrict__ stats)
{
    const long total = (long)g.ne * g.npix;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        if (__float_as_int(D[idx].x) == AF_APOD_OFF) continue;
        const int e = (int)(idx / g.npix), p = (int)(idx - (long)e * g.npix);
        const double th_e = elem_pol[e].x, rho = pix_pol[p].y, th_p = pix_pol[p].x;
        double dl, tl;
        exact_exit(G, th_e, rho, th_p, c, &dl, &tl);
        const double dp = th_p - th_e, sbar = 1.0 / c;
        const double xs = (double)phi_s[idx] - th_e;
        const double t_star = chord_d(G.re, G.RL, dl).len * G.inv_c_lens + chord_d(rho, G.RL, dl - dp).len * sbar;
        const double t_sur = chord_d(G.re, G.RL, xs).len * G.inv_c_lens + chord_d(rho, G.RL, xs - dp).len * sbar;
        const double derr = fabs(t_sur - t_star);           // >= 0 up to rounding (Fermat minimum)
        const double lerr = fabs((double)tl_s[idx] - tl);
        const bool bad = !(derr <= tol);
        if (bad) fb[idx] = 1;
        // stats: [0] count, [1] fallbacks (this speed), [2] max delay err (ps, as int),
        // [3] max lens-time err (ps), [4] sum of squared angle errors (1e-12 rad^2 units)
        atomicAdd(&stats[0], 1ull);
        if (bad) atomicAdd(&stats[1], 1ull);
        atomicMax(&stats[2], (unsigned long long)fmin(derr * 1e12, 1e18));
        atomicMax(&stats[3], (unsigned long long)fmin(lerr * 1e12, 1e18));
        const double ae = xs - dl;
        atomicAdd(&stats[4], (unsigned long long)fmin(ae * ae * 1e12, 1e15));
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
static constexpr int kTrainSmem = 6 * TB;          // bf16 tiles: W2, W3, H1, H2, H3, G
static constexpr int kInferSmem = 3 * TB;          // W2, W3, H

cudaError_t mlp_setup_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem);
    // the largest shared-memory carveout, so that two inference CTAs fit on an SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t mlp_init_params(af_plan_t pl, uint64_t seed)
{
    std::vector<float> h(AF_MLP_NPARAM, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int fan_in, int fan_out, int count) {
        const double a = sqrt(6.0 / (fan_in + fan_out));
        std::uniform_real_distribution<double> u(-a, a);
        for (int k = 0; k < count; ++k) h[off + k] = (float)u(rng);
    };
    fill(OFF_W1, 4, HID, HID * 4);
    fill(OFF_W2, HID, HID, HID * HID);
    fill(OFF_W3, HID, HID, HID * HID);
    fill(OFF_W4, HID, 2, 2 * HID);
    cudaError_t e = cudaMemcpyAsync(pl->mlp_p, h.data(), AF_MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, pl->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->mlp_m, 0, AF_MLP_NPARAM * sizeof(float), pl->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->mlp_v, 0, AF_MLP_NPARAM * sizeof(float), pl->stream);
    if (e == cudaSuccess)
        mlp_adam_kernel<<<(AF_MLP_NPARAM + 255) / 256, 256, 0, pl->stream>>>(
            pl->mlp_p, pl->mlp_m, pl->mlp_v, pl->mlp_g, 0, 0.0f, 1.0f, 1.0f,
            reinterpret_cast<__nv_bfloat16 *>(pl->mlp_w2b), reinterpret_cast<__nv_bfloat16 *>(pl->mlp_w3b), nullptr);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t mlp_generate(af_plan_t pl, long count, uint64_t seed, float4 *X, float2 *Y)
{
    mlp_gen_kernel<<<pl->sm_count * 8, 256, 0, pl->stream>>>(pl->mlp_geom, pl->mlp_norm, count, seed, X, Y);
    return cudaGetLastError();
}

// one optimisation step on samples [first, first + ntiles * 128); lr = 0 only
// computes the summed gradient into pl->mlp_g
cudaError_t mlp_train_step(af_plan_t pl, const float4 *X, const float2 *Y, long first, int ntiles, float lr,
                           int step, float *lpart, float *gpart)
{
    mlp_train_kernel<<<ntiles, 128, kTrainSmem, pl->stream>>>(
        X, Y, first, 1.0f / (ntiles * TILE), pl->mlp_p, reinterpret_cast<const __nv_bfloat16 *>(pl->mlp_w2b),
        reinterpret_cast<const __nv_bfloat16 *>(pl->mlp_w3b), gpart, lpart, &pl->scal->mlp_err, af_wait_tries());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double bc1 = 1.0 - pow(0.9, step), bc2 = 1.0 - pow(0.999, step);
    mlp_adam_kernel<<<(AF_MLP_NPARAM + 255) / 256, 256, 0, pl->stream>>>(
        pl->mlp_p, pl->mlp_m, pl->mlp_v, gpart, ntiles, lr, (float)bc1, (float)bc2,
        reinterpret_cast<__nv_bfloat16 *>(pl->mlp_w2b), reinterpret_cast<__nv_bfloat16 *>(pl->mlp_w3b), pl->mlp_g);
    return cudaGetLastError();
}

cudaError_t mlp_infer(af_plan_t pl, float c_fixed, const uint8_t *fb, float *phi_out, float *tl_out)
{
    if ((long)pl->g.ne * pl->g.npix == 0) return cudaSuccess;
    mlp_infer_kernel<<<pl->sm_count * 2, kInferThreads, kInferSmem, pl->stream>>>(
        pl->g, pl->mlp_norm, pl->mlp_p, reinterpret_cast<const __nv_bfloat16 *>(pl->mlp_w2b),
        reinterpret_cast<const __nv_bfloat16 *>(pl->mlp_w3b), pl->elem_pol, pl->pix_pol, pl->scal, c_fixed, fb,
        phi_out, tl_out, &pl->scal->mlp_err, af_wait_tries());
    return cudaGetLastError();
}

cudaError_t mlp_validate(af_plan_t pl, double c, const float *phi_s, const float *tl_s, double tol, uint8_t *fb,
                         unsigned long long *stats)
{
    mlp_validate_kernel<<<pl->sm_count * 8, 256, 0, pl->stream>>>(pl->g, pl->mlp_geom, pl->elem_pol, pl->pix_pol,
                                                                  pl->D, c, phi_s, tl_s, tol, fb, stats);
    return cudaGetLastError();
}

cudaError_t mlp_refresh_bf16(af_plan_t pl)
{
    mlp_adam_kernel<<<(AF_MLP_NPARAM + 255) / 256, 256, 0, pl->stream>>>(
        pl->mlp_p, pl->mlp_m, pl->mlp_v, pl->mlp_g, 0, 0.0f, 1.0f, 1.0f,
        reinterpret_cast<__nv_bfloat16 *>(pl->mlp_w2b), reinterpret_cast<__nv_bfloat16 *>(pl->mlp_w3b), nullptr);
    return cudaGetLastError();
}
