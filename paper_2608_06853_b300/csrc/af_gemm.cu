// BF16 GEMM on the fifth-generation tensor cores (tcgen05, accumulators in
// tensor memory): the dense-contraction building block of the lens-surrogate
// MLP.  D[M][N] (f32) = sum_k A(m, k) B(n, k) with A stored [M][K] (K-major) or
// [K][M] (MN-major) and B stored [N][K] or [K][N], all row-major in global
// memory.  One CTA of 4 warps per 128 x 128 output tile; K is staged through
// shared memory 64 at a time in the no-swizzle core-matrix layout of af_tc.cuh.
#include <cuda_bf16.h>

#include "af_internal.cuh"
#include "af_tc.cuh"

namespace {

constexpr int kTile = 128, kChunk = 64;
// Extra dynamic shared memory: keeps at most three CTAs per SM, so their
// tensor-memory allocations (3 x 128 of the 512 columns) never wait on each other.
constexpr int kGuardSmem = 40 * 1024;

// global -> shared, 16 bytes (8 elements) per store, in the canonical layout
__device__ __forceinline__ void stage_operand(uint8_t *dst, const __nv_bfloat16 *src, int rows0, int k0,
                                              int ld, int mn_major)
{
    for (int u = threadIdx.x; u < kTile * kChunk / 8; u += blockDim.x) {
        uint4 v;
        uint32_t off;
        if (!mn_major) {                                  // src[row][k], k contiguous
            const int r = u / (kChunk / 8), kc = (u % (kChunk / 8)) * 8;
            v = *reinterpret_cast<const uint4 *>(src + (long)(rows0 + r) * ld + k0 + kc);
            off = tc::kmajor_offset(r, kc, kChunk);
        } else {                                          // src[k][row], row contiguous
            const int k = u / (kTile / 8), rc = (u % (kTile / 8)) * 8;
            v = *reinterpret_cast<const uint4 *>(src + (long)(k0 + k) * ld + rows0 + rc);
            off = tc::mnmajor_offset(rc, k, kTile);
        }
        *reinterpret_cast<uint4 *>(dst + off) = v;
    }
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16 *__restrict__ A,
                                                        const __nv_bfloat16 *__restrict__ B,
                                                        float *__restrict__ D, int M, int N, int K,
                                                        int a_mn, int b_mn, int *__restrict__ err,
                                                        uint32_t wait_tries)
{
    __shared__ __align__(1024) uint8_t sA[kTile * kChunk * 2];
    __shared__ __align__(1024) uint8_t sB[kTile * kChunk * 2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
    if (warp == 0) tc::tmem_alloc(&tslot, kTile);
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(kTile, kTile, a_mn, b_mn);
    // descriptor strides and the per-instruction advance along K (16 elements)
    // K-major: LBO = 128 B (next 8 K), SBO = kChunk * 16 B (next 8 rows);
    // MN-major: LBO = kTile * 16 B (next 8 K), SBO = 128 B (next 8 rows)
    const uint32_t lbo_a = a_mn ? kTile * 16 : 128, sbo_a = a_mn ? 128 : kChunk * 16, step_a = 2 * lbo_a;
    const uint32_t lbo_b = b_mn ? kTile * 16 : 128, sbo_b = b_mn ? 128 : kChunk * 16, step_b = 2 * lbo_b;
    bool ok = true;
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K; k0 += kChunk) {
        stage_operand(sA, A, m0, k0, a_mn ? M : K, a_mn);
        stage_operand(sB, B, n0, k0, b_mn ? N : K, b_mn);
        tc::fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            for (int kk = 0; kk < kChunk / 16; ++kk) {
                const uint64_t da = tc::smem_desc(tc::smem_addr(sA) + kk * step_a, lbo_a, sbo_a);
                const uint64_t db = tc::smem_desc(tc::smem_addr(sB) + kk * step_b, lbo_b, sbo_b);
                tc::mma_bf16(tmem, da, db, idesc, (k0 > 0 || kk > 0) ? 1 : 0);
            }
            tc::mma_commit(&mbar);
        }
        ok = tc::mma_wait(&mbar, phase, wait_tries) && ok;
        phase ^= 1u;
        // the products are complete (or the second wait ran out): shared operands may be
        // overwritten; the CTA stops at the first timeout of any thread
        if (!__syncthreads_and(ok)) { ok = false; break; }
    }
    tc::fence_after_sync();
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < kTile / 32; ++c) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c * 32, v);
            float *row = D + (long)(m0 + warp * 32 + lane) * N + n0 + c * 32;
#pragma unroll
            for (int k = 0; k < 32; ++k) row[k] = v[k];
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::tmem_dealloc(tmem, kTile);
        tc::tmem_relinquish();
    }
}

}  // namespace

extern "C" af_status af_gemm_bf16(const void *d_A, const void *d_B, float *d_D, int M, int N, int K,
                                  int a_mn_major, int b_mn_major, int *d_err, void *stream)
{
    if (!d_A || !d_B || !d_D || !d_err) return af_set_error(AF_ERR_ARG, "af_gemm_bf16: NULL pointer");
    if (M <= 0 || N <= 0 || K <= 0 || M % kTile || N % kTile || K % kChunk)
        return af_set_error(AF_ERR_SHAPE, "af_gemm_bf16: M, N must be multiples of 128 and K of 64");
    if (((uintptr_t)d_A | (uintptr_t)d_B) & 15) return af_set_error(AF_ERR_ARG, "af_gemm_bf16: operands not 16-byte aligned");
    dim3 grid(N / kTile, M / kTile);
    cudaError_t a = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGuardSmem);
    if (a != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_gemm_bf16: %s", cudaGetErrorString(a));
    gemm_bf16_kernel<<<grid, 128, kGuardSmem, (cudaStream_t)stream>>>(
        reinterpret_cast<const __nv_bfloat16 *>(d_A), reinterpret_cast<const __nv_bfloat16 *>(d_B), d_D, M, N, K,
        a_mn_major ? 1 : 0, b_mn_major ? 1 : 0, d_err, af_wait_tries());
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_gemm_bf16: %s", cudaGetErrorString(e));
    return AF_OK;
}
