// af_cmpe_loss_noalloc: the CMPE focusing loss of caller-provided subaperture
// images, computed without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// real-time acquisition pipeline that reserves all of its GPU memory at
// start-up and forbids allocation while it streams, or a host framework that
// owns the device allocator and does not let plug-ins call cudaMalloc.  This
// entry point needs no plan and no workspace: its only scratch, the per-patch
// partial sums, lives in a fixed array in the library's own device memory
// (g_patch_partials below, AF_NOALLOC_MAX_PATCHES entries of 16 bytes), which
// every GPU that loads the library holds until the process exits.
//
// Rules of use (also stated in include/af.h):
//  - The first call on a device looks up the device address of the scratch
//    array (cudaGetSymbolAddress) with that device current; make that first
//    call before any stream capture.
//  - Every call shares the one scratch array.  Calls that overlap on the GPU
//    (different streams, or different host threads without ordering) race on
//    it; order them on one stream or synchronise between them.
//  - Each call writes every scratch entry it later reads, so nothing has to
//    start at zero and the contents left by an earlier call do not matter.
//  - n_patch above AF_NOALLOC_MAX_PATCHES is rejected with
//    AF_ERR_UNSUPPORTED; nothing here calls cudaMalloc or cudaFree.
#include <math.h>
#include <mutex>

#include "af_internal.cuh"

namespace {

struct PatchPartial {
    double sum;       // sum over active pairs of |arg z|
    int count;        // active pairs
    int pad;
};

static __device__ __align__(256) PatchPartial g_patch_partials[AF_NOALLOC_MAX_PATCHES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
PatchPartial *g_scratch[kMaxDevices] = {};

__device__ __forceinline__ float warp_sum_na(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one CTA per patch, warp w takes pairs w, w + 8, ... (same reading of the
// CMPE as the planned path: pairs (i,j) ~ (i+1, j-1), j = i + 1 skipped)
__global__ void __launch_bounds__(256) noalloc_patch_kernel(const float2 *__restrict__ B, int nsub,
                                                            int npix, int patch_npix, float rho_thresh,
                                                            PatchPartial *__restrict__ part)
{
    __shared__ double s_sum[8];
    __shared__ int s_cnt[8];
    const int P = blockIdx.x, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int npair = (nsub - 1) * (nsub - 2);
    const int base = P * patch_npix;
    double lsum = 0.0;
    int cnt = 0;
    for (int k = w; k < npair; k += 8) {
        const int i = k / (nsub - 2), jj = k - i * (nsub - 2);
        const int j = jj < i ? jj + 1 : jj + 2;
        const float2 *B1 = B + (long)(i * nsub + j) * npix + base;
        const float2 *B2 = B + (long)((i + 1) * nsub + (j - 1)) * npix + base;
        float zr = 0.f, zi = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll 4
        for (int q = lane; q < patch_npix; q += 32) {
            const float2 a = B1[q], c = B2[q];
            zr = fmaf(a.x, c.x, fmaf(a.y, c.y, zr));
            zi = fmaf(a.y, c.x, fmaf(-a.x, c.y, zi));
            e1 = fmaf(a.x, a.x, fmaf(a.y, a.y, e1));
            e2 = fmaf(c.x, c.x, fmaf(c.y, c.y, e2));
        }
        zr = warp_sum_na(zr); zi = warp_sum_na(zi); e1 = warp_sum_na(e1); e2 = warp_sum_na(e2);
        if (lane == 0) {
            // float epilogue (the sums are float); sqrt of each energy avoids overflow
            const float den = sqrtf(e1) * sqrtf(e2);
            const float rho = den > 0.0f ? hypotf(zr, zi) / den : 0.0f;
            if (rho >= rho_thresh) {
                lsum += (double)fabsf(atan2f(zi, zr));
                ++cnt;
            }
        }
    }
    if (lane == 0) { s_sum[w] = lsum; s_cnt[w] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        int c = 0;
        for (int k = 0; k < 8; ++k) { a += s_sum[k]; c += s_cnt[k]; }
        part[P].sum = a;        // written before the finalize kernel reads it
        part[P].count = c;
    }
}

__global__ void __launch_bounds__(256) noalloc_finalize_kernel(const PatchPartial *__restrict__ part,
                                                               int n_patch, float *__restrict__ loss,
                                                               int *__restrict__ n_active)
{
    __shared__ double s_a[256];
    __shared__ int s_c[256];
    double a = 0.0;
    int c = 0;
    for (int P = threadIdx.x; P < n_patch; P += 256) { a += part[P].sum; c += part[P].count; }
    s_a[threadIdx.x] = a;
    s_c[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s_a[threadIdx.x] += s_a[threadIdx.x + o]; s_c[threadIdx.x] += s_c[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int M = s_c[0];
        loss[0] = (float)(s_a[0] / (M > 1 ? M : 1));
        if (n_active) *n_active = M;
    }
}

// device address of the scratch array on the current device (looked up once per device)
cudaError_t scratch_for_current_device(PatchPartial **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_patch_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = static_cast<PatchPartial *>(p);
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" af_status af_cmpe_loss_noalloc(const float *d_B, int nsub, int n_patch, int patch_npix,
                                          double rho_thresh, float *d_loss, int *d_n_active,
                                          void *stream)
{
    if (!d_B || !d_loss) return af_set_error(AF_ERR_ARG, "af_cmpe_loss_noalloc: d_B and d_loss must be non-NULL");
    if (nsub < 1 || n_patch < 0 || patch_npix < 1 || !isfinite(rho_thresh))
        return af_set_error(AF_ERR_ARG, "af_cmpe_loss_noalloc: bad nsub / n_patch / patch_npix / rho_thresh");
    if (n_patch > AF_NOALLOC_MAX_PATCHES)
        return af_set_error(AF_ERR_UNSUPPORTED, "af_cmpe_loss_noalloc: n_patch %d exceeds the fixed scratch of "
                            "%d patches", n_patch, AF_NOALLOC_MAX_PATCHES);
    if ((long long)nsub * nsub * n_patch * patch_npix >= (1LL << 31))
        return af_set_error(AF_ERR_UNSUPPORTED, "af_cmpe_loss_noalloc: too many pixels");
    PatchPartial *part = nullptr;
    const cudaError_t e = scratch_for_current_device(&part);
    if (e != cudaSuccess)
        return af_set_error(AF_ERR_CUDA, "af_cmpe_loss_noalloc: scratch address lookup: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    const int npair = nsub >= 3 ? (nsub - 1) * (nsub - 2) : 0;
    const int np = npair > 0 ? n_patch : 0;
    if (np > 0) {
        noalloc_patch_kernel<<<np, 256, 0, st>>>(reinterpret_cast<const float2 *>(d_B), nsub,
                                                 n_patch * patch_npix, patch_npix, (float)rho_thresh, part);
        const cudaError_t k = cudaGetLastError();
        if (k != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_cmpe_loss_noalloc: %s", cudaGetErrorString(k));
    }
    noalloc_finalize_kernel<<<1, 256, 0, st>>>(part, np, d_loss, d_n_active);
    const cudaError_t k = cudaGetLastError();
    if (k != cudaSuccess) return af_set_error(AF_ERR_CUDA, "af_cmpe_loss_noalloc: %s", cudaGetErrorString(k));
    return af_set_error(AF_OK, "");
}
