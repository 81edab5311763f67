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
//  - Every call looks up the device address of the scratch array on the
//    current device (cudaGetSymbolAddress, no allocation); the first call on a
//    device may load the library's device code there, so make it before any
//    stream capture.  Nothing is cached, so a device reset between calls
//    (cudaDeviceReset) leaves the entry point usable.
//  - Every call shares the one scratch array.  Calls that overlap on the GPU
//    (different streams, or different host threads without ordering) race on
//    it; order them on one stream or synchronise between them.
//  - Each call writes every scratch entry it later reads, so nothing has to
//    start at zero and the contents left by an earlier call do not matter.
//  - n_patch above AF_NOALLOC_MAX_PATCHES is rejected with
//    AF_ERR_UNSUPPORTED; nothing here calls cudaMalloc or cudaFree.
#include <math.h>

#include "af_cmpe.cuh"
#include "af_internal.cuh"

namespace {

struct PatchPartial {
    double sum;       // sum over active pairs of |arg z|
    int count;        // active pairs
    int pad;
};

static __device__ __align__(256) PatchPartial g_patch_partials[AF_NOALLOC_MAX_PATCHES];

// one CTA per patch, warp w takes the kPairsPerWarp pairs from w kPairsPerWarp on,
// then those 8 kPairsPerWarp further, ... (the pair arithmetic and lane grouping
// of the planned path, cmpe::pair_terms, so both take the same mask decisions)
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
    const int slot = lane / cmpe::kPairLanes, sub = lane % cmpe::kPairLanes;
    for (int k0 = w * cmpe::kPairsPerWarp; k0 < npair; k0 += 8 * cmpe::kPairsPerWarp) {
        const int k = k0 + slot;
        const cmpe::PairTerms t = cmpe::pair_terms(B, nsub, npix, base, patch_npix, k, sub, k < npair);
        if (sub == 0 && k < npair && t.rho >= rho_thresh) {
            lsum += (double)fabsf(atan2f(t.zi, t.zr));
            ++cnt;
        }
    }
    lsum = cmpe::group_leaders_sum(lsum);
    cnt = cmpe::group_leaders_sum(cnt);
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

// device address of the scratch array on the current device (looked up on every call:
// host code cannot use the array's name as a device pointer)
cudaError_t scratch_for_current_device(PatchPartial **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_patch_partials);
    if (e != cudaSuccess) return e;
    *out = static_cast<PatchPartial *>(p);
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
