// The per-pair arithmetic of the common-midpoint phase error (Sec. II-D), shared
// by the planned forward (af_cmpe.cu) and the allocation-free entry point
// (af_noalloc.cu) so that both follow one reading of the CMPE:
// per patch and per pair of common-midpoint subaperture images (i, j) ~
// (i+1, j-1), with the reciprocal pair j = i + 1 skipped,
//   z = sum_p B_ij(p) conj(B_i+1,j-1(p)),
//   rho = |z| / sqrt(sum |B_ij|^2 sum |B_i+1,j-1|^2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cmpe {

// pair k of a patch -> (i, j) of its first image; the second is (i+1, j-1)
__device__ __forceinline__ void pair_ij(int k, int n, int &i, int &j)
{
    i = k / (n - 2);
    int jj = k - i * (n - 2);
    j = jj < i ? jj + 1 : jj + 2;
}

struct PairTerms {
    float zr, zi, rho;    // z and the correlation coefficient (every lane of the group holds them)
};

// A warp works on kPairsPerWarp pairs at once, kPairLanes lanes each: lane l takes
// pair slot l / kPairLanes and pixels l % kPairLanes, + kPairLanes, ...  For a 9 x 9
// patch that is ~10 pixels per lane and 3 shuffle steps per sum, against 3 pixels
// and 5 steps with a whole warp per pair (CMPE forward, 128 elements: 29.5 us
// against 40.0 us; 2 pairs per warp 32.9 us, 8 pairs 31.0 us).
constexpr int kPairLanes = 8;
constexpr int kPairsPerWarp = 32 / kPairLanes;

// The cross term and correlation of pair k of the patch whose pixels start at
// `base`, summed by the lane group that holds the pair (`sub` = lane within the
// group; B is [nsub * nsub][npix] complex).  Every lane of the warp calls it at
// once (the sums are reduced by shuffles within each group); a group with
// valid == false adds nothing.
__device__ __forceinline__ PairTerms pair_terms(const float2 *__restrict__ B, int nsub, int npix, int base,
                                               int patch_npix, int k, int sub, bool valid)
{
    float zr = 0.f, zi = 0.f, e1 = 0.f, e2 = 0.f;
    if (valid) {
        int i, j;
        pair_ij(k, nsub, i, j);
        const float2 *B1 = B + (long)(i * nsub + j) * npix + base;
        const float2 *B2 = B + (long)((i + 1) * nsub + (j - 1)) * npix + base;
#pragma unroll 4
        for (int q = sub; q < patch_npix; q += kPairLanes) {
            const float2 a = B1[q], c = B2[q];
            zr = fmaf(a.x, c.x, fmaf(a.y, c.y, zr));
            zi = fmaf(a.y, c.x, fmaf(-a.x, c.y, zi));
            e1 = fmaf(a.x, a.x, fmaf(a.y, a.y, e1));
            e2 = fmaf(c.x, c.x, fmaf(c.y, c.y, e2));
        }
    }
    for (int o = kPairLanes / 2; o > 0; o >>= 1) {
        zr += __shfl_xor_sync(0xffffffffu, zr, o);
        zi += __shfl_xor_sync(0xffffffffu, zi, o);
        e1 += __shfl_xor_sync(0xffffffffu, e1, o);
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    }
    // float epilogue (the sums are float); sqrt of each energy avoids overflow
    const float den = sqrtf(e1) * sqrtf(e2);
    return PairTerms{zr, zi, den > 0.0f ? hypotf(zr, zi) / den : 0.0f};
}

// sum over the first lanes of the warp's pair groups (lanes 0, kPairLanes, ...);
// every lane gets it (the other lanes must hold zero)
template <typename T> __device__ __forceinline__ T group_leaders_sum(T v)
{
    for (int o = 16; o >= kPairLanes; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// index of the pair whose first image is (i, j), or -1
__device__ __forceinline__ int pair_index(int i, int j, int n)
{
    if (i < 0 || i > n - 2 || j < 1 || j > n - 1 || j == i + 1) return -1;
    return i * (n - 2) + (j - 1) - (j > i + 1 ? 1 : 0);
}

// sign of arg z as atan2 defines it: the sign of Im z, and on the real axis
// +pi (or -pi for Im z = -0) left of the origin, 0 right of it
__device__ __forceinline__ float arg_sign(float2 z)
{
    if (z.y > 0.0f) return 1.0f;
    if (z.y < 0.0f) return -1.0f;
    if (z.x < 0.0f) return signbit(z.y) ? -1.0f : 1.0f;
    return 0.0f;
}

// dL_CMPE/dB_ij(p) (= dL/dRe B + j dL/dIm B) with the mask held constant: image
// (i, j) is the first member of at most one pair ((i,j) ~ (i+1,j-1)) and the second
// member of at most one ((i-1,j+1) ~ (i,j)) of its patch P:
//   first:  w j z B2 / |z|^2     second: -w j conj(z) B1 / |z|^2,  w = sgn(arg z) / max(1, M)
// B is [nsub * nsub][npix]; z, mask are [n_patch][npair].
__device__ __forceinline__ float2 image_grad(const float2 *__restrict__ B, const float2 *__restrict__ z,
                                             const uint8_t *__restrict__ mask, float inv_m, int n, int npix,
                                             int npair, int P, int i, int j, int p)
{
    const int k1 = pair_index(i, j, n), k2 = pair_index(i - 1, j + 1, n);
    float gr = 0.0f, gi = 0.0f;
    if (k1 >= 0) {
        const long o = (long)P * npair + k1;
        if (mask[o]) {
            const float2 zz = z[o];
            const float mag2 = zz.x * zz.x + zz.y * zz.y;
            const float sg = arg_sign(zz);
            if (sg != 0.0f && mag2 > 0.0f) {
                const float w = sg * inv_m / mag2;
                const float2 c = B[(long)((i + 1) * n + (j - 1)) * npix + p];
                const float tr = zz.x * c.x - zz.y * c.y, ti = zz.x * c.y + zz.y * c.x;
                gr += -w * ti;
                gi += w * tr;
            }
        }
    }
    if (k2 >= 0) {
        const long o = (long)P * npair + k2;
        if (mask[o]) {
            const float2 zz = z[o];
            const float mag2 = zz.x * zz.x + zz.y * zz.y;
            const float sg = arg_sign(zz);
            if (sg != 0.0f && mag2 > 0.0f) {
                const float w = sg * inv_m / mag2;
                const float2 a = B[(long)((i - 1) * n + (j + 1)) * npix + p];
                const float ur = zz.x * a.x + zz.y * a.y, ui = zz.x * a.y - zz.y * a.x;
                gr += w * ui;
                gi += -w * ur;
            }
        }
    }
    return make_float2(gr, gi);
}

}  // namespace cmpe
