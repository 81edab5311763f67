/*
 * Seeded synthetic full-synthetic-aperture acquisitions on the GPU (input
 * generator, test and benchmark fixture).
 *
 * The same acquisition physics as synth.c, for acquisitions too large for
 * the host (10 scatterers per resolution cell of the 128-element array is
 * about 7e5 scatterers):
 *   sy_gpu_oneway_times  true one-way times element -> scatterer: lens leg
 *                        with the exit point found by golden-section search
 *                        (Snell at the lens surface against the top layer),
 *                        tissue leg as the exact piecewise-constant integral
 *                        through the analytic layer interfaces, in float64;
 *   sy_gpu_echoes        Psi[t][r][n] = sum_k a_k g(t_n - tau) exp(-j 2 pi fd tau),
 *                        tau = T[t][k] + T[r][k] + t_ttp, g a Gaussian of std
 *                        sigma cut at +-4 sigma; pairs t <= r are computed and
 *                        written to both [t][r] and [r][t] (exact reciprocity).
 * It holds none of the autofocusing method's arithmetic (no slowness grid, no
 * bicubic ray sum, no beamforming, no loss); the library and the oracle read
 * what it writes and are never called from here.  The echoes accumulate in
 * float (synth.c accumulates in double), about 1e-6 relative.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define SY_MAX_IF 8
#define SY_GPU_MAX_CUTS 64            /* interface crossings of one segment (checked) */

typedef struct {
    int n_if;
    double base[SY_MAX_IF];
    double amp[SY_MAX_IF];
    double period[SY_MAX_IF];
    double phase[SY_MAX_IF];
    double slow[SY_MAX_IF + 1];
} sy_medium;

namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ double if_z(const sy_medium &m, int i, double x)
{
    if (m.amp[i] == 0.0) return m.base[i];
    return m.base[i] + m.amp[i] * sin(2.0 * kPi * x / m.period[i] + m.phase[i]);
}

__device__ int layer_of(const sy_medium &m, double x, double z)
{
    int l = 0;
    for (int i = 0; i < m.n_if; ++i)
        if (z > if_z(m, i, x)) l = i + 1;
    return l;
}

// exact travel time of the straight segment a -> b through the layers: the
// segment is cut where it crosses an interface (flat: closed form; wavy: sign
// changes on 24 samples of the interface's z band, refined by 48 bisections),
// and each piece is charged the slowness of the layer at its midpoint
__device__ double segment_time(const sy_medium &m, double ax, double az, double bx, double bz, int *overflow)
{
    double cuts[SY_GPU_MAX_CUTS + 2];
    int nc = 0;
    cuts[nc++] = 0.0;
    const double dx = bx - ax, dz = bz - az;
    for (int i = 0; i < m.n_if; ++i) {
        if (m.amp[i] == 0.0) {
            if (dz != 0.0) {
                const double t = (m.base[i] - az) / dz;
                if (t > 0.0 && t < 1.0) {
                    if (nc <= SY_GPU_MAX_CUTS) cuts[nc++] = t; else *overflow = 1;
                }
            }
            continue;
        }
        const double zlo = m.base[i] - fabs(m.amp[i]), zhi = m.base[i] + fabs(m.amp[i]);
        double t0 = 0.0, t1 = 1.0;
        if (dz != 0.0) {
            double ta = (zlo - az) / dz, tb = (zhi - az) / dz;
            if (ta > tb) { const double q = ta; ta = tb; tb = q; }
            t0 = ta > 0.0 ? ta : 0.0;
            t1 = tb < 1.0 ? tb : 1.0;
        } else if (az < zlo || az > zhi) {
            continue;
        }
        if (t1 <= t0) continue;
        const int ns = 24;
        double tp = t0, hp = az + tp * dz - if_z(m, i, ax + tp * dx);
        for (int k = 1; k <= ns; ++k) {
            const double tc = t0 + (t1 - t0) * k / ns;
            const double hc = az + tc * dz - if_z(m, i, ax + tc * dx);
            if ((hp < 0.0) != (hc < 0.0)) {
                double lo = tp, hi = tc, hlo = hp;
                for (int it = 0; it < 48; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    const double hm = az + mid * dz - if_z(m, i, ax + mid * dx);
                    if ((hm < 0.0) == (hlo < 0.0)) { lo = mid; hlo = hm; } else hi = mid;
                }
                const double t = 0.5 * (lo + hi);
                if (t > 0.0 && t < 1.0) {
                    if (nc <= SY_GPU_MAX_CUTS) cuts[nc++] = t; else *overflow = 1;
                }
            }
            tp = tc;
            hp = hc;
        }
    }
    cuts[nc++] = 1.0;
    for (int a = 1; a < nc; ++a) {                 // insertion sort of the few cuts
        const double v = cuts[a];
        int b = a - 1;
        while (b >= 0 && cuts[b] > v) { cuts[b + 1] = cuts[b]; --b; }
        cuts[b + 1] = v;
    }
    const double len = sqrt(dx * dx + dz * dz);
    double acc = 0.0;
    for (int k = 0; k + 1 < nc; ++k) {
        const double tm = 0.5 * (cuts[k] + cuts[k + 1]);
        acc += (cuts[k + 1] - cuts[k]) * m.slow[layer_of(m, ax + tm * dx, az + tm * dz)];
    }
    return acc * len;
}

struct LensArgs {
    double cx, cz, RL, lz, c_lens;
    int kind;                       // 0 no lens, 1 curved lens, 2 flat lens
};

// golden-section search of the exit point (an exit error d changes the time by O(d^2))
__device__ double oneway(const sy_medium &m, const LensArgs &L, double ex, double ez, double kx, double kz,
                         int *overflow)
{
    const double gr = 0.6180339887498949;
    if (L.kind == 0) return segment_time(m, ex, ez, kx, kz, overflow);
    const double s_top = m.slow[layer_of(m, ex, ez)];
    if (L.kind == 2) {
        const double h1 = L.lz - ez, h2 = kz - L.lz;
        double a = ex < kx ? ex : kx, b = ex < kx ? kx : ex;
        const double w = 4.0 * h1 + 1e-4;
        if (a < ex - w) a = ex - w;
        if (b > ex + w) b = ex + w;
        auto T = [&](double x) { return hypot(x - ex, h1) / L.c_lens + hypot(kx - x, h2) * s_top; };
        double c1 = b - gr * (b - a), c2 = a + gr * (b - a), f1 = T(c1), f2 = T(c2);
        for (int it = 0; it < 80 && b - a > 1e-12; ++it) {
            if (f1 < f2) { b = c2; c2 = c1; f2 = f1; c1 = b - gr * (b - a); f1 = T(c1); }
            else { a = c1; c1 = c2; f1 = f2; c2 = a + gr * (b - a); f2 = T(c2); }
        }
        const double qx = 0.5 * (a + b);
        return hypot(qx - ex, h1) / L.c_lens + segment_time(m, qx, L.lz, kx, kz, overflow);
    }
    const double the = atan2(ex - L.cx, ez - L.cz), thk = atan2(kx - L.cx, kz - L.cz);
    double a = the < thk ? the : thk, b = the < thk ? thk : the;
    const double w = 4.0 * (L.RL - hypot(ex - L.cx, ez - L.cz) + 1e-4) / L.RL;
    if (a < the - w) a = the - w;
    if (b > the + w) b = the + w;
    auto T = [&](double ph) {
        double sp, cp;
        sincos(ph, &sp, &cp);
        return hypot(L.cx + L.RL * sp - ex, L.cz + L.RL * cp - ez) / L.c_lens +
               hypot(kx - L.cx - L.RL * sp, kz - L.cz - L.RL * cp) * s_top;
    };
    double c1 = b - gr * (b - a), c2 = a + gr * (b - a), f1 = T(c1), f2 = T(c2);
    for (int it = 0; it < 80 && b - a > 1e-9; ++it) {
        if (f1 < f2) { b = c2; c2 = c1; f2 = f1; c1 = b - gr * (b - a); f1 = T(c1); }
        else { a = c1; c1 = c2; f1 = f2; c2 = a + gr * (b - a); f2 = T(c2); }
    }
    const double ph = 0.5 * (a + b);
    const double qx = L.cx + L.RL * sin(ph), qz = L.cz + L.RL * cos(ph);
    return hypot(qx - ex, qz - ez) / L.c_lens + segment_time(m, qx, qz, kx, kz, overflow);
}

__global__ void oneway_kernel(sy_medium m, LensArgs L, int ne, long long nk, const double *__restrict__ ex,
                              const double *__restrict__ ez, const double *__restrict__ kx,
                              const double *__restrict__ kz, double *__restrict__ T, int *__restrict__ flag)
{
    const long long total = (long long)ne * nk;
    int overflow = 0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(idx / nk);
        const long long k = idx - (long long)e * nk;
        T[idx] = oneway(m, L, ex[e], ez[e], kx[k], kz[k], &overflow);
    }
    if (overflow) atomicOr(flag, 1);
}

// Echo synthesis.  A CTA owns the traces of one transmit t and kRecv consecutive
// receivers r >= t in shared memory; its threads walk the scatterers, each adding
// its Gaussian-windowed, phase-rotated echo into the traces with shared-memory
// float atomics.  The window of a scatterer spans 8 sigma fs + 1 samples.
constexpr int kRecv = 4;
constexpr int kEchoThreads = 512;

__global__ void __launch_bounds__(kEchoThreads) echo_kernel(int ne, long long nk, const double *__restrict__ T,
                                                            const double *__restrict__ amp, int ns, double fs,
                                                            double fd, double t0, double t_ttp, double sigma,
                                                            float2 *__restrict__ psi)
{
    extern __shared__ float2 acc[];                 // [kRecv][ns]
    const int t = blockIdx.y;
    const int r0 = blockIdx.x * kRecv;
    if (r0 + kRecv - 1 < t) return;                 // whole block below the diagonal
    for (int i = threadIdx.x; i < kRecv * ns; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const double half = 4.0 * sigma * fs;           // window half width in samples
    const double inv_sfs = 1.0 / (sigma * fs);
    const double *Tt = T + (size_t)t * nk;
    for (long long k = threadIdx.x; k < nk; k += blockDim.x) {
        const double tt = Tt[k] + t_ttp;
        const double a = amp[k];
#pragma unroll
        for (int q = 0; q < kRecv; ++q) {
            const int r = r0 + q;
            if (r < t || r >= ne) continue;
            const double tau = tt + T[(size_t)r * nk + k];
            const double u = (tau - t0) * fs;
            int n0 = (int)ceil(u - half), n1 = (int)floor(u + half);
            if (n0 < 0) n0 = 0;
            if (n1 > ns - 1) n1 = ns - 1;
            if (n0 > n1) continue;
            // exp(-j 2 pi fd tau): the whole cycles of fd tau are dropped in float64
            const double cyc = fd * tau;
            float sp, cp;
            sincospif(-2.0f * (float)(cyc - floor(cyc)), &sp, &cp);
            float2 *tr = acc + q * ns;
            for (int n = n0; n <= n1; ++n) {
                const float x = (float)(((double)n - u) * inv_sfs);
                const float env = (float)a * expf(-0.5f * x * x);
                atomicAdd(&tr[n].x, env * cp);
                atomicAdd(&tr[n].y, env * sp);
            }
        }
    }
    __syncthreads();
    for (int q = 0; q < kRecv; ++q) {
        const int r = r0 + q;
        if (r < t || r >= ne) continue;
        float2 *o1 = psi + ((size_t)t * ne + r) * ns;
        float2 *o2 = psi + ((size_t)r * ne + t) * ns;
        for (int n = threadIdx.x; n < ns; n += blockDim.x) {
            o1[n] = acc[q * ns + n];
            o2[n] = acc[q * ns + n];
        }
    }
}

}  // namespace

extern "C" {

/* T[e][k] (device, float64) for every element and scatterer; every pointer is
 * device memory.  lens_kind 0 no lens, 1 curved lens (arc of radius RL about
 * (cx, cz)), 2 flat lens (line z = lz).  Returns a cudaError_t value, or -1 if
 * a segment crossed the interfaces more than SY_GPU_MAX_CUTS times.
 * Synchronises the device. */
int sy_gpu_oneway_times(int ne, const double *d_ex, const double *d_ez, double cx, double cz, double RL,
                        double lz, double c_lens, int lens_kind, const sy_medium *m, long long nk,
                        const double *d_kx, const double *d_kz, double *d_T)
{
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e != cudaSuccess) return (int)e;
    cudaMemset(flag, 0, sizeof(int));
    LensArgs L{cx, cz, RL, lz, c_lens, lens_kind};
    const long long total = (long long)ne * nk;
    const int threads = 128;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > (1 << 20)) blocks = 1 << 20;
    if (blocks < 1) blocks = 1;
    oneway_kernel<<<(unsigned)blocks, threads>>>(*m, L, ne, nk, d_ex, d_ez, d_kx, d_kz, d_T, flag);
    e = cudaDeviceSynchronize();
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e != cudaSuccess) return (int)e;
    return h ? -1 : 0;
}

/* Psi[t][r][n] (device, interleaved float32 complex) from the one-way times
 * d_T[e][k] and amplitudes d_amp[k] (device, float64).  Returns a cudaError_t
 * value.  Synchronises the device. */
int sy_gpu_echoes(int ne, long long nk, const double *d_T, const double *d_amp, int ns, double fs, double fd,
                  double t0, double t_ttp, double sigma, float *d_psi)
{
    const size_t smem = (size_t)kRecv * ns * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(echo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    dim3 grid((ne + kRecv - 1) / kRecv, ne);
    echo_kernel<<<grid, kEchoThreads, smem>>>(ne, nk, d_T, d_amp, ns, fs, fd, t0, t_ttp, sigma,
                                              reinterpret_cast<float2 *>(d_psi));
    return (int)cudaDeviceSynchronize();
}

}  // extern "C"
