/*
 * Seeded synthetic full-synthetic-aperture acquisitions (input generator).
 *
 * This file models the acquisition physics that produces the demodulated
 * channel data: point scatterers in a layered medium behind a curvilinear
 * array with a lens.  It holds none of the autofocusing method's arithmetic
 * (no slowness grid, no bicubic ray sum, no beamforming, no loss): the one-way
 * travel time of the "true" medium is an exact piecewise-constant line
 * integral through analytic layer interfaces, the lens exit point is found by
 * golden-section search, and the echo of each scatterer is the exact complex
 * baseband of a Gaussian-windowed tone.  Both the CUDA library and the oracle
 * consume what this file writes; neither is called from here.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SY_PI 3.14159265358979323846
#define SY_MAX_IF 8

typedef struct {
    int n_if;                         /* interfaces between n_if + 1 layers, top to bottom */
    double base[SY_MAX_IF];           /* z of interface i: base + amp sin(2 pi x / period + phase) */
    double amp[SY_MAX_IF];
    double period[SY_MAX_IF];
    double phase[SY_MAX_IF];
    double slow[SY_MAX_IF + 1];       /* slowness of each layer (s/m) */
} sy_medium;

static double if_z(const sy_medium *m, int i, double x)
{
    if (m->amp[i] == 0.0) return m->base[i];
    return m->base[i] + m->amp[i] * sin(2.0 * SY_PI * x / m->period[i] + m->phase[i]);
}

static int layer_of(const sy_medium *m, double x, double z)
{
    int l = 0;
    for (int i = 0; i < m->n_if; ++i)
        if (z > if_z(m, i, x)) l = i + 1;
    return l;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* exact travel time of the straight segment (ax,az) -> (bx,bz) through the layers */
double sy_segment_time(const sy_medium *m, double ax, double az, double bx, double bz)
{
    double cuts[2 + SY_MAX_IF * 48];
    int nc = 0;
    cuts[nc++] = 0.0;
    double dx = bx - ax, dz = bz - az;
    for (int i = 0; i < m->n_if; ++i) {
        if (m->amp[i] == 0.0) {
            if (dz != 0.0) {
                double t = (m->base[i] - az) / dz;
                if (t > 0.0 && t < 1.0) cuts[nc++] = t;
            }
            continue;
        }
        /* restrict to the part of the segment inside the interface's z band */
        double zlo = m->base[i] - fabs(m->amp[i]), zhi = m->base[i] + fabs(m->amp[i]);
        double t0 = 0.0, t1 = 1.0;
        if (dz != 0.0) {
            double ta = (zlo - az) / dz, tb = (zhi - az) / dz;
            if (ta > tb) { double q = ta; ta = tb; tb = q; }
            t0 = ta > 0.0 ? ta : 0.0;
            t1 = tb < 1.0 ? tb : 1.0;
        } else if (az < zlo || az > zhi) {
            continue;
        }
        if (t1 <= t0) continue;
        const int ns = 24;
        double tp = t0, hp = az + tp * dz - if_z(m, i, ax + tp * dx);
        for (int k = 1; k <= ns; ++k) {
            double tc = t0 + (t1 - t0) * k / ns;
            double hc = az + tc * dz - if_z(m, i, ax + tc * dx);
            if ((hp < 0.0) != (hc < 0.0)) {
                double lo = tp, hi = tc, hlo = hp;
                for (int it = 0; it < 48; ++it) {
                    double mid = 0.5 * (lo + hi);
                    double hm = az + mid * dz - if_z(m, i, ax + mid * dx);
                    if ((hm < 0.0) == (hlo < 0.0)) { lo = mid; hlo = hm; } else hi = mid;
                }
                double t = 0.5 * (lo + hi);
                if (t > 0.0 && t < 1.0 && nc < 1 + SY_MAX_IF * 48) cuts[nc++] = t;
            }
            tp = tc; hp = hc;
        }
    }
    cuts[nc++] = 1.0;
    qsort(cuts, (size_t)nc, sizeof(double), cmp_double);
    double len = sqrt(dx * dx + dz * dz), acc = 0.0;
    for (int k = 0; k + 1 < nc; ++k) {
        double tm = 0.5 * (cuts[k] + cuts[k + 1]);
        int l = layer_of(m, ax + tm * dx, az + tm * dz);
        acc += (cuts[k + 1] - cuts[k]) * m->slow[l];
    }
    return acc * len;
}

/* one-way time element -> scatterer through a flat lens whose outer surface is the
 * line z = lz: the exit point minimises lens time + straight distance in the top layer
 * (Snell at the lens surface).  The lens-side angle is below asin(c_lens / c_tissue),
 * so the exit point lies within a few lens thicknesses of the element foot;
 * golden-section search there. */
static double oneway_flat(const sy_medium *m, double ex, double ez, double lz, double c_lens,
                          double kx, double kz)
{
    double h1 = lz - ez, h2 = kz - lz;
    double s_top = m->slow[layer_of(m, ex, ez)];
    double a = ex < kx ? ex : kx, b = ex < kx ? kx : ex;
    double w = 4.0 * h1 + 1e-4;
    if (a < ex - w) a = ex - w;
    if (b > ex + w) b = ex + w;
    const double gr = 0.6180339887498949;
    double c1 = b - gr * (b - a), c2 = a + gr * (b - a);
#define SY_TF(x) (hypot((x) - ex, h1) / c_lens + hypot(kx - (x), h2) * s_top)
    double f1 = SY_TF(c1), f2 = SY_TF(c2);
    /* an exit-point error d only changes the time by O(d^2): 1e-12 m is ample */
    for (int it = 0; it < 80 && b - a > 1e-12; ++it) {
        if (f1 < f2) { b = c2; c2 = c1; f2 = f1; c1 = b - gr * (b - a); f1 = SY_TF(c1); }
        else { a = c1; c1 = c2; f1 = f2; c2 = a + gr * (b - a); f2 = SY_TF(c2); }
    }
#undef SY_TF
    double qx = 0.5 * (a + b);
    return hypot(qx - ex, h1) / c_lens + sy_segment_time(m, qx, lz, kx, kz);
}

/* one-way time element -> scatterer: lens leg (c_lens) + tissue leg through the layers.
 * lens_kind 0: no lens; 1: curved lens (arc of radius RL about (cx, cz)); 2: flat lens
 * (line z = lz).  For the curved lens the exit point minimises lens time + straight
 * distance in the top layer (Snell at the lens surface), found by golden-section
 * search between the element and the scatterer angles. */
static double oneway(const sy_medium *m, double ex, double ez, double cx, double cz,
                     double RL, double lz, double c_lens, int lens_kind, double kx, double kz)
{
    if (lens_kind == 0) return sy_segment_time(m, ex, ez, kx, kz);
    if (lens_kind == 2) return oneway_flat(m, ex, ez, lz, c_lens, kx, kz);
    double the = atan2(ex - cx, ez - cz), thk = atan2(kx - cx, kz - cz);
    double s_top = m->slow[layer_of(m, ex, ez)];
    double a = the < thk ? the : thk, b = the < thk ? thk : the;
    /* the lens leg leaves within a few lens thicknesses of the element foot */
    double w = 4.0 * (RL - hypot(ex - cx, ez - cz) + 1e-4) / RL;
    if (a < the - w) a = the - w;
    if (b > the + w) b = the + w;
    const double gr = 0.6180339887498949;
    double c1 = b - gr * (b - a), c2 = a + gr * (b - a);
#define SY_T(ph) (hypot(cx + RL * sin(ph) - ex, cz + RL * cos(ph) - ez) / c_lens + \
                  hypot(kx - cx - RL * sin(ph), kz - cz - RL * cos(ph)) * s_top)
    double f1 = SY_T(c1), f2 = SY_T(c2);
    /* an exit-angle error d only changes the time by O(d^2): 1e-9 rad is ample */
    for (int it = 0; it < 80 && b - a > 1e-9; ++it) {
        if (f1 < f2) { b = c2; c2 = c1; f2 = f1; c1 = b - gr * (b - a); f1 = SY_T(c1); }
        else { a = c1; c1 = c2; f1 = f2; c2 = a + gr * (b - a); f2 = SY_T(c2); }
    }
#undef SY_T
    double ph = 0.5 * (a + b);
    double qx = cx + RL * sin(ph), qz = cz + RL * cos(ph);
    return hypot(qx - ex, qz - ez) / c_lens + sy_segment_time(m, qx, qz, kx, kz);
}

/* T[e][k] one-way times for every element and scatterer */
void sy_oneway_times(int ne, const double *ex, const double *ez, double cx, double cz,
                     double RL, double lz, double c_lens, int lens_kind, const sy_medium *m,
                     int nk, const double *kx, const double *kz, double *T)
{
    long total = (long)ne * nk;
#pragma omp parallel for schedule(dynamic, 4096)
    for (long idx = 0; idx < total; ++idx) {
        int e = (int)(idx / nk), k = (int)(idx % nk);
        T[idx] = oneway(m, ex[e], ez[e], cx, cz, RL, lz, c_lens, lens_kind, kx[k], kz[k]);
    }
}

/* Psi[t][r][n] (complex64 interleaved) = sum_k a_k g(t_n - tau) exp(-j 2 pi fd tau),
 * tau = T[t][k] + T[r][k] + t_ttp, t_n = t0 + n / fs, g Gaussian of std sigma cut at
 * +-4 sigma.  Reciprocity Psi[t][r] = Psi[r][t] holds exactly by construction. */
void sy_echoes(int ne, int nk, const double *T, const double *amp, int ns, double fs,
               double fd, double t0, double t_ttp, double sigma, float *psi)
{
    long npair = (long)ne * (ne + 1) / 2;
    double delta = 1.0 / (fs * sigma);
    double cdec = exp(-delta * delta);
    /* exp(-j 2 pi fd tau) = P[t][k] P[r][k] exp(-j 2 pi fd t_ttp) */
    double *P = (double *)malloc(sizeof(double) * 2 * (size_t)ne * nk);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)ne * nk; ++i) {
        double ph = -2.0 * SY_PI * fd * T[i];
        P[2 * i] = cos(ph);
        P[2 * i + 1] = sin(ph);
    }
    double c0 = cos(-2.0 * SY_PI * fd * t_ttp), s0 = sin(-2.0 * SY_PI * fd * t_ttp);
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)ns);
#pragma omp for schedule(dynamic, 1)
        for (long pi = 0; pi < npair; ++pi) {
            /* unrank pi -> (t, r) with t <= r */
            int t = 0;
            long rem = pi;
            while (rem >= ne - t) { rem -= ne - t; ++t; }
            int r = t + (int)rem;
            memset(acc, 0, sizeof(double) * 2 * (size_t)ns);
            const double *Tt = T + (size_t)t * nk, *Tr = T + (size_t)r * nk;
            const double *Pt = P + 2 * (size_t)t * nk, *Pr = P + 2 * (size_t)r * nk;
            for (int k = 0; k < nk; ++k) {
                double tau = Tt[k] + Tr[k] + t_ttp;
                double u = (tau - t0) * fs;
                int n0 = (int)ceil(u - 4.0 * sigma * fs);
                int n1 = (int)floor(u + 4.0 * sigma * fs);
                if (n0 < 0) n0 = 0;
                if (n1 > ns - 1) n1 = ns - 1;
                if (n0 > n1) continue;
                double x = ((t0 + n0 / fs) - tau) / sigma;
                double env = amp[k] * exp(-0.5 * x * x);
                double ratio = exp(-x * delta - 0.5 * delta * delta);
                double pr = Pt[2 * k] * Pr[2 * k] - Pt[2 * k + 1] * Pr[2 * k + 1];
                double pim = Pt[2 * k] * Pr[2 * k + 1] + Pt[2 * k + 1] * Pr[2 * k];
                double c = pr * c0 - pim * s0, s = pr * s0 + pim * c0;
                for (int n = n0; n <= n1; ++n) {
                    acc[2 * n] += env * c;
                    acc[2 * n + 1] += env * s;
                    env *= ratio;
                    ratio *= cdec;
                }
            }
            float *o1 = psi + 2 * ((size_t)t * ne + r) * ns;
            float *o2 = psi + 2 * ((size_t)r * ne + t) * ns;
            for (int n = 0; n < 2 * ns; ++n) {
                o1[n] = (float)acc[n];
                o2[n] = (float)acc[n];
            }
        }
        free(acc);
    }
    free(P);
}

int sy_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
