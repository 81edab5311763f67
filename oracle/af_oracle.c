/*
 * FP64 CPU oracle for lens-aware differentiable-beamforming autofocus
 * (Frey et al., "Lens-Aware Differentiable Beamforming for In Vivo
 * Distributed Aberration Correction with Curvilinear Transducers").
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  Plain loops in the order of the
 * paper's equations, double precision, one thread, no blocking or fusion.
 * The same source built with -fopenmp runs the loops over elements, pixels
 * and patches on all host cores (the `omp` pragmas below; a plain build
 * ignores them).  Every such loop writes disjoint outputs, so that build
 * gives the single-threaded results bit for bit, except the ray adjoint,
 * whose per-node sums are then reduced across threads in a different order.
 *
 * Readings of passages the paper leaves open (each also listed in the
 * design notes of the repository):
 *  R1 Eq. 4 is printed as |x'| <= (F/2) z'; the default is the usual
 *     f-number form |x'| <= z'/(2F) with z' > 0 (apod_mode 0); the printed
 *     form is apod_mode 1.
 *  R2 Eq. 3 needs both neighbours; the end elements take the linear
 *     extrapolation theta_0 = 2 theta_1 - theta_2 (exact on a uniform arc).
 *  R3 CMPE (Sec. II-D defers to Simson et al.): per patch and per pair of
 *     common-midpoint subaperture images (i,j)~(i+1,j-1), z = sum_p
 *     B_ij conj(B_i+1,j-1); rho = |z| / sqrt(sum|B_ij|^2 sum|B_i+1,j-1|^2);
 *     mask m = [rho >= rho_thresh]; L_CMPE = sum m |arg z| / max(1, sum m).
 *     Pairs with j = i+1 (the reciprocal pair (i,i+1)~(i+1,i)) are skipped.
 *  R4 the correlation mask is a constant of the adjoint (stop-gradient).
 *  R5 discrete ray sum: |q - r| times the mean of the N+1 endpoint values.
 *  R6 bicubic = Keys cubic convolution (a = -1/2), clamp-to-edge indices.
 *  R7 exit points are found at the current c_med = mean(1/s) and held
 *     constant in the adjoint (Sec. III-A).
 *  R8 the update of Eq. 9 acts on the sound speed c, as printed, measured in
 *     km/s (c_unit = 1000 m/s).  Both the plain gradient step as printed
 *     (or_gd) and a step with Adam moments (or_adam) are provided; with Adam,
 *     Table II's learning rates are speed steps of 3 m/s (phantom) and 50 m/s
 *     (in vivo).
 *  R9 Eq. 10-11 ("physical units"): forward first differences and central
 *     second differences of c in km/s per mm (per mm^2), so Table II's
 *     kappa = 0.01 allows gradients up to 10 m/s per mm; N = number of
 *     difference terms of each family.
 *  R10 Psi(tau): linear interpolation at u = (tau - t0) fs, zero unless
 *     0 <= u < ns - 1.
 *  R11 the brute search over N_search lens points is replaced by a
 *     safeguarded Newton/bisection root solve of dT/dphi = 0.
 */
#include "af_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* threads of the OpenMP build (1 for the plain build) */
int or_omp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Sec. II-A, Eq. 3: element orientation from the neighbouring elements */
void or_element_angles(int ne, const double *ex, const double *ez, double *theta)
{
    for (int a = 1; a + 1 < ne; ++a)
        theta[a] = -atan((ez[a + 1] - ez[a - 1]) / (ex[a + 1] - ex[a - 1]));
    if (ne >= 3) {
        theta[0] = 2.0 * theta[1] - theta[2];                 /* R2 */
        theta[ne - 1] = 2.0 * theta[ne - 2] - theta[ne - 3];
    } else {
        for (int a = 0; a < ne; ++a) theta[a] = 0.0;
    }
}

/* Eq. 2 (rotation into the element frame) and Eq. 4 (constant f-number) */
int or_apod(const or_geom *g, const double *theta, int e, double x, double z)
{
    double c = cos(theta[e]), s = sin(theta[e]);
    double dx = x - g->ex[e], dz = z - g->ez[e];
    double xp = c * dx - s * dz;
    double zp = s * dx + c * dz;
    if (!(zp > 0.0)) return 0;
    if (g->apod_mode == 1) return fabs(xp) <= 0.5 * g->fnum * zp;
    return fabs(xp) <= zp / (2.0 * g->fnum);                   /* R1 */
}

/* Sec. III-A: c_med is the mean sound speed of the current map */
double or_mean_speed(const or_geom *g, const double *s)
{
    int n = g->nx * g->nz;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += 1.0 / s[k];
    return acc / n;
}

/* ------------------------------------------------------------------ */
/* Sec. III-A: dynamic grid of the global-speed sweep.  At speed c0 the echo of a
 * reflector at depth h below the lens arrives as from depth h c0 / c_true, so
 * the patch and its kernel spacing are stretched by c0 / c_ref about the lens
 * surface to keep observing the same echoes. */
void or_dynamic_pixels(const or_geom *g, double c0, double c_ref, double *px_out, double *pz_out)
{
    double scale = c0 / c_ref;
    int n = g->patch_npix;
    for (int P = 0; P < g->n_patch; ++P) {
        const double *xs = g->px + (size_t)P * n, *zs = g->pz + (size_t)P * n;
        double mx = 0.0, mz = 0.0;
        for (int q = 0; q < n; ++q) { mx += xs[q]; mz += zs[q]; }
        mx /= n;
        mz /= n;
        double nx, nz;                               /* moved patch centre */
        if (g->lens_mode == 2) {
            nx = mx;
            nz = g->lens_z + scale * (mz - g->lens_z);
        } else {
            double r = sqrt((mx - g->arc_cx) * (mx - g->arc_cx) + (mz - g->arc_cz) * (mz - g->arc_cz));
            double depth = r - g->lens_radius;
            double r_new = g->lens_radius + scale * depth;
            nx = g->arc_cx + (mx - g->arc_cx) * (r_new / r);
            nz = g->arc_cz + (mz - g->arc_cz) * (r_new / r);
        }
        for (int q = 0; q < n; ++q) {
            px_out[(size_t)P * n + q] = nx + scale * (xs[q] - mx);
            pz_out[(size_t)P * n + q] = nz + scale * (zs[q] - mz);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Eq. 8: two-layer path element -> lens surface point q(phi) -> pixel.
 * q(phi) = C + R_L (sin phi, cos phi).  With the element at polar
 * (Re, th_e) and the pixel at (rp, th_p) about the same centre C:
 *   d1(phi) = |q - r_e| , d2(phi) = |r - q|,
 *   T(phi)  = d1 / c_lens + d2 * sbar.
 * Chord lengths are written as sqrt((R1-R2)^2 + 4 R1 R2 sin^2(delta/2)). */
static void chord(double r1, double r2, double delta, double *d, double *d1, double *d2)
{
    double sh = sin(0.5 * delta);
    double len = sqrt((r1 - r2) * (r1 - r2) + 4.0 * r1 * r2 * sh * sh);
    double k = r1 * r2;
    *d = len;
    *d1 = k * sin(delta) / len;                                 /* d len / d phi */
    *d2 = k * cos(delta) / len - (k * sin(delta)) * (k * sin(delta)) / (len * len * len);
}

void or_exit_from_angle(const or_geom *g, int e, double phi, double *t_lens,
                        double *qx, double *qz)
{
    if (g->lens_mode == 2) {
        /* flat lens: the exit point is (phi, lens_z) */
        *qx = phi;
        *qz = g->lens_z;
        *t_lens = sqrt((phi - g->ex[e]) * (phi - g->ex[e]) + (g->lens_z - g->ez[e]) * (g->lens_z - g->ez[e]))
                  / g->c_lens;
        return;
    }
    double ux = g->ex[e] - g->arc_cx, uz = g->ez[e] - g->arc_cz;
    double re = sqrt(ux * ux + uz * uz), the = atan2(ux, uz);
    double d, d1, d2;
    chord(re, g->lens_radius, phi - the, &d, &d1, &d2);
    *t_lens = d / g->c_lens;
    *qx = g->arc_cx + g->lens_radius * sin(phi);
    *qz = g->arc_cz + g->lens_radius * cos(phi);
}

/* Flat lens (lens_mode 2, Eq. 7-8 with the lens surface the line z = lens_z):
 *   T(u) = sqrt((u - x_e)^2 + h1^2) / c_lens + sqrt((x - u)^2 + h2^2) * sbar,
 * h1 = lens_z - z_e > 0, h2 = z - lens_z > 0.  T'' > 0 and T' changes sign between
 * x_e and x, so the exit point is the root of T' there: safeguarded Newton. */
static int exit_point_flat(const or_geom *g, int e, double x, double z, double sbar, double *u_out)
{
    double xe = g->ex[e], h1 = g->lens_z - g->ez[e], h2 = z - g->lens_z;
    if (!(h1 > 0.0) || !(h2 > 0.0)) return -1;
    double lo = xe < x ? xe : x, hi = xe < x ? x : xe, u = xe;
    int it = 0;
    if (hi - lo > 0.0) {
        for (it = 1; it <= 200; ++it) {
            double d1 = sqrt((u - xe) * (u - xe) + h1 * h1), d2 = sqrt((x - u) * (x - u) + h2 * h2);
            double dT = (u - xe) / (g->c_lens * d1) - (x - u) * sbar / d2;
            double d2T = h1 * h1 / (g->c_lens * d1 * d1 * d1) + sbar * h2 * h2 / (d2 * d2 * d2);
            if (dT == 0.0) break;                /* Fermat: stationary point reached */
            if (dT < 0.0) lo = u; else hi = u;
            double un = u - dT / d2T;
            if (!(un >= lo && un <= hi)) un = 0.5 * (lo + hi);
            double step = fabs(un - u);
            u = un;
            if (step <= 1e-15 || hi - lo <= 1e-15) break;
        }
    }
    *u_out = u;
    return it;
}

int or_exit_point(const or_geom *g, int e, double x, double z, double sbar,
                  double *phi, double *t_lens, double *qx, double *qz)
{
    if (g->lens_mode == 2) {
        double u = g->ex[e];
        int it = exit_point_flat(g, e, x, z, sbar, &u);
        if (it < 0) return it;
        *phi = u;
        or_exit_from_angle(g, e, u, t_lens, qx, qz);
        return it;
    }
    double ux = g->ex[e] - g->arc_cx, uz = g->ez[e] - g->arc_cz;
    double re = sqrt(ux * ux + uz * uz), the = atan2(ux, uz);
    double vx = x - g->arc_cx, vz = z - g->arc_cz;
    double rp = sqrt(vx * vx + vz * vz), thp = atan2(vx, vz);
    double RL = g->lens_radius;
    int it = 0;
    if (rp <= RL) return -1;
    /* T is monotone outside [min(th_e, th_p), max(th_e, th_p)], so the
     * minimiser lies in that bracket where dT/dphi changes sign (R11). */
    double lo = the < thp ? the : thp, hi = the < thp ? thp : the;
    double f = the;
    if (hi - lo > 0.0) {
        for (it = 1; it <= 200; ++it) {
            double a, a1, a2, b, b1, b2;
            chord(re, RL, f - the, &a, &a1, &a2);
            chord(rp, RL, f - thp, &b, &b1, &b2);
            double dT = a1 / g->c_lens + b1 * sbar;
            double d2T = a2 / g->c_lens + b2 * sbar;
            if (dT == 0.0) break;                /* Fermat: stationary point reached */
            if (dT < 0.0) lo = f; else hi = f;
            double fn = (d2T > 0.0) ? f - dT / d2T : 0.5 * (lo + hi);
            if (!(fn >= lo && fn <= hi)) fn = 0.5 * (lo + hi);
            double step = fabs(fn - f);
            f = fn;
            if (step <= 1e-15 || hi - lo <= 1e-15) break;
        }
    }
    *phi = f;
    or_exit_from_angle(g, e, f, t_lens, qx, qz);
    return it;
}

/* ------------------------------------------------------------------ */
/* Sec. III-A bicubic interpolation (R6): Keys cubic-convolution kernel */
static double keys(double x)
{
    const double a = -0.5;
    x = fabs(x);
    if (x <= 1.0) return ((a + 2.0) * x - (a + 3.0)) * x * x + 1.0;
    if (x < 2.0) return ((a * x - 5.0 * a) * x + 8.0 * a) * x - 4.0 * a;
    return 0.0;
}

void or_keys_weights(double t, double w[4])
{
    w[0] = keys(1.0 + t);
    w[1] = keys(t);
    w[2] = keys(1.0 - t);
    w[3] = keys(2.0 - t);
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* the 16 (node index, weight) pairs of one bicubic evaluation */
static void bicubic_stencil(const or_geom *g, double x, double z, int idx[16], double w[16])
{
    double gx = (x - g->x0) / g->dx, gz = (z - g->z0) / g->dz;
    double fx = floor(gx), fz = floor(gz);
    int i0 = (int)fx, j0 = (int)fz;
    double wx[4], wz[4];
    or_keys_weights(gx - fx, wx);
    or_keys_weights(gz - fz, wz);
    for (int b = 0; b < 4; ++b) {
        int j = clampi(j0 - 1 + b, 0, g->nz - 1);
        for (int a = 0; a < 4; ++a) {
            int i = clampi(i0 - 1 + a, 0, g->nx - 1);
            idx[b * 4 + a] = j * g->nx + i;
            w[b * 4 + a] = wz[b] * wx[a];
        }
    }
}

double or_bicubic(const or_geom *g, const double *s, double x, double z)
{
    int idx[16];
    double w[16], acc = 0.0;
    bicubic_stencil(g, x, z, idx, w);
    for (int k = 0; k < 16; ++k) acc += w[k] * s[idx[k]];
    return acc;
}

/* Eq. 1 discretised as in Sec. III-A (R5): N segments, N+1 endpoints */
double or_ray_time(const or_geom *g, const double *s, double qx, double qz,
                   double x, double z)
{
    int n = g->nseg;
    double len = sqrt((x - qx) * (x - qx) + (z - qz) * (z - qz));
    double acc = 0.0;
    for (int k = 0; k <= n; ++k) {
        double f = (double)k / n;
        acc += or_bicubic(g, s, qx + f * (x - qx), qz + f * (z - qz));
    }
    return len * acc / (n + 1);
}

/* ------------------------------------------------------------------ */
/* Eq. 7-8 + Eq. 1: one-way delays for every (element, pixel) */
void or_delays(const or_geom *g, const double *s, const uint8_t *apod_in,
               const double *phi_in, double *T, uint8_t *apod, double *phi)
{
    int ne = g->ne, np = g->n_patch * g->patch_npix;
    double *theta = (double *)malloc(sizeof(double) * (ne > 0 ? ne : 1));
    or_element_angles(ne, g->ex, g->ez, theta);
    double sbar = 1.0 / or_mean_speed(g, s);
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < ne; ++e) {
        for (int p = 0; p < np; ++p) {
            size_t k = (size_t)e * np + p;
            double x = g->px[p], z = g->pz[p];
            int h = apod_in ? apod_in[k] : or_apod(g, theta, e, x, z);
            if (apod) apod[k] = (uint8_t)h;
            double tl = 0.0, qx = g->ex[e], qz = g->ez[e], f = 0.0;
            if (g->lens_mode == 0 || g->lens_mode == 2) {
                if (phi_in) {
                    f = phi_in[k];
                    or_exit_from_angle(g, e, f, &tl, &qx, &qz);
                } else {
                    or_exit_point(g, e, x, z, sbar, &f, &tl, &qx, &qz);
                }
            }
            if (phi) phi[k] = f;
            T[k] = tl + or_ray_time(g, s, qx, qz, x, z);
        }
    }
    free(theta);
}

/* ------------------------------------------------------------------ */
/* Eq. 5: delay-and-sum over subaperture blocks with phase rotation (R10) */
void or_das(const or_geom *g, const float *psi, const double *T, const uint8_t *apod,
            double *B)
{
    int ne = g->ne, np = g->n_patch * g->patch_npix, w = g->sub_width;
    int nsub = ne / w;
    memset(B, 0, sizeof(double) * 2 * (size_t)nsub * nsub * np);
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < np; ++p) {
        for (int t = 0; t < ne; ++t) {
            if (!apod[(size_t)t * np + p]) continue;
            for (int r = 0; r < ne; ++r) {
                if (!apod[(size_t)r * np + p]) continue;
                double tau = T[(size_t)t * np + p] + T[(size_t)r * np + p] + g->t_ttp;
                double u = (tau - g->t0) * g->fs;
                if (!(u >= 0.0 && u < g->ns - 1)) continue;
                int n = (int)floor(u);
                double fr = u - n;
                const float *tr = psi + 2 * ((size_t)t * ne + r) * g->ns;
                double re = tr[2 * n] + fr * ((double)tr[2 * n + 2] - tr[2 * n]);
                double im = tr[2 * n + 1] + fr * ((double)tr[2 * n + 3] - tr[2 * n + 1]);
                double ph = 2.0 * OR_PI * g->fd * tau;
                double c = cos(ph), sn = sin(ph);
                size_t b = (size_t)(t / w) * nsub + (r / w);
                B[2 * (b * np + p)] += re * c - im * sn;
                B[2 * (b * np + p) + 1] += re * sn + im * c;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* CMPE (R3): common-midpoint image pairs (i,j) ~ (i+1, j-1) */
int or_cmpe_pairs(const or_geom *g, int *pairs)
{
    int nsub = g->ne / g->sub_width, k = 0;
    for (int i = 0; i + 1 < nsub; ++i)
        for (int j = 1; j < nsub; ++j) {
            if (j == i + 1) continue;
            if (pairs) {
                pairs[2 * k] = i * nsub + j;
                pairs[2 * k + 1] = (i + 1) * nsub + (j - 1);
            }
            ++k;
        }
    return k;
}

double or_cmpe(const or_geom *g, const double *B, const uint8_t *mask_in,
               double *z, double *rho, uint8_t *mask, int *n_active)
{
    int np = g->n_patch * g->patch_npix;
    int npair = or_cmpe_pairs(g, NULL);
    int *pairs = (int *)malloc(sizeof(int) * 2 * (npair > 0 ? npair : 1));
    or_cmpe_pairs(g, pairs);
    size_t nt = (size_t)g->n_patch * npair;
    double *term = (double *)malloc(sizeof(double) * (nt ? nt : 1));   /* m |arg z| */
    uint8_t *mt = (uint8_t *)malloc(nt ? nt : 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int P = 0; P < g->n_patch; ++P) {
        for (int k = 0; k < npair; ++k) {
            const double *B1 = B + 2 * (size_t)pairs[2 * k] * np;
            const double *B2 = B + 2 * (size_t)pairs[2 * k + 1] * np;
            double zr = 0.0, zi = 0.0, e1 = 0.0, e2 = 0.0;
            for (int q = 0; q < g->patch_npix; ++q) {
                size_t p = (size_t)P * g->patch_npix + q;
                double ar = B1[2 * p], ai = B1[2 * p + 1];
                double br = B2[2 * p], bi = B2[2 * p + 1];
                zr += ar * br + ai * bi;           /* B1 conj(B2) */
                zi += ai * br - ar * bi;
                e1 += ar * ar + ai * ai;
                e2 += br * br + bi * bi;
            }
            size_t o = (size_t)P * npair + k;
            double den = sqrt(e1 * e2);
            double r = den > 0.0 ? sqrt(zr * zr + zi * zi) / den : 0.0;
            int m = mask_in ? mask_in[o] : (r >= g->rho_thresh);
            if (z) { z[2 * o] = zr; z[2 * o + 1] = zi; }
            if (rho) rho[o] = r;
            if (mask) mask[o] = (uint8_t)m;
            mt[o] = (uint8_t)m;
            term[o] = m ? fabs(atan2(zi, zr)) : 0.0;
        }
    }
    /* sum of the masked phase errors, patch by patch in pair order */
    double sum = 0.0;
    int m_count = 0;
    for (size_t o = 0; o < nt; ++o) {
        if (!mt[o]) continue;
        sum += term[o];
        ++m_count;
    }
    free(term);
    free(mt);
    free(pairs);
    if (n_active) *n_active = m_count;
    return sum / (m_count > 1 ? m_count : 1);
}

/* d L_CMPE / dB for L_CMPE = sum m |arg z| / max(1, M), mask held fixed (R4):
 *   d arg z = Im(conj(z) dz) / |z|^2, dz = conj(B2) dB1 + B1 conj(dB2)
 *   => G1 = w j z B2 / |z|^2,  G2 = -w j conj(z) B1 / |z|^2,
 *      w = sign(arg z) / max(1, M). */
void or_cmpe_adjoint(const or_geom *g, const double *B, const double *z,
                     const uint8_t *mask, int n_active, double *G)
{
    int np = g->n_patch * g->patch_npix;
    int nsub = g->ne / g->sub_width;
    int npair = or_cmpe_pairs(g, NULL);
    int *pairs = (int *)malloc(sizeof(int) * 2 * (npair > 0 ? npair : 1));
    or_cmpe_pairs(g, pairs);
    memset(G, 0, sizeof(double) * 2 * (size_t)nsub * nsub * np);
    double inv_m = 1.0 / (n_active > 1 ? n_active : 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int P = 0; P < g->n_patch; ++P) {
        for (int k = 0; k < npair; ++k) {
            size_t o = (size_t)P * npair + k;
            if (!mask[o]) continue;
            double zr = z[2 * o], zi = z[2 * o + 1];
            double ang = atan2(zi, zr);
            double sg = ang > 0.0 ? 1.0 : (ang < 0.0 ? -1.0 : 0.0);
            double mag2 = zr * zr + zi * zi;
            if (sg == 0.0 || mag2 == 0.0) continue;
            double w = sg * inv_m / mag2;
            size_t b1 = (size_t)pairs[2 * k], b2 = (size_t)pairs[2 * k + 1];
            for (int q = 0; q < g->patch_npix; ++q) {
                size_t p = (size_t)P * g->patch_npix + q;
                double ar = B[2 * (b1 * np + p)], ai = B[2 * (b1 * np + p) + 1];
                double br = B[2 * (b2 * np + p)], bi = B[2 * (b2 * np + p) + 1];
                /* z * B2 */
                double tr = zr * br - zi * bi, ti = zr * bi + zi * br;
                /* j (z B2) = (-ti, tr) */
                G[2 * (b1 * np + p)] += w * (-ti);
                G[2 * (b1 * np + p) + 1] += w * tr;
                /* conj(z) B1 */
                double ur = zr * ar + zi * ai, ui = zr * ai - zi * ar;
                /* -j (conj(z) B1) = (ui, -ur) */
                G[2 * (b2 * np + p)] += w * ui;
                G[2 * (b2 * np + p) + 1] += w * (-ur);
            }
        }
    }
    free(pairs);
}

/* d/dtau of Psi(tau) exp(j 2 pi fd tau) = exp(j phi) (fs dPsi/du + j 2 pi fd Psi);
 * dL/dtau = Re(conj(G) * that); tau = T_t + T_r + t_ttp feeds both T_t and T_r. */
void or_das_adjoint(const or_geom *g, const float *psi, const double *T,
                    const uint8_t *apod, const double *G, double *gT)
{
    int ne = g->ne, np = g->n_patch * g->patch_npix, w = g->sub_width;
    int nsub = ne / w;
    memset(gT, 0, sizeof(double) * (size_t)ne * np);
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < np; ++p) {
        for (int t = 0; t < ne; ++t) {
            if (!apod[(size_t)t * np + p]) continue;
            for (int r = 0; r < ne; ++r) {
                if (!apod[(size_t)r * np + p]) continue;
                double tau = T[(size_t)t * np + p] + T[(size_t)r * np + p] + g->t_ttp;
                double u = (tau - g->t0) * g->fs;
                if (!(u >= 0.0 && u < g->ns - 1)) continue;
                int n = (int)floor(u);
                double fr = u - n;
                const float *tr = psi + 2 * ((size_t)t * ne + r) * g->ns;
                double sr = (double)tr[2 * n + 2] - tr[2 * n];
                double si = (double)tr[2 * n + 3] - tr[2 * n + 1];
                double vr = tr[2 * n] + fr * sr, vi = tr[2 * n + 1] + fr * si;
                double ph = 2.0 * OR_PI * g->fd * tau;
                double c = cos(ph), sn = sin(ph);
                double wd = 2.0 * OR_PI * g->fd;
                /* fs * slope + j wd * v */
                double dr = g->fs * sr - wd * vi, di = g->fs * si + wd * vr;
                /* exp(j ph) * d */
                double er = c * dr - sn * di, ei = sn * dr + c * di;
                size_t b = (size_t)(t / w) * nsub + (r / w);
                double Gr = G[2 * (b * np + p)], Gi = G[2 * (b * np + p) + 1];
                double q = Gr * er + Gi * ei;          /* Re(conj(G) e) */
                gT[(size_t)t * np + p] += q;
                gT[(size_t)r * np + p] += q;
            }
        }
    }
}

/* transpose of the discretised ray integral: dT/ds_node = |q - r|/(N+1) sum_k W_node(x_k) */
void or_ray_adjoint(const or_geom *g, const double *s, const double *phi,
                    const uint8_t *apod, const double *gT, double *grad)
{
    (void)s;
    int ne = g->ne, np = g->n_patch * g->patch_npix, n = g->nseg;
    int ng = g->nx * g->nz;
    (void)ng;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : grad[:ng])
    for (int e = 0; e < ne; ++e) {
        for (int p = 0; p < np; ++p) {
            size_t k = (size_t)e * np + p;
            if (apod && !apod[k]) continue;
            double gv = gT[k];
            if (gv == 0.0) continue;
            double x = g->px[p], z = g->pz[p];
            double qx = g->ex[e], qz = g->ez[e], tl;
            if (g->lens_mode == 0 || g->lens_mode == 2) or_exit_from_angle(g, e, phi[k], &tl, &qx, &qz);
            double len = sqrt((x - qx) * (x - qx) + (z - qz) * (z - qz));
            double c = gv * len / (n + 1);
            for (int kk = 0; kk <= n; ++kk) {
                double f = (double)kk / n;
                int idx[16];
                double wt[16];
                bicubic_stencil(g, qx + f * (x - qx), qz + f * (z - qz), idx, wt);
                for (int m = 0; m < 16; ++m) grad[idx[m]] += c * wt[m];
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Eq. 10 (R_TV) and Eq. 11 (R_SV) with the deadzone D_k(x) = max(0, |x| - k) */
static double deadzone(double x, double k) { double a = fabs(x) - k; return a > 0.0 ? a : 0.0; }
static double deadzone_d(double x, double k)
{
    if (fabs(x) <= k) return 0.0;
    return x > 0.0 ? 1.0 : -1.0;
}

/* sound speed of a slowness value in the units of Eq. 9-11 (R8, R9) */
static double speed_u(const or_geom *g, double s) { return 1.0 / (s * g->c_unit); }

void or_regularizers(const or_geom *g, const double *s, double *rtv, double *rsv)
{
    int nx = g->nx, nz = g->nz;
    double hx = g->dx * 1e3, hz = g->dz * 1e3;       /* mm (R9) */
    double a = 0.0, b = 0.0;
    long na = 0, nb = 0;
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nx; ++i) {
            double c0 = speed_u(g, s[j * nx + i]);
            if (i + 1 < nx) { a += deadzone((speed_u(g, s[j * nx + i + 1]) - c0) / hx, g->kx1); ++na; }
            if (j + 1 < nz) { a += deadzone((speed_u(g, s[(j + 1) * nx + i]) - c0) / hz, g->kz1); ++na; }
            if (i >= 1 && i + 1 < nx) {
                double d = (speed_u(g, s[j * nx + i + 1]) - 2.0 * c0 + speed_u(g, s[j * nx + i - 1])) / (hx * hx);
                b += deadzone(d, g->kx2); ++nb;
            }
            if (j >= 1 && j + 1 < nz) {
                double d = (speed_u(g, s[(j + 1) * nx + i]) - 2.0 * c0 + speed_u(g, s[(j - 1) * nx + i])) / (hz * hz);
                b += deadzone(d, g->kz2); ++nb;
            }
        }
    *rtv = na ? a / na : 0.0;
    *rsv = nb ? b / nb : 0.0;
}

void or_regularizer_grad(const or_geom *g, const double *s, double *grad)
{
    int nx = g->nx, nz = g->nz;
    double hx = g->dx * 1e3, hz = g->dz * 1e3;
    long na = (long)(nx - 1) * nz + (long)nx * (nz - 1);
    long nb = (long)(nx > 2 ? nx - 2 : 0) * nz + (long)nx * (nz > 2 ? nz - 2 : 0);
    if (nx < 2) na = (long)nx * (nz - 1);
    if (nz < 2) na = (long)(nx - 1) * nz;
    int n = nx * nz;
    double *gc = (double *)calloc((size_t)n, sizeof(double));   /* dR/dc, c in c_unit */
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            double c0 = speed_u(g, s[k]);
            if (na > 0 && i + 1 < nx) {
                double d = deadzone_d((speed_u(g, s[k + 1]) - c0) / hx, g->kx1) * g->w1 / (na * hx);
                gc[k + 1] += d; gc[k] -= d;
            }
            if (na > 0 && j + 1 < nz) {
                double d = deadzone_d((speed_u(g, s[k + nx]) - c0) / hz, g->kz1) * g->w1 / (na * hz);
                gc[k + nx] += d; gc[k] -= d;
            }
            if (nb > 0 && i >= 1 && i + 1 < nx) {
                double v = (speed_u(g, s[k + 1]) - 2.0 * c0 + speed_u(g, s[k - 1])) / (hx * hx);
                double d = deadzone_d(v, g->kx2) * g->w2 / (nb * hx * hx);
                gc[k + 1] += d; gc[k - 1] += d; gc[k] -= 2.0 * d;
            }
            if (nb > 0 && j >= 1 && j + 1 < nz) {
                double v = (speed_u(g, s[k + nx]) - 2.0 * c0 + speed_u(g, s[k - nx])) / (hz * hz);
                double d = deadzone_d(v, g->kz2) * g->w2 / (nb * hz * hz);
                gc[k + nx] += d; gc[k - nx] += d; gc[k] -= 2.0 * d;
            }
        }
    for (int k = 0; k < n; ++k) grad[k] += -gc[k] / (g->c_unit * s[k] * s[k]);   /* c = 1/(c_unit s) */
    free(gc);
}

/* ------------------------------------------------------------------ */
/* Eq. 12: L = L_CMPE + w1 R_TV + w2 R_SV, and its gradient (Fig. 1g) */
double or_loss_grad(const or_geom *g, const float *psi, const double *s,
                    const uint8_t *apod_in, const uint8_t *mask_in,
                    const double *phi_in, double *grad, double parts[4],
                    uint8_t *mask_out, int *n_active)
{
    int ne = g->ne, np = g->n_patch * g->patch_npix;
    int nsub = ne / g->sub_width;
    int npair = or_cmpe_pairs(g, NULL);
    size_t nep = (size_t)ne * np, nb = (size_t)nsub * nsub * np;
    size_t nzp = (size_t)g->n_patch * npair;
    double *T = (double *)malloc(sizeof(double) * (nep ? nep : 1));
    double *phi = (double *)malloc(sizeof(double) * (nep ? nep : 1));
    uint8_t *apod = (uint8_t *)malloc(nep ? nep : 1);
    double *B = (double *)malloc(sizeof(double) * 2 * (nb ? nb : 1));
    double *z = (double *)malloc(sizeof(double) * 2 * (nzp ? nzp : 1));
    uint8_t *mask = (uint8_t *)malloc(nzp ? nzp : 1);
    int M = 0;

    or_delays(g, s, apod_in, phi_in, T, apod, phi);
    or_das(g, psi, T, apod, B);
    double lc = or_cmpe(g, B, mask_in, z, NULL, mask, &M);
    double rtv, rsv;
    or_regularizers(g, s, &rtv, &rsv);
    double L = lc + g->w1 * rtv + g->w2 * rsv;
    if (parts) { parts[0] = L; parts[1] = lc; parts[2] = rtv; parts[3] = rsv; }
    if (mask_out) memcpy(mask_out, mask, nzp);
    if (n_active) *n_active = M;

    if (grad) {
        double *G = (double *)malloc(sizeof(double) * 2 * (nb ? nb : 1));
        double *gT = (double *)malloc(sizeof(double) * (nep ? nep : 1));
        memset(grad, 0, sizeof(double) * (size_t)g->nx * g->nz);
        or_cmpe_adjoint(g, B, z, mask, M, G);
        or_das_adjoint(g, psi, T, apod, G, gT);
        or_ray_adjoint(g, s, phi, apod, gT, grad);
        or_regularizer_grad(g, s, grad);
        free(G);
        free(gT);
    }
    free(T); free(phi); free(apod); free(B); free(z); free(mask);
    return L;
}

/* Eq. 9 as printed: one gradient step on c = 1 / (s c_unit), dL/dc = -dL/ds c_unit s^2 */
void or_gd(int n, double *s, const double *grad, double lr, double c_unit)
{
    for (int k = 0; k < n; ++k) {
        double c = 1.0 / (s[k] * c_unit);
        double gc = -grad[k] * c_unit * s[k] * s[k];
        s[k] = 1.0 / ((c - lr * gc) * c_unit);
    }
}

/* Adam on the sound speed c = 1 / (s c_unit) (R8); with beta1 = beta2 = 0 each
 * step is lr times the sign of the Eq. 9 step.  dL/dc = dL/ds ds/dc with
 * ds/dc = -c_unit s^2. */
void or_adam(int n, double *s, const double *grad, double *m, double *v, int step,
             double lr, double beta1, double beta2, double eps, double c_unit)
{
    double bc1 = 1.0 - pow(beta1, step), bc2 = 1.0 - pow(beta2, step);
    for (int k = 0; k < n; ++k) {
        double gc = -grad[k] * c_unit * s[k] * s[k];
        m[k] = beta1 * m[k] + (1.0 - beta1) * gc;
        v[k] = beta2 * v[k] + (1.0 - beta2) * gc * gc;
        double mh = m[k] / bc1, vh = v[k] / bc2;
        double c = 1.0 / (s[k] * c_unit) - lr * mh / (sqrt(vh) + eps);
        s[k] = 1.0 / (c * c_unit);
    }
}
