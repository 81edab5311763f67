/*
 * FP64 CPU oracle for lens-aware differentiable-beamforming autofocus.
 *
 * TEST INFRASTRUCTURE ONLY.  This header and af_oracle.c are the plain,
 * slow, single-threaded reference that the CUDA library is checked against.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library, and it never reads anything the CUDA library produced except the
 * three discrete decisions a parity test may inject (apodization bits, CMPE
 * correlation-mask bits and frozen lens exit angles), each documented below.
 *
 * Conventions: SI units (m, s, s/m), z grows into the tissue, complex
 * numbers are interleaved (re, im) pairs of doubles.
 */
#ifndef AF_ORACLE_H
#define AF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    /* transducer array, Sec. II-A: element positions r_a */
    int ne;
    const double *ex, *ez;
    /* lens, Sec. II-B Eq. 7-8 and Sec. III-B: lens_mode 0 = bent-ray (Fermat)
     * model with a curved lens whose outer surface is an arc of radius
     * lens_radius about (arc_cx, arc_cz), concentric with the element arc;
     * 1 = no lens (rays start at the element, Eq. 1; with t_ttp this is the
     * conventional model of Eq. 6); 2 = bent-ray model with a flat lens whose
     * outer surface is the line z = lens_z (linear array). */
    int lens_mode;
    double arc_cx, arc_cz, lens_radius;
    double c_lens, t_ttp, lens_z;
    /* apodization, Eq. 2-4: apod_mode 0 = |x'| <= z'/(2F), 1 = |x'| <= (F/2) z' */
    int apod_mode;
    double fnum;
    /* image points r_Omega, patch-major: pixel p belongs to patch p / patch_npix */
    int n_patch, patch_npix;
    const double *px, *pz;
    /* slowness grid, Sec. III-A: node (i, j) at (x0 + i dx, z0 + j dz), s[j*nx + i] */
    int nx, nz;
    double x0, z0, dx, dz;
    int nseg;                      /* ray segments N (N+1 endpoints) */
    /* demodulated FSA data Psi[t][r][n], sample n at time t0 + n/fs */
    int ns;
    double fs, fd, t0;
    int sub_width;                 /* elements per subaperture block */
    double rho_thresh;             /* Table II correlation threshold */
    /* Eq. 10-12 regularisation; c_unit = m/s per unit of the sound speed c
     * that Eq. 9-11 act on (1000: c in km/s, the reading R9) */
    double w1, kx1, kz1, w2, kx2, kz2;
    double c_unit;
} or_geom;

/* threads the library runs on: 1 for the plain build, all host cores for the
 * OpenMP build of the same source */
int or_omp_threads(void);
/* Sec. III-A dynamic CMPE grid for the global-speed sweep at speed c0: each
 * patch keeps its direction from the lens centre (curved lens) or its lateral
 * position (flat lens), its depth below the lens surface is multiplied by
 * c0 / c_ref, and its pixels' offsets from the patch centre (the mean of its
 * pixels) are multiplied by c0 / c_ref.  Writes n_patch * patch_npix positions. */
void or_dynamic_pixels(const or_geom *g, double c0, double c_ref, double *px_out, double *pz_out);
/* Eq. 3 (+ linear extrapolation at the two end elements) */
void or_element_angles(int ne, const double *ex, const double *ez, double *theta);
/* Eq. 2 + Eq. 4 */
int or_apod(const or_geom *g, const double *theta, int e, double x, double z);
/* Sec. III-A: mean sound speed of the grid, c_med = mean(1/s) */
double or_mean_speed(const or_geom *g, const double *s);
/* Eq. 8 + Sec. III-A: lens exit point by Fermat's principle at slowness sbar.
 * Returns the number of iterations (negative if the pixel lies inside the lens).
 * phi is the exit angle about the arc centre (lens_mode 0) or the exit x on
 * the line z = lens_z (lens_mode 2). */
int or_exit_point(const or_geom *g, int e, double x, double z, double sbar,
                  double *phi, double *t_lens, double *qx, double *qz);
/* lens time and exit point for a given (frozen) exit angle / exit x phi */
void or_exit_from_angle(const or_geom *g, int e, double phi, double *t_lens,
                        double *qx, double *qz);
/* Keys cubic-convolution weights (a = -1/2) for taps -1, 0, 1, 2 at fraction t */
void or_keys_weights(double t, double w[4]);
/* Sec. III-A bicubic interpolation of the slowness grid (clamp to edge) */
double or_bicubic(const or_geom *g, const double *s, double x, double z);
/* Eq. 1 discretised (Sec. III-A): straight ray from (qx,qz) to (x,z) */
double or_ray_time(const or_geom *g, const double *s, double qx, double qz,
                   double x, double z);
/* One-way delays T[e][p] (s) and apodization bits for every (element, pixel).
 * apod_in / phi_in may be NULL; when given they replace the oracle's own
 * apodization decision / exit angle. */
void or_delays(const or_geom *g, const double *s, const uint8_t *apod_in,
               const double *phi_in, double *T, uint8_t *apod, double *phi);
/* Eq. 5 over transmit/receive subaperture blocks: B[b][p][2], b = i*nsub + j */
void or_das(const or_geom *g, const float *psi, const double *T, const uint8_t *apod,
            double *B);
/* number of common-midpoint pairs per patch and the pair table [npair][2] */
int or_cmpe_pairs(const or_geom *g, int *pairs);
/* CMPE focusing loss (builder's reading, see header of af_oracle.c).
 * mask_in may be NULL.  z: [n_patch][npair][2], rho, mask: [n_patch][npair]. */
double or_cmpe(const or_geom *g, const double *B, const uint8_t *mask_in,
               double *z, double *rho, uint8_t *mask, int *n_active);
/* Eq. 10 and Eq. 11 */
void or_regularizers(const or_geom *g, const double *s, double *rtv, double *rsv);
/* d(w1 R_TV + w2 R_SV)/ds added into grad */
void or_regularizer_grad(const or_geom *g, const double *s, double *grad);
/* dL_CMPE/dB (G = dL/dRe B + j dL/dIm B), same layout as B */
void or_cmpe_adjoint(const or_geom *g, const double *B, const double *z,
                     const uint8_t *mask, int n_active, double *G);
/* dL/dT[e][p] from G (exit points and masks held constant) */
void or_das_adjoint(const or_geom *g, const float *psi, const double *T,
                    const uint8_t *apod, const double *G, double *gT);
/* dL/ds from dL/dT through the discretised ray integral; added into grad */
void or_ray_adjoint(const or_geom *g, const double *s, const double *phi,
                    const uint8_t *apod, const double *gT, double *grad);
/* Eq. 12 loss and dL/ds.  parts = {L, L_CMPE, R_TV, R_SV}.  Any of the
 * *_in arguments may be NULL.  grad may be NULL (forward only). */
double or_loss_grad(const or_geom *g, const float *psi, const double *s,
                    const uint8_t *apod_in, const uint8_t *mask_in,
                    const double *phi_in, double *grad, double parts[4],
                    uint8_t *mask_out, int *n_active);
/* Eq. 9 as printed: c <- c - lr dL/dc on c = 1 / (s * c_unit); grad is dL/ds */
void or_gd(int n, double *s, const double *grad, double lr, double c_unit);
/* Eq. 9 generalised to Adam on the sound speed c = 1 / (s * c_unit), i.e. c in
 * units of c_unit m/s (R8); grad is dL/ds, s is updated in place */
void or_adam(int n, double *s, const double *grad, double *m, double *v, int step,
             double lr, double beta1, double beta2, double eps, double c_unit);

#ifdef __cplusplus
}
#endif
#endif
