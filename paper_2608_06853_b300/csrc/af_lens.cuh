// Lens exit point by Fermat's principle (Eq. 8, Sec. III-A): chord lengths on
// the concentric element / lens / pixel circles and the safeguarded Newton
// solve of dT/dphi = 0, shared by the delay kernel (float32 solve with float64
// fallback) and the surrogate's label generator (float64).
#pragma once

#include <math.h>

namespace {

// chord length between radius r1 at angle 0 and radius r2 at angle d, with
// its first two derivatives in d; sh = sin(d/2), ch = cos(d/2)
struct Chord { float len, d1, d2; };
__device__ __forceinline__ Chord chord(float r1, float r2, float d)
{
    float sh, ch;
    sincosf(0.5f * d, &sh, &ch);
    float k = r1 * r2, dr = r1 - r2;
    float len = sqrtf(fmaf(dr, dr, 4.0f * k * sh * sh));
    float sd = 2.0f * sh * ch, cd = fmaf(-2.0f * sh, sh, 1.0f);
    float inv = 1.0f / len;
    float ks = k * sd * inv;
    return {len, ks, (k * cd - ks * ks) * inv};
}

struct ChordD { double len, d1, d2; };
__device__ ChordD chord_d(double r1, double r2, double d)
{
    double sh, ch;
    sincos(0.5 * d, &sh, &ch);
    double k = r1 * r2, dr = r1 - r2;
    double len = sqrt(dr * dr + 4.0 * k * sh * sh);
    double ks = k * 2.0 * sh * ch / len;
    return {len, ks, (k * (1.0 - 2.0 * sh * sh) - ks * ks) / len};
}

// float64 safeguarded Newton / bisection on dT/dd = 0 over [lo, hi]
__device__ double exit_solve_fp64(double re, double rp, double RL, double dp, double inv_cl,
                                  double sbar)
{
    double lo = fmin(0.0, dp), hi = fmax(0.0, dp), x = 0.0;
    for (int it = 0; it < 100; ++it) {
        ChordD a = chord_d(re, RL, x), b = chord_d(rp, RL, x - dp);
        double f = a.d1 * inv_cl + b.d1 * sbar;
        double fp = a.d2 * inv_cl + b.d2 * sbar;
        if (f == 0.0) break;
        if (f < 0.0) lo = x; else hi = x;
        double xn = fp > 0.0 ? x - f / fp : 0.5 * (lo + hi);
        if (!(xn >= lo && xn <= hi)) xn = 0.5 * (lo + hi);
        double step = fabs(xn - x);
        x = xn;
        if (step < 1e-13 || hi - lo < 1e-13) break;
    }
    return x;
}

// Flat lens (outer surface the line z = zl): exit x u minimising
//   T(u) = sqrt((u - xe)^2 + h1^2) / c_lens + sqrt((xp - u)^2 + h2^2) sbar,
// h1 = zl - ze, h2 = zp - zl.  T'' > 0 and T' changes sign between xe and xp:
// float64 safeguarded Newton / bisection on T' = 0 over that bracket.
__device__ double exit_solve_flat_fp64(double xe, double h1, double xp, double h2, double inv_cl,
                                       double sbar)
{
    double lo = fmin(xe, xp), hi = fmax(xe, xp), u = xe;
    for (int it = 0; it < 100 && hi > lo; ++it) {
        const double d1 = sqrt((u - xe) * (u - xe) + h1 * h1), d2 = sqrt((xp - u) * (xp - u) + h2 * h2);
        const double f = (u - xe) * inv_cl / d1 - (xp - u) * sbar / d2;
        const double fp = h1 * h1 * inv_cl / (d1 * d1 * d1) + h2 * h2 * sbar / (d2 * d2 * d2);
        if (f == 0.0) break;
        if (f < 0.0) lo = u; else hi = u;
        double un = u - f / fp;
        if (!(un >= lo && un <= hi)) un = 0.5 * (lo + hi);
        const double step = fabs(un - u);
        u = un;
        if (step < 1e-15 || hi - lo < 1e-15) break;
    }
    return u;
}

}  // namespace
