// Transit templates: the last column of the design matrix (Sect. 2.1), unit
// depth, evaluated at a sample inside the half-open window
// t0 - D/2 <= t < t0 + D/2.  Each FP64 operation is rounded once, in the
// order written, so that the template values do not depend on contraction.
//   NU_BOX        -1 (Sect. 2.1).
//   NU_TRAPEZOID  -min(1, (D/2 - |t - t0|) / ramp), ramp = ingress_frac D.
//   NU_LIMB_QUAD  a limb-darkened transit as base model (the prospect of
//                 Sect. 4.4): small-planet limit of a central transit
//                 (Mandel & Agol 2002, ApJ 580, L171, Sect. 5) under the
//                 quadratic law, -I(mu) with r = 2 (t - t0) / D,
//                 mu = sqrt(1 - r^2), x = 1 - mu, I = 1 - u1 x - u2 x^2
//                 (I = 1 at the centre, 1 - u1 - u2 at the limb).
#pragma once

#include <cmath>

#include "nu_internal.cuh"

namespace nu {

// Template parameters as passed across the ABI: trapezoid p0 = ingress_frac;
// limb darkening p0 = u1, p1 = u2.
struct TmplArgs {
    double p0, p1;
};

template <int TMPL>
__device__ __forceinline__ double template_value(double t, double t0, double half, double D,
                                                 const TmplArgs& a) {
    if (TMPL == NU_BOX) return -1.0;
    if (TMPL == NU_TRAPEZOID) {
        const double ramp = __dmul_rn(a.p0, D);
        const double dd = __ddiv_rn(__dsub_rn(half, fabs(__dsub_rn(t, t0))), ramp);
        return -fmin(fmax(dd, 0.0), 1.0);
    }
    const double r = __ddiv_rn(__dmul_rn(2.0, __dsub_rn(t, t0)), D);
    const double mu = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(r, r)));
    const double x = __dsub_rn(1.0, mu);
    return -__dsub_rn(__dsub_rn(1.0, __dmul_rn(a.p0, x)), __dmul_rn(__dmul_rn(a.p1, x), x));
}

// Host-side validation and unpacking of the ABI's template parameters;
// returns false (message in *why) when they are not acceptable.
inline bool template_args(int tmpl, const double* params, TmplArgs* out, const char** why) {
    out->p0 = 0.0;
    out->p1 = 0.0;
    if (tmpl == NU_BOX) return true;
    if (tmpl == NU_TRAPEZOID) {
        if (!params || !(params[0] > 0.0 && params[0] <= 0.5)) {
            *why = "trapezoid needs params[0] = ingress_frac in (0, 0.5]";
            return false;
        }
        out->p0 = params[0];
        return true;
    }
    if (tmpl == NU_LIMB_QUAD) {
        if (!params || !std::isfinite(params[0]) || !std::isfinite(params[1])) {
            *why = "limb-darkened template needs finite params[0] = u1, params[1] = u2";
            return false;
        }
        out->p0 = params[0];
        out->p1 = params[1];
        return true;
    }
    *why = "unknown template";
    return false;
}

}  // namespace nu
