// phase_eval.cuh -- per-sample orbital phases, reduced modulo 2 pi, in FP64.
//
// The phase integrals of Sec. 2 reach 1e5-1e7 rad over one to four years, where one FP64 ulp
// is 1e-11-1e-9 rad; every harmonic multiplies that by |m| or |n| (up to 10 and 30).  So the
// spline of each phase is kept in radians as given, and each segment's constant term c0 (the
// knot value) is reduced modulo 2 pi once per segment with a two-constant Cody-Waite step whose
// product k * C_hi is made exact by an FMA (C_hi = fl(2 pi), C_lo = fl(2 pi - C_hi)); the
// reduced c0 is then within 1e-15 rad of the exact residue.  Per sample the cubic in
// u = (t - t_k)/h_k adds at most a few thousand radians, so the remaining FP64 rounding stays
// near 1e-12 rad, and the result is converted to turns and reduced again, f = x - rint(x).
#pragma once

#include "fewsum_internal.h"

namespace fewsum {

struct SegPhase {
    double c0phi, c0r;   // reduced constant terms (rad), offsets included
    double pphi[3], pr[3];  // u^1..u^3 coefficients (rad)
    double tk, ih;       // segment start and 1/h
};

// x modulo 2 pi, in (-pi, pi] up to rounding, for |x| up to ~1e15.
__device__ __forceinline__ double reduce_2pi(double x)
{
    const double kInv2Pi = 0.15915494309189533577;
    const double kC_hi = 6.283185307179586232;      // fl(2 pi)
    const double kC_lo = 2.4492935982947064e-16;    // fl(2 pi - fl(2 pi))
    const double k = rint(x * kInv2Pi);
    const double p = k * kC_hi;
    const double e = fma(k, kC_hi, -p);  // exact: k * C_hi = p + e
    return ((x - p) - e) - k * kC_lo;
}

__device__ __forceinline__ SegPhase seg_phase(const TrajDev &tr, int s, double dphi_phi,
                                              double dphi_r)
{
    const double *pc = tr.coef + (size_t)s * tr.J * 4;
    const double hk = tr.h[s];
    double cphi[4], cr[4];
    hermite_to_power(pc[0], pc[1], pc[2], pc[3], hk, cphi);
    hermite_to_power(pc[4], pc[5], pc[6], pc[7], hk, cr);
    SegPhase sp;
    sp.c0phi = reduce_2pi(cphi[0]) + reduce_2pi(dphi_phi);
    sp.c0r = reduce_2pi(cr[0]) + reduce_2pi(dphi_r);
    sp.pphi[0] = cphi[1]; sp.pphi[1] = cphi[2]; sp.pphi[2] = cphi[3];
    sp.pr[0] = cr[1]; sp.pr[1] = cr[2]; sp.pr[2] = cr[3];
    sp.tk = tr.t[s];
    sp.ih = tr.inv_h[s];
    return sp;
}

// Reduced phases of sample i (turns, each in [-1/2, 1/2]) and its local coordinate u.
__device__ __forceinline__ void sample_phase(const SegPhase &sp, double t0, double dt, int i,
                                             double &fphi, double &fr, double &u)
{
    const double kInv2Pi = 0.15915494309189533577;
    const double t = fma((double)i, dt, t0);
    u = (t - sp.tk) * sp.ih;
    const double aphi = fma(fma(fma(sp.pphi[2], u, sp.pphi[1]), u, sp.pphi[0]), u, sp.c0phi);
    const double ar = fma(fma(fma(sp.pr[2], u, sp.pr[1]), u, sp.pr[0]), u, sp.c0r);
    const double xphi = aphi * kInv2Pi;
    const double xr = ar * kInv2Pi;
    fphi = xphi - rint(xphi);
    fr = xr - rint(xr);
}

}  // namespace fewsum
