// harmonics.cuh -- spin-weighted spherical harmonics -2Y_lm on the device.
//
// The paper lists the harmonics as a utility (Sec. 3.D) without a formula; the convention used is
//     sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi},  s = -2,
// with the Wigner small-d through its Jacobi-polynomial form
//     d^l_{m',m}(b) = xi sqrt(k! (k+mu+nu)! / ((k+mu)! (k+nu)!)) sin^mu(b/2) cos^nu(b/2)
//                      P_k^{(mu,nu)}(cos b),
//     mu = |m - m'|, nu = |m + m'|, k = l - (mu+nu)/2, xi = 1 if m >= m' else (-1)^(m-m'),
// and the Jacobi polynomial by its three-term recurrence in the degree.
#pragma once

namespace fewsum {

__device__ inline double jacobi_p(int n, int a, int b, double x)
{
    if (n == 0) return 1.0;
    double p0 = 1.0;
    double p1 = (a + 1) + 0.5 * (a + b + 2) * (x - 1.0);
    for (int k = 2; k <= n; ++k) {
        const double c = 2.0 * k + a + b;
        const double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
        const double a2 = (c - 1.0) * (c * (c - 2.0) * x + (double)(a * a - b * b));
        const double a3 = 2.0 * (k + a - 1) * (k + b - 1) * c;
        const double p2 = (a2 * p1 - a3 * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

__device__ inline double ipow(double x, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= x;
    return r;
}

// -2Y_{l,m}(theta, phi)
__device__ inline double2 swsh_m2(int l, int m, double theta, double phi)
{
    const int mu = abs(2 - m), nu = abs(2 + m);
    const int k = l - ((mu + nu) >> 1);
    if (k < 0) return make_double2(0.0, 0.0);
    double ratio = 1.0;
    for (int q = 1; q <= mu; ++q) ratio *= (double)(k + nu + q) / (double)(k + q);
    const double xi = (m <= 2) ? 1.0 : ((m & 1) ? -1.0 : 1.0);
    double sh, ch;
    sincos(0.5 * theta, &sh, &ch);
    const double d = xi * sqrt(ratio) * ipow(sh, mu) * ipow(ch, nu) * jacobi_p(k, mu, nu, cos(theta));
    const double kInv4Pi = 0.079577471545947667884;  // 1/(4 pi)
    const double amp = sqrt((2.0 * l + 1.0) * kInv4Pi) * d;
    double s, c;
    sincos((double)m * phi, &s, &c);
    return make_double2(amp * c, amp * s);
}

}  // namespace fewsum
