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

// Arithmetic-type overloads (double for the FP64 path, float for the mixed path).
__device__ inline void sincos_t(double x, double *s, double *c) { sincos(x, s, c); }
__device__ inline void sincos_t(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ inline double sqrt_t(double x) { return sqrt(x); }
__device__ inline float sqrt_t(float x) { return sqrtf(x); }
__device__ inline double cos_t(double x) { return cos(x); }
__device__ inline float cos_t(float x) { return cosf(x); }

template <typename T>
__device__ inline T jacobi_p(int n, int a, int b, T x)
{
    if (n == 0) return T(1);
    T p0 = T(1);
    T p1 = T(a + 1) + T(0.5) * T(a + b + 2) * (x - T(1));
    for (int k = 2; k <= n; ++k) {
        const T c = T(2 * k + a + b);
        const T a1 = T(2 * k) * T(k + a + b) * (c - T(2));
        const T a2 = (c - T(1)) * (c * (c - T(2)) * x + T(a * a - b * b));
        const T a3 = T(2) * T(k + a - 1) * T(k + b - 1) * c;
        const T p2 = (a2 * p1 - a3 * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

template <typename T>
__device__ inline T ipow(T x, int e)
{
    T r = T(1);
    for (int k = 0; k < e; ++k) r *= x;
    return r;
}

// -2Y_{l,m}(theta, phi), evaluated in the arithmetic type T.
template <typename T>
__device__ inline double2 swsh_m2_t(int l, int m, T theta, T phi)
{
    const int mu = abs(2 - m), nu = abs(2 + m);
    const int k = l - ((mu + nu) >> 1);
    if (k < 0) return make_double2(0.0, 0.0);
    T ratio = T(1);
    for (int q = 1; q <= mu; ++q) ratio *= T(k + nu + q) / T(k + q);
    const T xi = (m <= 2) ? T(1) : ((m & 1) ? T(-1) : T(1));
    T sh, ch;
    sincos_t(T(0.5) * theta, &sh, &ch);
    const T d = xi * sqrt_t(ratio) * ipow(sh, mu) * ipow(ch, nu) * jacobi_p(k, mu, nu, cos_t(theta));
    const T kInv4Pi = T(0.079577471545947667884);  // 1/(4 pi)
    const T amp = sqrt_t(T(2 * l + 1) * kInv4Pi) * d;
    T s, c;
    sincos_t(T(m) * phi, &s, &c);
    return make_double2((double)(amp * c), (double)(amp * s));
}

__device__ inline double2 swsh_m2(int l, int m, double theta, double phi)
{
    return swsh_m2_t<double>(l, m, theta, phi);
}

}  // namespace fewsum
