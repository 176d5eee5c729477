// fold.cu -- per-request harmonics and fold of the harmonics into the spline coefficients.
//
// Sec. 4 sum: h = scale * sum_{lmn} A_lmn(t) -2Y_lm(theta, phi) e^{-i Phi_mn}, with the m < 0
// modes given by Eq. (amp_symmetry), k = 0: A_{l,-m,-n} = (-1)^l conj(A_lmn).  Grouping every
// term by its signed frequency (m, n) gives
//     h = sum_{(m,n) signed} K_{m,n}(u) e^{-i (m Phi_phi + n Phi_r)},
//     K_{m,n}   = scale * sum_l A_lmn(u) Y+_lm                        (m >= 0 entries),
//     K_{-m,-n} = scale * sum_l conj(A_lmn(u)) Y-_lm,  Y- = (-1)^l -2Y_{l,-m}   (m > 0),
// and each K is again a complex cubic in u per segment (a fixed linear combination of the
// amplitude splines).  k_fold forms these "slot" cubics for one request; the summation kernel
// then evaluates sum K z_phi^m z_r^n by Horner's rule.  This is exact algebra on the
// coefficients (only the rounding order differs from summing mode by mode).
//
// Spin-weighted harmonics (the paper lists them as a utility, Sec. 3.D, without a formula):
//     sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi},  s = -2,
// with the Wigner small-d evaluated through its Jacobi-polynomial form
//     d^l_{m',m}(b) = xi sqrt(k! (k+mu+nu)! / ((k+mu)! (k+nu)!)) sin^mu(b/2) cos^nu(b/2)
//                      P_k^{(mu,nu)}(cos b),
//     mu = |m - m'|, nu = |m + m'|, k = l - (mu+nu)/2, xi = 1 if m >= m' else (-1)^(m-m'),
// and the Jacobi polynomial by its three-term recurrence in the degree.
#include "fewsum_internal.h"
#include "harmonics.cuh"
#include "convert.cuh"

namespace fewsum {

__device__ __forceinline__ int wave_of(const WaveDev *waves, int n, int g, bool by_pair)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int b = by_pair ? waves[mid].pair_begin : waves[mid].fold_begin;
        if (b <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Frame transformation (Sec. 2.A): from the sky position (tS, pS) and the spin direction
// (tK, pK) in the barycentre frame, the source-frame viewing angles of the propagation direction
// -R in the basis x = R x S/|R x S|, y = (R - (R.S) S)/|R x S|, z = S, and the polarization
// angle psi with tan psi = (cos tS sin tK cos(pS - pK) - sin tS cos tK)/(sin tK sin(pS - pK)).
// The detector-frame waveform is -e^{-2 i psi} times the source-frame one (a pi phase shift for
// the pi/2 basis rotation, then the 2 psi rotation), a constant folded into the harmonics.
__device__ void frame_angles(double tS, double pS, double tK, double pK, double &theta,
                             double &phi, double &psi)
{
    double stS, ctS, spS, cpS, stK, ctK, spK, cpK;
    sincos(tS, &stS, &ctS);
    sincos(pS, &spS, &cpS);
    sincos(tK, &stK, &ctK);
    sincos(pK, &spK, &cpK);
    const double R[3] = {stS * cpS, stS * spS, ctS};
    const double S[3] = {stK * cpK, stK * spK, ctK};
    const double X[3] = {R[1] * S[2] - R[2] * S[1], R[2] * S[0] - R[0] * S[2],
                         R[0] * S[1] - R[1] * S[0]};
    const double nx = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    const double rs = R[0] * S[0] + R[1] * S[1] + R[2] * S[2];
    // components of -R: along x (R x S is orthogonal to R), along y, along z = S
    const double vx = 0.0;
    const double vy = -((R[0] - rs * S[0]) * R[0] + (R[1] - rs * S[1]) * R[1] +
                        (R[2] - rs * S[2]) * R[2]) / nx;
    const double vz = -rs;
    theta = acos(fmax(-1.0, fmin(1.0, vz)));
    phi = atan2(vy, vx);
    double sd, cd;
    sincos(pS - pK, &sd, &cd);
    psi = atan2(ctS * stK * cd - stS * ctK, stK * sd);
}

// Two threads per (wave, (l, m) pair): one computes Y+, the other Y- (halves the dependency
// chain each thread waits on).  FP64 plans evaluate the harmonics in FP64; mixed plans, whose
// folded coefficients are FP32, evaluate them in FP32 (relative error near 1e-7, far below the
// path's 1e-6 mismatch budget) and stay off GB300's narrow FP64 pipe.  The frame angles are FP64.
// One instantiation per arithmetic type keeps each kernel's code small (it runs cold, once).
template <bool FP64>
__global__ void __launch_bounds__(kYlmThreads) k_ylm(const PlanHdr *__restrict__ hp)
{
    const PlanHdr h = *hp;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t >> 1, which = t & 1;
    if (g >= h.total_pairs) return;
    const int w = wave_of(h.waves, h.n_waves, g, true);
    const WaveDev &W = h.waves[w];
    const int p = g - W.pair_begin;
    if (p >= W.tr.n_pairs) {
        atomicOr(h.err, ERRBIT_INTERNAL);
        return;
    }
    const int2 lm = W.tr.pair_lm[p];
    double theta = W.theta, phi = W.phi, psi = 0.0;
    if (W.frame == FEW_FRAME_SSB) frame_angles(W.theta, W.phi, W.theta_K, W.phi_K, theta, phi, psi);
    double2 y = make_double2(0.0, 0.0);
    const int mm = which == 0 ? lm.y : -lm.y;
    if (which == 0 || lm.y > 0) {
        y = FP64 ? swsh_m2_t<double>(lm.x, mm, theta, phi)
                 : swsh_m2_t<float>(lm.x, mm, (float)theta, (float)phi);
        if (which == 1 && (lm.x & 1)) y = make_double2(-y.x, -y.y);
    }
    if (W.frame == FEW_FRAME_SSB) {
        double s2, c2;
        sincos(2.0 * psi, &s2, &c2);
        const double fr = -c2, fi = s2;  // -e^{-2 i psi}
        y = make_double2(y.x * fr - y.y * fi, y.x * fi + y.y * fr);
    }
    W.ylm[2 * p + which] = y;
}

cudaError_t launch_ylm(const PlanHdr *hdr_dev, int total_pairs, bool fp64, cudaStream_t st)
{
    if (total_pairs <= 0) return cudaSuccess;
    const int threads = 2 * total_pairs, grid = (threads + kYlmThreads - 1) / kYlmThreads;
    if (fp64)
        k_ylm<true><<<grid, kYlmThreads, 0, st>>>(hdr_dev);
    else
        k_ylm<false><<<grid, kYlmThreads, 0, st>>>(hdr_dev);
    return cudaGetLastError();
}

__device__ __forceinline__ double cvt(double v, double) { return v; }
__device__ __forceinline__ float cvt(double v, float) { return f64_to_f32_fast(v); }

template <typename T> struct Slot8;
template <> struct Slot8<double> {
    __device__ static void store(double *dst, const double (&re)[4], const double (&im)[4])
    {
        double2 *d = reinterpret_cast<double2 *>(dst);
        d[0] = make_double2(re[0], re[1]);
        d[1] = make_double2(re[2], re[3]);
        d[2] = make_double2(im[0], im[1]);
        d[3] = make_double2(im[2], im[3]);
    }
};
template <> struct Slot8<float> {
    __device__ static void store(float *dst, const float (&re)[4], const float (&im)[4])
    {
        float4 *d = reinterpret_cast<float4 *>(dst);
        d[0] = make_float4(re[0], re[1], re[2], re[3]);
        d[1] = make_float4(im[0], im[1], im[2], im[3]);
    }
};

// One thread per (wave, segment, slot): K_slot = scale * sum of its contributions, summed on the
// splines' Hermite data (values and slopes at the segment's two knots) and turned into power
// coefficients in u once.
// T is the arithmetic and storage type of the folded coefficients (double for FEW_FP64,
// float for FEW_MIXED, whose amplitudes are FP32 by design).
template <typename T>
__global__ void __launch_bounds__(kFoldThreads) k_fold(const PlanHdr *__restrict__ hp)
{
    const PlanHdr h = *hp;
    const int b = blockIdx.x;
    const int w = wave_of(h.waves, h.n_waves, b, false);
    const WaveDev &W = h.waves[w];
    const int local = b - W.fold_begin;
    const int s = local / W.fold_blocks_per_seg;
    const int slot = (local % W.fold_blocks_per_seg) * kFoldThreads + threadIdx.x;
    const TrajDev &tr = W.tr;
    if (s >= tr.S || slot >= tr.n_slots) return;
    T re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
    const int c0 = tr.slot_ptr[slot], c1 = tr.slot_ptr[slot + 1];
    const double *__restrict__ cs = tr.coef + (size_t)s * tr.J * 4;
    for (int c = c0; c < c1; ++c) {
        const int2 code = tr.contrib[c];  // (mode * 2 + kind, harmonic-table index)
        const int i = code.x >> 1, kind = code.x & 1;
        const double2 Yd = W.ylm[code.y];
        const T yr = cvt(Yd.x, T()), yi = cvt(Yd.y, T());
        const double2 *ca = reinterpret_cast<const double2 *>(cs + (size_t)(2 + 2 * i) * 4);
        const double2 r01 = ca[0], r23 = ca[1], i01 = ca[2], i23 = ca[3];
        const T ar[4] = {cvt(r01.x, T()), cvt(r01.y, T()), cvt(r23.x, T()), cvt(r23.y, T())};
        T ai[4] = {cvt(i01.x, T()), cvt(i01.y, T()), cvt(i23.x, T()), cvt(i23.y, T())};
        if (kind) {
#pragma unroll
            for (int q = 0; q < 4; ++q) ai[q] = -ai[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            re[q] += ar[q] * yr - ai[q] * yi;
            im[q] += ar[q] * yi + ai[q] * yr;
        }
    }
    // the folded values are Hermite data (the fold is linear in them): power coefficients in u
    // once per (segment, slot)
    const T hk = cvt(tr.h[s], T()), sc = cvt(W.scale, T());
    T pre[4], pim[4];
    hermite_to_power(re[0], re[1], re[2], re[3], hk, pre);
    hermite_to_power(im[0], im[1], im[2], im[3], hk, pim);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        pre[q] *= sc;
        pim[q] *= sc;
    }
    T *dst = reinterpret_cast<T *>(W.fcoef) + ((size_t)s * tr.n_slots + slot) * 8;
    Slot8<T>::store(dst, pre, pim);
}

cudaError_t launch_fold(const PlanHdr *hdr_dev, int total_fold_blocks, bool fp64, cudaStream_t st)
{
    if (total_fold_blocks <= 0) return cudaSuccess;
    if (fp64)
        k_fold<double><<<total_fold_blocks, kFoldThreads, 0, st>>>(hdr_dev);
    else
        k_fold<float><<<total_fold_blocks, kFoldThreads, 0, st>>>(hdr_dev);
    return cudaGetLastError();
}

}  // namespace fewsum
