// direct.cu -- direct (non-interpolated) mode summation (arXiv:2104.04582 Sec. 3.C).
//
// The "more basic" summation of the paper: the phases and every mode's amplitude are given at
// the output's own sample density, so there is no spline; at each sample i
//     h_i = scale * sum_modes [ A_i Y+ e^{-i Phi_mn,i} + (m > 0) conj(A_i) Y- e^{+i Phi_mn,i} ],
// Phi_mn,i = m Phi_phi,i + n Phi_r,i, Y+ = -2Y_lm, Y- = (-1)^l -2Y_{l,-m}  (Eq. amp_symmetry).
//
// Each mode-sample reads 16 bytes of FP64 amplitude and nothing is reused across samples, so in
// mixed precision the kernel is bound by HBM bandwidth (FP64 arithmetic throughout is bound by
// the FP64 pipe instead).  One warp per sample: lanes stride over the modes (coalesced reads of
// the [sample][mode] arrays, several loads in flight per lane), each lane forms its modes'
// exponentials from the sample's reduced phases (FP64 reduction of Phi_phi and Phi_r modulo 2 pi,
// then the sine and cosine of the reduced integer combination), and the warp reduces its partial
// sums with shuffles.
#include "fewsum_internal.h"
#include "harmonics.cuh"
#include "phase_eval.cuh"
#include "convert.cuh"

namespace fewsum {

// Per-mode constants in the arithmetic type of the path.  With Y+ = -2Y_lm and
// Y- = (-1)^l -2Y_{l,-m} (zero for m = 0), a mode contributes
//     A Y+ e^{-i Phi} + conj(A) Y- e^{+i Phi}
//   = Re A [ (a c + b s) + i (g c - d s) ] + Im A [ (a s - b c) + i (d c + g s) ],
// c = cos Phi, s = sin Phi, with a = Re(Y+ + Y-), b = Im(Y+ - Y-), g = Im(Y+ + Y-),
// d = Re(Y+ - Y-).  The record is 16-byte aligned so a lane fetches it in wide loads.
template <typename T>
struct alignas(16) ModeConst {
    T a, b, g, d;
    T m, n;
};

template <typename T>
__global__ void k_mode_consts(const int *__restrict__ l, const int *__restrict__ m,
                              const int *__restrict__ n, int N, double theta, double phi,
                              ModeConst<T> *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 yp = swsh_m2(l[i], m[i], theta, phi);
    double2 ym = make_double2(0.0, 0.0);
    if (m[i] > 0) {
        ym = swsh_m2(l[i], -m[i], theta, phi);
        if (l[i] & 1) ym = make_double2(-ym.x, -ym.y);
    }
    ModeConst<T> c;
    c.a = (T)(yp.x + ym.x); c.b = (T)(yp.y - ym.y);
    c.g = (T)(yp.y + ym.y); c.d = (T)(yp.x - ym.x);
    c.m = (T)m[i]; c.n = (T)n[i];
    out[i] = c;
}

// Amplitude conversion of the arithmetic path: the mixed path uses the branchless integer-pipe
// conversion (ties away from zero, below 2^-126 flushed, from 2^128 up given as infinity): the
// exact even-tie conversion costs about 15 integer operations per value and bounded this kernel.
__device__ __forceinline__ double to_t(double v, double) { return v; }
__device__ __forceinline__ float to_t(double v, float) { return f64_to_f32_fast(v); }

// Nearest integer of |x| < 2^22 by the 1.5 * 2^23 addition (FP32 add pipe); FP64 uses rint.
__device__ __forceinline__ float round_near(float x)
{
    const float k = 12582912.0f;
    return (x + k) - k;
}
__device__ __forceinline__ double round_near(double x) { return rint(x); }

// Exponential of the reduced phase ph (turns, |ph| <= 1/2): FP64 sincospi for the plain path;
// for the mixed path the SFU sine and cosine of 2 pi ph (|x| <= pi, absolute error below 1e-6).
__device__ __forceinline__ void expi_turns(double ph, double *s, double *c) { sincospi(2.0 * ph, s, c); }
__device__ __forceinline__ void expi_turns(float ph, float *s, float *c)
{
    __sincosf(6.283185307179586f * ph, s, c);
}

constexpr int kDirectUnroll = 8;  // amplitude loads in flight per lane before any arithmetic

template <typename T>
__global__ void __launch_bounds__(256)
k_direct(const double *__restrict__ pphi, const double *__restrict__ pr,
         const double *__restrict__ are, const double *__restrict__ aim, long long ns, int N,
         const ModeConst<T> *__restrict__ mc, double scale, void *__restrict__ out, int out_c64)
{
    const double kInv2Pi = 0.15915494309189533577;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < ns; i += nwarps) {
        const double xp = reduce_2pi(pphi[i]) * kInv2Pi, xr = reduce_2pi(pr[i]) * kInv2Pi;
        const T fphi = (T)(xp - rint(xp)), fr = (T)(xr - rint(xr));
        const double *ar = are + (size_t)i * N, *ai = aim + (size_t)i * N;
        T hr = 0, hi = 0;
        for (int j0 = lane; j0 < N; j0 += 32 * kDirectUnroll) {
            double vr[kDirectUnroll], vi[kDirectUnroll];
#pragma unroll
            for (int u = 0; u < kDirectUnroll; ++u) {
                const int j = j0 + 32 * u;
                vr[u] = j < N ? __ldcs(ar + j) : 0.0;  // streamed once: evict-first
                vi[u] = j < N ? __ldcs(ai + j) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kDirectUnroll; ++u) {
                const int j = j0 + 32 * u;
                if (j >= N) break;
                const ModeConst<T> c = mc[j];
                const T Ar = to_t(vr[u], T()), Ai = to_t(vi[u], T());
                T ph = c.m * fphi + c.n * fr;
                ph -= round_near(ph);
                T s, co;
                expi_turns(ph, &s, &co);
                hr += Ar * (c.a * co + c.b * s) + Ai * (c.a * s - c.b * co);
                hi += Ar * (c.g * co - c.d * s) + Ai * (c.d * co + c.g * s);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hr += __shfl_down_sync(0xffffffffu, hr, o);
            hi += __shfl_down_sync(0xffffffffu, hi, o);
        }
        if (lane == 0) {
            const double vr0 = (double)hr * scale, vi0 = (double)hi * scale;
            if (out_c64)
                reinterpret_cast<float2 *>(out)[i] = make_float2((float)vr0, (float)vi0);
            else
                reinterpret_cast<double2 *>(out)[i] = make_double2(vr0, vi0);
        }
    }
}

cudaError_t launch_direct(const double *pphi, const double *pr, const double *are,
                          const double *aim, long long ns, const int *l, const int *m, const int *n,
                          int N, double theta, double phi, double scale, bool fp64, void *out,
                          int out_c64, void *mode_consts, int sm_count, cudaStream_t st)
{
    // one wave of resident blocks (8 warps, i.e. 8 samples, per block per round)
    static int resident[2] = {0, 0};
    int &rb = resident[fp64 ? 1 : 0];
    if (rb == 0) {
        const cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                         &rb, k_direct<double>, 256, 0)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                         &rb, k_direct<float>, 256, 0);
        if (e != cudaSuccess) return e;
        if (rb < 1) rb = 1;
    }
    const long long want = (ns + 7) / 8, cap = (long long)sm_count * rb;
    const int grid = (int)(want < cap ? want : cap);
    if (fp64) {
        auto *mc = static_cast<ModeConst<double> *>(mode_consts);
        k_mode_consts<double><<<(N + 63) / 64, 64, 0, st>>>(l, m, n, N, theta, phi, mc);
        if (ns > 0)
            k_direct<double><<<grid, 256, 0, st>>>(pphi, pr, are, aim, ns, N, mc, scale, out, out_c64);
    } else {
        auto *mc = static_cast<ModeConst<float> *>(mode_consts);
        k_mode_consts<float><<<(N + 63) / 64, 64, 0, st>>>(l, m, n, N, theta, phi, mc);
        if (ns > 0)
            k_direct<float><<<grid, 256, 0, st>>>(pphi, pr, are, aim, ns, N, mc, scale, out, out_c64);
    }
    return cudaGetLastError();
}

size_t direct_mode_const_bytes(int N) { return sizeof(ModeConst<double>) * (size_t)N; }

}  // namespace fewsum
