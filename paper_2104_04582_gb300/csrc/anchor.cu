// anchor.cu -- phase anchors of the mixed-precision summation (arXiv:2104.04582 Sec. 3.C, with
// the phase integrals of Sec. 2): at every kAnchorGroup-th output sample the FP64 phase splines
// are evaluated and reduced modulo one turn, and the Taylor coefficients of each phase cubic
// about that sample are stored for the summation kernel's FP32 in-group increments.
#include "fewsum_internal.h"
#include "phase_eval.cuh"
#include "convert.cuh"

namespace fewsum {

// Phase anchors of the mixed path, a few blocks per (wave, segment) sharing the segment's
// reduced constants, one thread per anchor of the segment: for group q of the anchor, at the
// anchor sample a = kAnchorGroup * q (which may precede the segment's first
// sample: the segment's cubic is used on both sides) the FP64 phases reduced modulo one turn and
// the Taylor coefficients of each phase cubic in sample units,
//   Phi(u + k du) - Phi(u) = k du Phi'(u) + (k du)^2 Phi''(u)/2 + (k du)^3 p3,  du = dt / h,
// divided by 2 pi (turns).  The identity is exact for a cubic; only its FP32 evaluation over
// k < kAnchorGroup samples in the summation kernel rounds.  The third stream is the phase of
// the final factor, g = m_last f_phi + lo_last f_r (an integer combination of the reduced
// phases, so equal to m_last Phi_phi + lo_last Phi_r modulo one turn), reduced again.
__global__ void __launch_bounds__(kAnchorThreads) k_anchor(const PlanHdr *__restrict__ hp)
{
    // kAnchorBlocksPerSeg blocks per (wave, segment); block -> wave by its first block
    const int n_waves = hp->n_waves;
    const WaveDev *waves = hp->waves;
    const int g = blockIdx.x / kAnchorBlocksPerSeg, part = blockIdx.x % kAnchorBlocksPerSeg;
    int lo = 0, hi = n_waves - 1;
    while (lo < hi) {  // largest w with anchor_seg_begin <= g
        const int mid = (lo + hi + 1) >> 1;
        if (waves[mid].anchor_seg_begin <= g) lo = mid; else hi = mid - 1;
    }
    const WaveDev &W = waves[lo];
    const int s = g - W.anchor_seg_begin;
    if (s >= W.tr.S) return;
    const int a0 = W.anchor_off[s], a1 = W.anchor_off[s + 1];
    if (a0 >= a1) return;
    const SegPhase sp = seg_phase(W.tr, s, W.dphi_phi, W.dphi_r);
    const double kInv2Pi = 0.15915494309189533577;
    const double du = W.dt * sp.ih;
    // the increment coefficients are small (a few tenths of a turn over a group) and are
    // stored in FP32: they are formed in FP32 from the segment's coefficients in turns per
    // sample^k; only the phase values and their reductions need FP64
    float c1[2], c2[2], c3[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double *p = k ? sp.pr : sp.pphi;
        c1[k] = (float)(p[0] * du * kInv2Pi);
        c2[k] = (float)(p[1] * du * du * kInv2Pi);
        c3[k] = (float)(p[2] * du * du * du * kInv2Pi);
    }
    const double ml = (double)W.tr.m_last, ll = (double)W.tr.lo_last;
    const float mlf = (float)W.tr.m_last, llf = (float)W.tr.lo_last;
    const int q0 = W.seg_start[s] / kAnchorGroup;
    // anchor position of the segment's first group, in samples from the knot
    const float v0 = (float)((fma((double)q0 * kAnchorGroup, W.dt, W.t0) - sp.tk) / W.dt);
    const double gdt = kAnchorGroup * W.dt;  // exact: a power-of-two multiple
    const int stride = kAnchorThreads * kAnchorBlocksPerSeg;
    // FP64 issue is scarce: integer -> FP64 by the exponent trick, rounding to an integer by
    // adding and subtracting 1.5 * 2^52 (exact for |x| < 2^51), FP64 -> FP32 on the integer pipe
    const double kRound = 6755399441055744.0, kTwo52 = 4503599627370496.0;
    for (int j = a0 + part * kAnchorThreads + threadIdx.x; j < a1; j += stride) {
        const int q = q0 + (j - a0);
        const double qd = __dsub_rn(__hiloint2double(0x43300000, q), kTwo52);
        const double t = fma(qd, gdt, W.t0);
        const double u = (t - sp.tk) * sp.ih;
        // v: the anchor's position in samples from the knot (u = v du), for the FP32 Taylor
        // coefficients of Phi(v + k) - Phi(v) = k Phi'(v) + k^2 Phi''(v)/2 + k^3 c3
        const float v = v0 + (float)((j - a0) * kAnchorGroup);
        double f0[2];
        float f[2][4];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const double c0 = k ? sp.c0r : sp.c0phi;
            const double *p = k ? sp.pr : sp.pphi;
            const double x = fma(fma(fma(p[2], u, p[1]), u, p[0]), u, c0) * kInv2Pi;
            f0[k] = x - __dsub_rn(__dadd_rn(x, kRound), kRound);
            f[k][0] = f64_to_f32(f0[k]);
            f[k][1] = fmaf(fmaf(3.0f * c3[k], v, 2.0f * c2[k]), v, c1[k]);
            f[k][2] = fmaf(3.0f * c3[k], v, c2[k]);
            f[k][3] = c3[k];
        }
        const double g0 = fma(ml, f0[0], ll * f0[1]);
        Anchor a;
        a.phi = make_float4(f[0][0], f[0][1], f[0][2], f[0][3]);
        a.r = make_float4(f[1][0], f[1][1], f[1][2], f[1][3]);
        a.g = make_float4(f64_to_f32(g0 - __dsub_rn(__dadd_rn(g0, kRound), kRound)),
                          fmaf(mlf, f[0][1], llf * f[1][1]), fmaf(mlf, f[0][2], llf * f[1][2]),
                          fmaf(mlf, f[0][3], llf * f[1][3]));
        W.anchors[j] = a;
    }
}

cudaError_t launch_anchor(const PlanHdr *hdr_dev, int total_anchor_segs, cudaStream_t st)
{
    if (total_anchor_segs <= 0) return cudaSuccess;
    k_anchor<<<total_anchor_segs * kAnchorBlocksPerSeg, kAnchorThreads, 0, st>>>(hdr_dev);
    return cudaGetLastError();
}

}  // namespace fewsum
