// sum.cu -- per-sample interpolation and mode sum (arXiv:2104.04582 Sec. 3.C, Sec. 4 sum).
//
// At every dense sample t_i the kernel evaluates
//     h(t_i) = sum_{(m,n) signed} K_{m,n}(u) z_phi^m z_r^n,
//     z_phi = e^{-i Phi_phi(t_i)},  z_r = e^{-i Phi_r(t_i)},  u = (t_i - t_k)/h_k,
// where K_{m,n} are the per-segment complex cubics produced by k_fold (amplitude splines with
// the spin-weighted harmonics, the m < 0 partners of Eq. amp_symmetry and the prefactor folded
// in).  Since e^{-i Phi_mn} = z_phi^m z_r^n exactly, the whole sum is a bivariate Laurent
// polynomial in (z_phi, z_r) and is evaluated by Horner's rule: along each row of constant m,
// over n >= 0 in z_r and over n < 0 in conj(z_r); then over the rows, m >= 0 in z_phi and
// m < 0 in conj(z_phi).  Per (slot, sample) that is one complex cubic (6 FMA) and one complex
// multiply-add (4 FMA) -- no transcendental per mode.
//
// Phases: FEW_FP64 evaluates the phase splines (in rad) in FP64 for every sample and reduces
// each phase modulo one turn, x - rint(x), in FP64; the reduced phases give z_phi and z_r
// (sincospi).  FEW_MIXED reads the phases from anchors written by k_anchor: at every
// kAnchorGroup-th sample the FP64 splines are evaluated and reduced modulo one turn, and the
// phase cubic's exact Taylor coefficients about that sample (in turns per sample^k) are stored;
// the kernel adds the in-group increment r (d1 + r (d2 + r d3)), r < kAnchorGroup (at most a
// few tenths of a turn), in FP32.  So every large phase value and every reduction is FP64,
// and the mixed kernel itself issues no FP64 instruction per sample (FP64 issue is scarce on
// this chip).  The integer combination m Phi_phi + n Phi_r is then carried exactly by the
// unit-modulus powers, so (m Phi_phi + n Phi_r) mod 2 pi never has to be formed explicitly.
// FEW_FP64 does everything else in FP64; FEW_MIXED evaluates amplitudes, exponential powers
// and the accumulation in FP32.
//
// Work decomposition: a persistent grid; each CTA owns an equal-cost, contiguous slice of the
// concatenated (waveform, sample) space (cost = samples x slots), walks it segment by segment,
// and stages each segment's folded coefficient table into shared memory with TMA bulk copies
// (cp.async.bulk + mbarrier transaction counts), double-buffered so the next segment's table
// arrives while the current one is in use.  Within a segment a pass covers threads x R
// consecutive samples, R per thread, each thread holding its samples' Horner state in
// registers and reusing every coefficient it reads from shared memory R times.  Every sample
// is summed by one thread in a fixed slot order, so results do not depend on the grid, the
// tile shape or on which other waveforms share the launch.
#include "fewsum_internal.h"
#include "phase_eval.cuh"
#include "async.cuh"

namespace fewsum {

namespace {

constexpr int kSlotUnroll = 2;  // slots per iteration of the Horner chain loop
constexpr int kBulkChunk = 32768;

struct Piece {
    int w, s, i0, i1;
};

__device__ __forceinline__ bool before(int w, int i, const CtaStart &e)
{
    return w < e.wave || (w == e.wave && i < e.sample);
}

// Move (w, i) forward to the first existing sample at or after it; false once past `end`.
__device__ bool normalize(const PlanHdr &h, int &w, int &i, const CtaStart &end)
{
    while (before(w, i, end) && w < h.n_waves) {
        if (i < h.waves[w].n_samples) return true;
        ++w;
        i = 0;
    }
    return false;
}

// The piece starting at sample i of wave w: the rest of i's segment inside [.., end).
__device__ Piece piece_at(const PlanHdr &h, int w, int i, const CtaStart &end)
{
    const WaveDev &W = h.waves[w];
    const int *ss = W.seg_start;
    int lo = 0, hi = W.tr.S - 1;
    while (lo < hi) {  // largest s with seg_start[s] <= i
        const int mid = (lo + hi + 1) >> 1;
        if (ss[mid] <= i) lo = mid; else hi = mid - 1;
    }
    int i1 = ss[lo + 1];
    if (w == end.wave && end.sample < i1) i1 = end.sample;
    return Piece{w, lo, i, i1};
}

template <typename T> struct Cf;
template <> struct Cf<float> {
    __device__ __forceinline__ static void load(const float *p, float (&c)[8])
    {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
        c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
    }
};
template <> struct Cf<double> {
    __device__ __forceinline__ static void load(const double *p, double (&c)[8])
    {
        const double2 *q = reinterpret_cast<const double2 *>(p);
        const double2 a = q[0], b = q[1], d = q[2], e = q[3];
        c[0] = a.x; c[1] = a.y; c[2] = b.x; c[3] = b.y;
        c[4] = d.x; c[5] = d.y; c[6] = e.x; c[7] = e.y;
    }
};

// Per-sample local coordinate u and the powers' bases (cos, sin of 2 pi f) of one segment.
template <typename T> struct PhaseSrc;

// FP64: both phase splines evaluated and reduced for every sample.
template <> struct PhaseSrc<double> {
    SegPhase sp;
    double t0, dt;
    __device__ __forceinline__ void init(const WaveDev &W, int s)
    {
        sp = seg_phase(W.tr, s, W.dphi_phi, W.dphi_r);
        t0 = W.t0;
        dt = W.dt;
    }
    __device__ __forceinline__ void at(int i, double &u, double &cphi, double &sphi, double &cr,
                                       double &sr) const
    {
        double fphi, fr;
        sample_phase(sp, t0, dt, i, fphi, fr, u);
        sincospi(2.0 * fphi, &sphi, &cphi);
        sincospi(2.0 * fr, &sr, &cr);
    }
};

// FP32: the anchor of the sample's group plus the in-group increment; u from the segment's
// first sample.
template <> struct PhaseSrc<float> {
    const Anchor *anc;
    int aidx;  // anc[aidx + (i / kAnchorGroup)] is sample i's anchor
    int i0;    // first sample of the segment
    float u0, du;
    __device__ __forceinline__ void init(const WaveDev &W, int s)
    {
        i0 = W.seg_start[s];
        anc = W.anchors;
        aidx = W.anchor_off[s] - i0 / kAnchorGroup;
        const double ih = W.tr.inv_h[s];
        u0 = (float)((fma((double)i0, W.dt, W.t0) - W.tr.t[s]) * ih);
        du = (float)(W.dt * ih);
    }
    __device__ __forceinline__ void at(int i, float &u, float &cphi, float &sphi, float &cr,
                                       float &sr) const
    {
        const float4 *a = reinterpret_cast<const float4 *>(anc + aidx + i / kAnchorGroup);
        const float4 ap = __ldg(a), ar = __ldg(a + 1);
        const float x = (float)(i % kAnchorGroup);
        const float fphi = fmaf(fmaf(fmaf(ap.w, x, ap.z), x, ap.y), x, ap.x);
        const float fr = fmaf(fmaf(fmaf(ar.w, x, ar.z), x, ar.y), x, ar.x);
        sincospif(2.0f * fphi, &sphi, &cphi);
        sincospif(2.0f * fr, &sr, &cr);
        u = fmaf((float)(i - i0), du, u0);
    }
};

// acc <- acc * z + K(u) along n consecutive slots (Horner in z = (zr, zi)).
template <typename T, int R>
__device__ __forceinline__ void horner_chain(const T *__restrict__ cf, int n, const T (&u)[R],
                                             const T (&zr)[R], const T (&zi)[R], T (&ar)[R],
                                             T (&ai)[R])
{
#pragma unroll (kSlotUnroll)
    for (int k = 0; k < n; ++k) {
        T c[8];
        Cf<T>::load(cf + 8 * k, c);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const T kr = fma(fma(fma(c[3], u[r], c[2]), u[r], c[1]), u[r], c[0]);
            const T ki = fma(fma(fma(c[7], u[r], c[6]), u[r], c[5]), u[r], c[4]);
            const T nr = fma(ar[r], zr[r], fma(-ai[r], zi[r], kr));
            const T ni = fma(ar[r], zi[r], fma(ai[r], zr[r], ki));
            ar[r] = nr;
            ai[r] = ni;
        }
    }
}

// One pass of the scalar path: R consecutive samples per thread, one value per register.
template <typename T, int R>
struct ScalarPass {
    using Scalar = T;
    static constexpr int kSamples = R;
    static constexpr int kSlotBytes = 8 * (int)sizeof(T);

    __device__ __forceinline__ static void run(const WaveDev &W, const unsigned char *buf, int p0,
                                               int i1, const PhaseSrc<T> &ps)
    {
        const T *__restrict__ cf = reinterpret_cast<const T *>(buf);
        const int tid = threadIdx.x;
        const int base = p0 + tid * R;
        T u[R], zr[R], zi[R], fr[R], fi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = min(base + r, i1 - 1);
            T sp_, cp, sr, cr;
            ps.at(i, u[r], cp, sp_, cr, sr);
            fr[r] = cp;   // z_phi = e^{-i 2 pi f_phi}
            fi[r] = -sp_;
            zr[r] = cr;   // z_r = e^{-i 2 pi f_r}
            zi[r] = -sr;
        }
        T tpr[R], tpi[R], tnr[R], tni[R], nzi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            tpr[r] = tpi[r] = tnr[r] = tni[r] = (T)0;
            nzi[r] = -zi[r];
        }
        const int2 *__restrict__ rows = W.tr.rows;
        const int nrp = W.tr.n_rows_pos, nrows = nrp + W.tr.n_rows_neg;
        int slot = 0;
        for (int row = 0; row < nrows; ++row) {
            const int2 rw = __ldg(rows + row);
            T ar[R], ai[R], br[R], bi[R];
#pragma unroll
            for (int r = 0; r < R; ++r) ar[r] = ai[r] = br[r] = bi[r] = (T)0;
            horner_chain<T, R>(cf + 8 * slot, rw.x, u, zr, zi, ar, ai);
            slot += rw.x;
            horner_chain<T, R>(cf + 8 * slot, rw.y, u, zr, nzi, br, bi);
            slot += rw.y;
            const bool pos = row < nrp;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                // row value: a + conj(z_r) * b
                const T vr = fma(br[r], zr[r], fma(bi[r], zi[r], ar[r]));
                const T vi = fma(bi[r], zr[r], fma(br[r], nzi[r], ai[r]));
                // T+ <- T+ z_phi + v  (m >= 0 rows),  T- <- T- conj(z_phi) + v  (m < 0 rows)
                if (pos) {
                    const T nr = fma(tpr[r], fr[r], fma(tpi[r], -fi[r], vr));
                    const T ni = fma(tpr[r], fi[r], fma(tpi[r], fr[r], vi));
                    tpr[r] = nr;
                    tpi[r] = ni;
                } else {
                    const T nr = fma(tnr[r], fr[r], fma(tni[r], fi[r], vr));
                    const T ni = fma(tni[r], fr[r], fma(tnr[r], -fi[r], vi));
                    tnr[r] = nr;
                    tni[r] = ni;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = base + r;
            if (i >= i1) break;
            // h = T+ + conj(z_phi) T-
            const T hr = fma(tnr[r], fr[r], fma(tni[r], fi[r], tpr[r]));
            const T hi = fma(tni[r], fr[r], fma(tnr[r], -fi[r], tpi[r]));
            if (W.out_c64)
                reinterpret_cast<float2 *>(W.out)[i] = make_float2((float)hr, (float)hi);
            else
                reinterpret_cast<double2 *>(W.out)[i] = make_double2((double)hr, (double)hi);
        }
    }
};

}  // namespace

template <typename V>
__global__ void __launch_bounds__(256) k_sum(const PlanHdr *__restrict__ hp)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_abort;
    const PlanHdr h = *hp;
    const int tid = threadIdx.x;
    const int U = blockDim.x * V::kSamples;
    const CtaStart beg = h.cta[blockIdx.x];
    const CtaStart end = h.cta[blockIdx.x + 1];
    int w = beg.wave, i = beg.sample;
    if (!normalize(h, w, i, end)) return;  // uniform across the CTA

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    // Producer state (thread 0): the last issued piece.
    Piece cur = piece_at(h, w, i, end);
    int prod_w = cur.w, prod_i1 = cur.i1;
    bool prod_more = true;
    auto issue = [&](const Piece &p, int b) {
        const WaveDev &P = h.waves[p.w];
        const uint32_t bytes = (uint32_t)P.tr.n_slots * (uint32_t)V::kSlotBytes;
        const unsigned char *src =
            reinterpret_cast<const unsigned char *>(P.fcoef) + (size_t)p.s * bytes;
        unsigned char *dst = smem + (size_t)b * h.buf_bytes;
        mbar_arrive_expect_tx(&bar[b], bytes);
        for (uint32_t off = 0; off < bytes; off += kBulkChunk) {
            const uint32_t n = min((uint32_t)kBulkChunk, bytes - off);
            bulk_g2s(dst + off, src + off, n, &bar[b]);
        }
    };
    auto issue_next = [&](int b) {
        int nw = prod_w, ni = prod_i1;
        if (prod_more && normalize(h, nw, ni, end)) {
            const Piece p = piece_at(h, nw, ni, end);
            issue(p, b);
            prod_w = p.w;
            prod_i1 = p.i1;
        } else {
            prod_more = false;
        }
    };
    if (tid == 0) {
        fence_proxy_async_smem();
        issue(cur, 0);
        issue_next(1);
    }

    int k = 0;
    for (;; ++k) {
        const int b = k & 1;
        if (!mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1))) s_abort = 1;
        __syncthreads();
        if (s_abort) break;

        const WaveDev &W = h.waves[cur.w];
        const unsigned char *buf = smem + (size_t)b * h.buf_bytes;
        PhaseSrc<typename V::Scalar> ps;
        ps.init(W, cur.s);
        const int warp_first = (tid & ~31) * V::kSamples;
        for (int p0 = cur.i0; p0 < cur.i1; p0 += U) {
            if (p0 + warp_first >= cur.i1) continue;  // whole warp past the end: idle
            V::run(W, buf, p0, cur.i1, ps);
        }

        int nw = cur.w, ni = cur.i1;
        if (!normalize(h, nw, ni, end)) break;
        cur = piece_at(h, nw, ni, end);
        __syncthreads();  // every thread is done with buffer b before it is refilled
        if (tid == 0) {
            fence_proxy_async_smem();
            issue_next(b);
        }
    }

    if (s_abort && tid == 0) {
        atomicOr(h.err, ERRBIT_TIMEOUT);
        // Give the copies still in flight (the one that expired, and the next piece's if it
        // was issued) a second bounded wait before the CTA exits and its shared memory goes.
        mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1));
        if (prod_more) mbar_wait_bounded(&bar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1));
    }
}

// Reduced orbital phases of every sample (the per-sample phase step on its own), in turns:
// out[2 i] = f_phi, out[2 i + 1] = f_r.  Segments follow the same sample ranges as k_sum.
__global__ void __launch_bounds__(256) k_phases(TrajDev tr, const int *__restrict__ seg_start,
                                                double t0, double dt, int n, double dphi_phi,
                                                double dphi_r, double2 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = tr.S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_start[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const SegPhase sp = seg_phase(tr, lo, dphi_phi, dphi_r);
    double fphi, fr, u;
    sample_phase(sp, t0, dt, i, fphi, fr, u);
    out[i] = make_double2(fphi, fr);
}

cudaError_t launch_phases(const TrajDev &tr, const int *seg_start, double t0, double dt, int n,
                          double dphi_phi, double dphi_r, double *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_phases<<<(n + 255) / 256, 256, 0, st>>>(tr, seg_start, t0, dt, n, dphi_phi, dphi_r,
                                               reinterpret_cast<double2 *>(out));
    return cudaGetLastError();
}

// Phase anchors of the mixed path, one thread per anchor: wave w, segment s and group q of the
// anchor, then at the anchor sample a = kAnchorGroup * q (which may precede the segment's first
// sample: the segment's cubic is used on both sides) the FP64 phases reduced modulo one turn and
// the Taylor coefficients of each phase cubic in sample units,
//   Phi(u + k du) - Phi(u) = k du Phi'(u) + (k du)^2 Phi''(u)/2 + (k du)^3 p3,  du = dt / h,
// divided by 2 pi (turns).  The identity is exact for a cubic; only its FP32 evaluation over
// k < kAnchorGroup samples in the summation kernel rounds.
__global__ void __launch_bounds__(256) k_anchor(const PlanHdr *__restrict__ hp)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_waves = hp->n_waves;
    if (g >= hp->total_anchors) return;
    const WaveDev *waves = hp->waves;
    int lo = 0, hi = n_waves - 1;
    while (lo < hi) {  // largest w with anchor_begin <= g
        const int mid = (lo + hi + 1) >> 1;
        if (waves[mid].anchor_begin <= g) lo = mid; else hi = mid - 1;
    }
    const WaveDev &W = waves[lo];
    const int j = g - W.anchor_begin;
    int s0 = 0, s1 = W.tr.S - 1;
    while (s0 < s1) {  // largest s with anchor_off[s] <= j
        const int mid = (s0 + s1 + 1) >> 1;
        if (W.anchor_off[mid] <= j) s0 = mid; else s1 = mid - 1;
    }
    const int s = s0;
    const int q = W.seg_start[s] / kAnchorGroup + (j - W.anchor_off[s]);
    const SegPhase sp = seg_phase(W.tr, s, W.dphi_phi, W.dphi_r);
    const double kInv2Pi = 0.15915494309189533577;
    const double t = fma((double)q * kAnchorGroup, W.dt, W.t0);
    const double u = (t - sp.tk) * sp.ih;
    const double du = W.dt * sp.ih, du2 = du * du, du3 = du2 * du;
    float f[2][4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double c0 = k ? sp.c0r : sp.c0phi;
        const double *p = k ? sp.pr : sp.pphi;
        const double ph = fma(fma(fma(p[2], u, p[1]), u, p[0]), u, c0);
        const double d1 = fma(fma(3.0 * p[2], u, 2.0 * p[1]), u, p[0]) * du;
        const double d2 = fma(3.0 * p[2], u, p[1]) * du2;
        const double d3 = p[2] * du3;
        const double x = ph * kInv2Pi;
        f[k][0] = (float)(x - rint(x));
        f[k][1] = (float)(d1 * kInv2Pi);
        f[k][2] = (float)(d2 * kInv2Pi);
        f[k][3] = (float)(d3 * kInv2Pi);
    }
    Anchor a;
    a.phi = make_float4(f[0][0], f[0][1], f[0][2], f[0][3]);
    a.r = make_float4(f[1][0], f[1][1], f[1][2], f[1][3]);
    W.anchors[j] = a;
}

cudaError_t launch_anchor(const PlanHdr *hdr_dev, int total_anchors, cudaStream_t st)
{
    if (total_anchors <= 0) return cudaSuccess;
    k_anchor<<<(total_anchors + 255) / 256, 256, 0, st>>>(hdr_dev);
    return cudaGetLastError();
}

namespace {
template <typename V>
cudaError_t configure_one(int max_dyn)
{
    return cudaFuncSetAttribute(k_sum<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
}
template <typename V>
int occupancy_one(int threads, int smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sum<V>, threads, smem) != cudaSuccess)
        return 0;
    return n;
}
template <typename V>
cudaError_t launch_one(const PlanHdr *hdr, int grid, int threads, int smem, cudaStream_t st)
{
    k_sum<V><<<grid, threads, smem, st>>>(hdr);
    return cudaGetLastError();
}
}  // namespace

int sum_slot_bytes(int variant) { return variant == kVariantFp64 ? 64 : 32; }

cudaError_t sum_configure()
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int max_dyn = optin - 1024;  // leaves room for the static mbarriers and flag
    if ((e = configure_one<ScalarPass<double, 1>>(max_dyn)) != cudaSuccess) return e;
    if ((e = configure_one<ScalarPass<double, 2>>(max_dyn)) != cudaSuccess) return e;
    if ((e = configure_one<ScalarPass<float, 2>>(max_dyn)) != cudaSuccess) return e;
    if ((e = configure_one<ScalarPass<float, 4>>(max_dyn)) != cudaSuccess) return e;
    if ((e = configure_one<ScalarPass<float, 8>>(max_dyn)) != cudaSuccess) return e;
    return cudaSuccess;
}

int sum_occupancy(int variant, int R, int threads, int smem)
{
    if (variant == kVariantFp64) {
        if (R == 1) return occupancy_one<ScalarPass<double, 1>>(threads, smem);
        if (R == 2) return occupancy_one<ScalarPass<double, 2>>(threads, smem);
    } else if (variant == kVariantScalar) {
        if (R == 2) return occupancy_one<ScalarPass<float, 2>>(threads, smem);
        if (R == 4) return occupancy_one<ScalarPass<float, 4>>(threads, smem);
        if (R == 8) return occupancy_one<ScalarPass<float, 8>>(threads, smem);
    }
    return 0;
}

cudaError_t launch_sum(const PlanHdr *hdr_dev, int grid, int threads, int R, int smem, int variant,
                       cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    if (variant == kVariantFp64) {
        if (R == 1) return launch_one<ScalarPass<double, 1>>(hdr_dev, grid, threads, smem, st);
        if (R == 2) return launch_one<ScalarPass<double, 2>>(hdr_dev, grid, threads, smem, st);
    } else if (variant == kVariantScalar) {
        if (R == 2) return launch_one<ScalarPass<float, 2>>(hdr_dev, grid, threads, smem, st);
        if (R == 4) return launch_one<ScalarPass<float, 4>>(hdr_dev, grid, threads, smem, st);
        if (R == 8) return launch_one<ScalarPass<float, 8>>(hdr_dev, grid, threads, smem, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fewsum
