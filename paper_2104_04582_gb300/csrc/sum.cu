// sum.cu -- per-sample interpolation and mode sum (arXiv:2104.04582 Sec. 3.C, Sec. 4 sum).
//
// At every dense sample t_i the kernel evaluates
//     h(t_i) = sum_{(m,n) signed} K_{m,n}(u) z_phi^m z_r^n,
//     z_phi = e^{-i Phi_phi(t_i)},  z_r = e^{-i Phi_r(t_i)},  u = (t_i - t_k)/h_k,
// where K_{m,n} are the per-segment complex cubics produced by k_fold (amplitude splines with
// the spin-weighted harmonics, the m < 0 partners of Eq. amp_symmetry and the prefactor folded
// in).  Since e^{-i Phi_mn} = z_phi^m z_r^n exactly, the whole sum is a bivariate Laurent
// polynomial in (z_phi, z_r) and is evaluated by Horner's rule.  The slot table is laid out in
// rows of constant signed m, from the largest m down to m_last; row j holds n = hi_j .. lo_j.
// One Horner chain in z_r per row gives A_j = sum_n K_{m_j,n} z_r^{n - lo_j}; the rows are
// combined by Horner's rule in z_phi in a frame shifted by each row's lowest n,
//     T_j = T_{j-1} z_phi z_r^{lo_{j-1} - lo_j} + A_j,     h = T_last z_phi^{m_last} z_r^{lo_last},
// so a row with no gap to its neighbour's lowest n costs one complex multiply and no power is
// formed per row.  Per (slot, sample) that is one complex cubic (6 FMA) and one complex
// multiply-add (4 FMA) -- no transcendental per mode.
//
// Phases: FEW_FP64 evaluates the phase splines (in rad) in FP64 for every sample and reduces
// each phase modulo one turn, x - rint(x), in FP64; the reduced phases give z_phi, z_r and the
// final factor (sincospi).  FEW_MIXED reads the phases from anchors written by k_anchor: at
// every kAnchorGroup-th sample the FP64 splines are evaluated and reduced modulo one turn (and
// the final factor's phase m_last Phi_phi + lo_last Phi_r formed from the reduced phases and
// reduced again, all in FP64), and each phase cubic's exact Taylor coefficients about that
// sample (in turns per sample^k) are stored; the kernel adds the in-group increment
// r (d1 + r (d2 + r d3)), r < kAnchorGroup, in FP32.  So every large phase value and every
// reduction is FP64, and the mixed kernel issues no FP64 instruction per sample (FP64 issue is
// scarce on this chip).  FEW_FP64 does everything else in FP64; FEW_MIXED evaluates amplitudes,
// exponential powers and the accumulation in FP32.
//
// Work decomposition: a persistent grid; each CTA owns a contiguous slice of the concatenated
// (waveform, sample) space, cut at pass boundaries with equal pass cost per slice (a pass costs
// threads x R samples x slots whether or not its segment ends first), and walks it segment by
// segment in passes of threads x R consecutive samples, R per thread (a warp owns 32 R of them,
// its lanes strided by 32), each thread holding its samples' Horner state in registers.  The
// segment's folded coefficient table is streamed into
// shared memory once per pass, in tiles of stage_slots slots (the mode tile), through a ring of
// `ring` stages: the last warp to release a stage issues the TMA bulk copies (cp.async.bulk with
// mbarrier transaction counts) of the tile `ring` positions ahead into it, so no warp ever waits
// for a stage to empty, a table of any size passes through a fixed amount of shared memory, and
// every coefficient read from it is reused R times.  Every wait is bounded: it gives up after
// 2 s, latches FEW_ERR_TIMEOUT and the CTA winds down (letting its copies in flight land).
// Every sample is summed by one thread in a fixed slot order, so results do not depend on the
// grid, the tile shape or on which other waveforms share the launch.
#include "fewsum_internal.h"
#include "phase_eval.cuh"
#include "async.cuh"

namespace fewsum {

namespace {

constexpr int kSlotUnroll = 8;  // slots per iteration of the Horner chain loop
// R = 8 already issues 40 packed FMA per slot, so four slots per iteration keep the pipe fed and
// leave a one-slot remainder on a 61-slot row instead of five (0.7 % faster than eight).
constexpr int kSlotUnrollR8 = 4;
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

// Per-sample local coordinate u, the powers' bases (cos, sin of 2 pi f) of one segment, and the
// final factor z_phi^{m_last} z_r^{lo_last} = e^{-2 pi i g}.
template <typename T> struct PhaseSrc;

// FP64: both phase splines evaluated and reduced for every sample.
template <> struct PhaseSrc<double> {
    SegPhase sp;
    double t0, dt;
    int m_last, lo_last;
    __device__ __forceinline__ void init(const WaveDev &W, int s)
    {
        sp = seg_phase(W.tr, s, W.dphi_phi, W.dphi_r);
        t0 = W.t0;
        dt = W.dt;
        m_last = W.tr.m_last;
        lo_last = W.tr.lo_last;
    }
    __device__ __forceinline__ void at(int i, double &u, double &cphi, double &sphi, double &cr,
                                       double &sr) const
    {
        double fphi, fr;
        sample_phase(sp, t0, dt, i, fphi, fr, u);
        sincospi(2.0 * fphi, &sphi, &cphi);
        sincospi(2.0 * fr, &sr, &cr);
    }
    // cos and sin of 2 pi g, g = m_last f_phi + lo_last f_r reduced modulo one turn
    __device__ __forceinline__ void last(int i, double &cg, double &sg) const
    {
        double fphi, fr, u;
        sample_phase(sp, t0, dt, i, fphi, fr, u);
        const double g = fma((double)m_last, fphi, (double)lo_last * fr);
        sincospi(2.0 * (g - rint(g)), &sg, &cg);
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
    __device__ __forceinline__ static float phase(const float4 a, float x)
    {
        return fmaf(fmaf(fmaf(a.w, x, a.z), x, a.y), x, a.x);
    }
    __device__ __forceinline__ void at(int i, float &u, float &cphi, float &sphi, float &cr,
                                       float &sr) const
    {
        const Anchor *a = anc + aidx + i / kAnchorGroup;
        const float4 ap = __ldg(&a->phi), ar = __ldg(&a->r);
        const float x = (float)(i % kAnchorGroup);
        sincospif(2.0f * phase(ap, x), &sphi, &cphi);
        sincospif(2.0f * phase(ar, x), &sr, &cr);
        u = fmaf((float)(i - i0), du, u0);
    }
    __device__ __forceinline__ void last(int i, float &cg, float &sg) const
    {
        const Anchor *a = anc + aidx + i / kAnchorGroup;
        const float4 ag = __ldg(&a->g);
        sincospif(2.0f * phase(ag, (float)(i % kAnchorGroup)), &sg, &cg);
    }
};

// acc <- acc * z + K(u) along n consecutive slots (Horner in z = (zr, zi)).
// The cubic in Estrin's form, (c0 + c1 u) + u^2 (c2 + c3 u), and the complex step with the
// a z products first: the same 10 FMA per (slot, sample) as Horner's form, in an operand order
// that measured 2.5 % faster on GB300 (fewer register-operand dispatch stalls).
// FP32 form of the same chain on packed pairs: samples 2q and 2q+1 share one float2, and every
// FMA above becomes one packed FMA (fma.rn.f32x2) on the pair -- the same operands and rounding
// per lane, so the results are bit-identical to the scalar form, in half the issued instructions
// (the scalar chain is bounded by instruction issue, not by the FMA pipe).  Each slot's
// coefficient is broadcast to both lanes of a pair.
template <int R>
__device__ __forceinline__ void horner_chain_f32x2(const float *__restrict__ cf, int n,
                                                   const float (&u)[R], const float (&zr)[R],
                                                   const float (&zi)[R], float (&ar)[R],
                                                   float (&ai)[R])
{
    static_assert(R % 2 == 0, "samples are paired");
    constexpr int Q = R / 2;
    float2 U[Q], U2[Q], ZR[Q], ZI[Q], NZI[Q], AR[Q], AI[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        U[q] = make_float2(u[2 * q], u[2 * q + 1]);
        U2[q] = make_float2(u[2 * q] * u[2 * q], u[2 * q + 1] * u[2 * q + 1]);
        ZR[q] = make_float2(zr[2 * q], zr[2 * q + 1]);
        ZI[q] = make_float2(zi[2 * q], zi[2 * q + 1]);
        NZI[q] = make_float2(-zi[2 * q], -zi[2 * q + 1]);
        AR[q] = make_float2(ar[2 * q], ar[2 * q + 1]);
        AI[q] = make_float2(ai[2 * q], ai[2 * q + 1]);
    }
    constexpr int kUnroll = R >= 8 ? kSlotUnrollR8 : kSlotUnroll;
#pragma unroll (kUnroll)
    for (int k = 0; k < n; ++k) {
        float c[8];
        Cf<float>::load(cf + 8 * k, c);
        float2 C[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) C[i] = make_float2(c[i], c[i]);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const float2 kr = __ffma2_rn(__ffma2_rn(C[3], U[q], C[2]), U2[q], __ffma2_rn(C[1], U[q], C[0]));
            const float2 ki = __ffma2_rn(__ffma2_rn(C[7], U[q], C[6]), U2[q], __ffma2_rn(C[5], U[q], C[4]));
            const float2 nr = __ffma2_rn(AI[q], NZI[q], __ffma2_rn(AR[q], ZR[q], kr));
            const float2 ni = __ffma2_rn(AI[q], ZR[q], __ffma2_rn(AR[q], ZI[q], ki));
            AR[q] = nr;
            AI[q] = ni;
        }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        ar[2 * q] = AR[q].x;
        ar[2 * q + 1] = AR[q].y;
        ai[2 * q] = AI[q].x;
        ai[2 * q + 1] = AI[q].y;
    }
}

template <typename T, int R>
__device__ __forceinline__ void horner_chain(const T *__restrict__ cf, int n, const T (&u)[R],
                                             const T (&zr)[R], const T (&zi)[R], T (&ar)[R],
                                             T (&ai)[R])
{
    if constexpr (sizeof(T) == sizeof(float) && R % 2 == 0) {
        horner_chain_f32x2<R>(cf, n, u, zr, zi, ar, ai);
    } else {
        T u2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u2[r] = u[r] * u[r];
#pragma unroll (kSlotUnroll)
        for (int k = 0; k < n; ++k) {
            T c[8];
            Cf<T>::load(cf + 8 * k, c);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T kr = fma(fma(c[3], u[r], c[2]), u2[r], fma(c[1], u[r], c[0]));
                const T ki = fma(fma(c[7], u[r], c[6]), u2[r], fma(c[5], u[r], c[4]));
                const T nr = fma(-ai[r], zi[r], fma(ar[r], zr[r], kr));
                const T ni = fma(ai[r], zr[r], fma(ar[r], zi[r], ki));
                ar[r] = nr;
                ai[r] = ni;
            }
        }
    }
}

// Shared-memory ring of the coefficient tiles.  A stage is refilled by the last consumer warp
// to release it (a per-stage arrival counter), so no thread ever waits for a stage to empty.
struct Ring {
    unsigned char *buf;   // ring x stage_bytes
    uint64_t *full;       // [ring] transaction barrier of the tile in the stage
    int *count;           // [ring] warps done with the stage's current tile
    int *issued;          // [ring] CTA stage index last copied into the stage (-1: none)
    volatile int *abort;
    int ring, stage_slots, stage_bytes, n_warps;
};

// Position in the CTA's sequence of tiles: piece (wave, segment, samples), pass, tile.
struct Walk {
    int w, i;          // wave and first sample of the current piece
    int s, i1;         // its segment and end
    int n_tiles, n_pass, pass, tile;
    bool valid;
};

__device__ __forceinline__ void walk_piece(Walk &a, const PlanHdr &h, const CtaStart &end, int U,
                                           int stage_slots)
{
    a.valid = normalize(h, a.w, a.i, end);
    if (!a.valid) return;
    const Piece pc = piece_at(h, a.w, a.i, end);
    a.s = pc.s;
    a.i1 = pc.i1;
    a.n_tiles = (h.waves[pc.w].tr.n_slots + stage_slots - 1) / stage_slots;
    a.n_pass = (pc.i1 - pc.i0 + U - 1) / U;
    a.pass = 0;
    a.tile = 0;
}

__device__ __forceinline__ void walk_next(Walk &a, const PlanHdr &h, const CtaStart &end, int U,
                                          int stage_slots)
{
    if (!a.valid) return;
    if (++a.tile < a.n_tiles) return;
    a.tile = 0;
    if (++a.pass < a.n_pass) return;
    a.i = a.i1;
    walk_piece(a, h, end, U, stage_slots);
}

// Copy the tile at `a` into stage b (one thread): its slots of the segment's folded table.
template <typename T>
__device__ void issue_tile(const PlanHdr &h, const Walk &a, int b, int k, const Ring &rg)
{
    constexpr int kSlotBytes = 8 * (int)sizeof(T);
    const WaveDev &W = h.waves[a.w];
    const int n_slots = W.tr.n_slots;
    const int first = a.tile * rg.stage_slots;
    const uint32_t bytes = (uint32_t)(min(rg.stage_slots, n_slots - first) * kSlotBytes);
    const unsigned char *src = reinterpret_cast<const unsigned char *>(W.fcoef) +
                               ((size_t)a.s * n_slots + first) * kSlotBytes;
    unsigned char *dst = rg.buf + (size_t)b * rg.stage_bytes;
    rg.issued[b] = k;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&rg.full[b], bytes);
    for (uint32_t off = 0; off < bytes; off += kBulkChunk)
        bulk_g2s(dst + off, src + off, min((uint32_t)kBulkChunk, bytes - off), &rg.full[b]);
}

// A warp is done with stage b (CTA stage index k): the last warp to say so refills the stage
// with tile k + ring (the walk `ahead` points there), if the CTA has one.
template <typename T>
__device__ __forceinline__ void release_stage(const PlanHdr &h, const Walk &ahead, int b, int k,
                                              const Ring &rg)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence_block();  // this warp's reads of the stage come before the refill
        if (atomicAdd(&rg.count[b], 1) == rg.n_warps - 1) {
            __threadfence_block();
            rg.count[b] = 0;
            if (ahead.valid) issue_tile<T>(h, ahead, b, k + rg.ring, rg);
        }
    }
}

// One pass of the consumer warps over piece [.., i1), every tile of the segment's table in turn
// (CTA stage indices k0, k0 + 1, ...).  Warp w owns the 32 R samples from p0 + 32 R w, its lane
// l the samples p0 + 32 R w + 32 r + l (r < R): each output store of the warp then covers 32
// consecutive samples (whole 128-byte lines, which matters when the output is host memory
// reached over the chip-to-chip link), and a warp past the end of a short pass skips it whole.
// Warps with no sample in the pass still take part in the tile hand-over.  False if a wait gave
// up.
template <typename T, int R>
__device__ bool consume_pass(const PlanHdr &h, const WaveDev &W, const PhaseSrc<T> &ps, int p0,
                             int i1, bool active, const Ring &rg, int k0, int n_tiles, Walk &ahead,
                             const CtaStart &end, int U)
{
    const int tid = threadIdx.x;
    const int base = p0 + (tid & ~31) * R + (tid & 31);  // sample r of the thread: base + 32 r
    T u[R], zr[R], zi[R], fr[R], fi[R], tr_[R], ti_[R], ar[R], ai[R];
    const int2 *__restrict__ rows = W.tr.rows;
    const int n_rows = W.tr.n_rows, n_slots = W.tr.n_slots;
    int row = 0, row_left = 0;
    if (active) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = min(base + 32 * r, i1 - 1);
            T sp_, cp, sr, cr;
            ps.at(i, u[r], cp, sp_, cr, sr);
            fr[r] = cp;   // z_phi = e^{-i 2 pi f_phi}
            fi[r] = -sp_;
            zr[r] = cr;   // z_r = e^{-i 2 pi f_r}
            zi[r] = -sr;
            tr_[r] = ti_[r] = ar[r] = ai[r] = (T)0;
        }
        row_left = __ldg(rows).x;
    }
    // close every finished row: T <- T z_phi z_r^{shift} + A, then start the next row
    auto close_rows = [&]() {
        while (row < n_rows && row_left == 0) {
            const int shift = __ldg(rows + row).y;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T nr = fma(tr_[r], fr[r], -ti_[r] * fi[r]);
                const T ni = fma(tr_[r], fi[r], ti_[r] * fr[r]);
                tr_[r] = nr;
                ti_[r] = ni;
            }
            for (int d = 0; d < (shift < 0 ? -shift : shift); ++d) {
                const T s = shift < 0 ? (T)-1 : (T)1;  // z_r or conj(z_r)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T nr = fma(tr_[r], zr[r], -ti_[r] * (s * zi[r]));
                    const T ni = fma(tr_[r], s * zi[r], ti_[r] * zr[r]);
                    tr_[r] = nr;
                    ti_[r] = ni;
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                tr_[r] += ar[r];
                ti_[r] += ai[r];
                ar[r] = ai[r] = (T)0;
            }
            if (++row < n_rows) row_left = __ldg(rows + row).x;
        }
    };
    if (active) close_rows();  // leading empty rows (none in a well-formed plan)
    for (int t = 0; t < n_tiles; ++t) {
        const int k = k0 + t;
        const int b = k % rg.ring;
        if (*rg.abort) return false;
        if (!mbar_wait_bounded(&rg.full[b], (uint32_t)(k / rg.ring) & 1u)) {
            *rg.abort = 1;
            return false;
        }
        if (active) {
            const T *__restrict__ cf = reinterpret_cast<const T *>(rg.buf + (size_t)b * rg.stage_bytes);
            const int a = t * rg.stage_slots;
            const int e = min(a + rg.stage_slots, n_slots);
            int slot = a;
            while (slot < e) {
                const int n = min(row_left, e - slot);
                if (n <= 0) break;  // slots beyond the last row: an inconsistent plan, never hang
                horner_chain<T, R>(cf + 8 * (slot - a), n, u, zr, zi, ar, ai);
                slot += n;
                row_left -= n;
                if (row_left == 0) close_rows();
            }
        }
        release_stage<T>(h, ahead, b, k, rg);
        walk_next(ahead, h, end, U, rg.stage_slots);
    }
    if (active) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = base + 32 * r;
            if (i >= i1) break;
            // h = T z_phi^{m_last} z_r^{lo_last}
            T cg, sg;
            ps.last(i, cg, sg);
            const T hr = fma(tr_[r], cg, ti_[r] * sg);   // (tr + i ti)(cg - i sg)
            const T hi = fma(ti_[r], cg, -tr_[r] * sg);
            if (W.out_c64)
                reinterpret_cast<float2 *>(W.out)[i] = make_float2((float)hr, (float)hi);
            else
                reinterpret_cast<double2 *>(W.out)[i] = make_double2((double)hr, (double)hi);
        }
    }
    return true;
}


// R samples per thread; T the arithmetic type (float: FEW_MIXED, double: FEW_FP64); MB the
// resident CTAs per SM that the register budget is sized for.
template <typename T, int R, int MB = 2>
struct ScalarPass {
    using Scalar = T;
    static constexpr int kSamples = R;
    static constexpr int kMinBlocks = MB;
};

// R = 8 holds four packed sample pairs of state and the coefficients of the slots in flight in
// 218 registers: one 256-thread CTA per SM (a budget for two caps it at 128 registers and
// spills).  Eight warps per SM then run the packed FMA chain faster than sixteen at R = 4.
using MixedR8 = ScalarPass<float, 8, 1>;

}  // namespace

// blockDim.x consumer threads (all of them compute; the refills are issued by whichever warp
// releases a stage last).
template <typename V>
__global__ void __launch_bounds__(kSumMaxThreads, V::kMinBlocks) k_sum(const PlanHdr *__restrict__ hp)
{
    using T = typename V::Scalar;
    constexpr int R = V::kSamples;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_full[kMaxRing];
    __shared__ int s_count[kMaxRing], s_issued[kMaxRing];
    __shared__ int s_abort, s_exit;
    const PlanHdr h = *hp;
    const int tid = threadIdx.x;
    const int U = blockDim.x * R;
    const CtaStart beg = h.cta[blockIdx.x];
    const CtaStart end = h.cta[blockIdx.x + 1];
    {
        int w = beg.wave, i = beg.sample;
        if (!normalize(h, w, i, end)) return;  // uniform across the CTA: no work
    }
    Ring rg;
    rg.buf = smem;
    rg.full = s_full;
    rg.count = s_count;
    rg.issued = s_issued;
    rg.abort = &s_abort;
    rg.ring = h.ring;
    rg.stage_slots = h.stage_slots;
    rg.stage_bytes = h.buf_bytes;
    rg.n_warps = blockDim.x / 32;
    if (tid == 0) {
        for (int b = 0; b < rg.ring; ++b) {
            mbar_init(&rg.full[b], 1);
            s_count[b] = 0;
            s_issued[b] = -1;
        }
        fence_mbar_init();
        s_abort = 0;
        s_exit = 0;
    }
    __syncthreads();

    // `ahead` walks `ring` tiles in front of this warp's position; thread 0 fills the ring first
    Walk ahead;
    ahead.w = beg.wave;
    ahead.i = beg.sample;
    walk_piece(ahead, h, end, U, rg.stage_slots);
    for (int k = 0; k < rg.ring; ++k) {
        if (tid == 0 && ahead.valid) issue_tile<T>(h, ahead, k, k, rg);
        walk_next(ahead, h, end, U, rg.stage_slots);
    }

    int k = 0;
    const int warp_first = (tid & ~31) * R;
    int w = beg.wave, i = beg.sample;
    bool ok = true;
    while (ok && normalize(h, w, i, end)) {
        const Piece pc = piece_at(h, w, i, end);
        const WaveDev &W = h.waves[pc.w];
        PhaseSrc<T> ps;
        ps.init(W, pc.s);
        const int n_tiles = (W.tr.n_slots + rg.stage_slots - 1) / rg.stage_slots;
        for (int p0 = pc.i0; p0 < pc.i1 && ok; p0 += U) {
            const bool active = p0 + warp_first < pc.i1;  // else the whole warp is past the end
            ok = consume_pass<T, R>(h, W, ps, p0, pc.i1, active, rg, k, n_tiles, ahead, end, U);
            k += n_tiles;
        }
        w = pc.w;
        i = pc.i1;
    }
    if ((tid & 31) == 0) {
        if (!ok) atomicOr(h.err, ERRBIT_TIMEOUT);
        __threadfence_block();
        // the last warp out lets every copy still in flight land before the CTA's shared
        // memory goes away (immediate when everything issued was consumed)
        if (atomicAdd(&s_exit, 1) == rg.n_warps - 1) {
            __threadfence_block();
            for (int b = 0; b < rg.ring; ++b) {
                const int kk = s_issued[b];
                if (kk >= 0) mbar_wait_bounded(&rg.full[b], (uint32_t)(kk / rg.ring) & 1u);
            }
        }
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
    if ((e = configure_one<MixedR8>(max_dyn)) != cudaSuccess) return e;
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
        if (R == 8) return occupancy_one<MixedR8>(threads, smem);
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
        if (R == 8) return launch_one<MixedR8>(hdr_dev, grid, threads, smem, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fewsum
