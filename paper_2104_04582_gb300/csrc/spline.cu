// spline.cu -- batched not-a-knot cubic spline build (arXiv:2104.04582 Sec. 3.C).
//
// Every real array on a trajectory grid (Phi_phi, Phi_r and Re/Im of every mode amplitude,
// J = 2 + 2N arrays) gets a not-a-knot cubic spline on the shared knots.  The unknowns are the
// knot slopes s_k; the interior rows are the C2 conditions
//     h_k s_{k-1} + 2 (h_{k-1} + h_k) s_k + h_{k-1} s_{k+1} = 3 (h_k d_{k-1} + h_{k-1} d_k)
// and the two end rows express a continuous third derivative at t_1 and t_{K-2} (reduced to
// tridiagonal form by eliminating s_2 / s_{K-3}):
//     h_1 s_0 + (h_0 + h_1) s_1 = ((2 h_1 + 3 h_0) h_1 d_0 + h_0^2 d_1) / (h_0 + h_1)
//     (h_{K-2} + h_{K-3}) s_{K-2} + h_{K-3} s_{K-1}
//         = (h_{K-2}^2 d_{K-3} + (2 h_{K-3} + 3 h_{K-2}) h_{K-3} d_{K-2}) / (h_{K-3} + h_{K-2}).
// Substituting the end rows' s_0 and s_{K-1} into rows 1 and K-2 leaves a strictly diagonally
// dominant tridiagonal system for s_1 .. s_{K-2}:
//     row 1:    (h_0 + h_1) s_1 + h_0 s_2 = r_1 - R_0,
//     row K-2:  h_{K-2} s_{K-3} + (h_{K-3} + h_{K-2}) s_{K-2} = r_{K-2} - R_L,
// (R_0, R_L the end rows' right-hand sides), interior rows as above.  Its matrix depends only on
// the knots, so it is factorised once per trajectory (k_factor), partitioned into up to
// kBuildParts blocks separated by single rows; every spline then reuses the factors with
// kBuildParts lanes (k_build): each lane solves one block, the lanes combine through the small
// separator system, s_0 and s_{K-1} follow from the end rows, and each lane stores the Hermite
// data (y_k, y_{k+1}, s_k, s_{k+1}) of the segments next to its rows.  A spline's solve is thus
// several short chains of FP64 operations in parallel instead of one long one (FP64 latency is
// long on this chip), and the build issues only the solve's FP64 operations (the cubic's power
// coefficients, hermite_to_power, are formed by the consumers: in FP32 by the mixed fold).  The
// two phase arrays are fitted in radians as given (their reduction modulo 2 pi happens per
// segment and per sample in the summation kernel).
#include "fewsum_internal.h"

namespace fewsum {

constexpr int kFactorThreads = 32;  // one warp: per-knot loops strided, one thread per block

// Partitioned factorisation of the reduced not-a-knot matrix of one knot grid (one warp; O(K)
// work, each block's elimination on its own thread), rows k = 1..K-2 with diagonal dg(k), lower
// coefficient sub(k) = h_k (k >= 2) and upper sup(k) = h_{k-1} (k <= K-3).  The rows are split into P blocks separated by single rows (the
// separators): block b spans rows start_b .. start_b + size_b - 1, separator b + 1 is the row
// after it.  With x_sigma the separators' unknowns, block b's rows solve
//     A_b x_b = f_b - sub(first) x_{sigma_b} e_first - sup(last) x_{sigma_{b+1}} e_last,
// i.e. x_b = y_b - x_{sigma_b} v_b - x_{sigma_{b+1}} w_b with y_b = A_b^-1 f_b and the spline-
// independent responses v_b = A_b^-1 sub(first) e_first, w_b = A_b^-1 sup(last) e_last; the
// separator rows then form a tridiagonal system in the x_sigma alone,
//     (dg - sub w_{b-1}[last] - sup v_b[first]) x_sigma - sub v_{b-1}[last] x_{sigma_{b-1}}
//         - sup w_b[first] x_{sigma_{b+1}} = f_sigma - sub y_{b-1}[last] - sup y_b[first].
// Within a block, Thomas elimination with every row divided by its pivot p_k gives
//     g_k = (ra_k D_{k-1} + rb_k D_k)/p_k - (sub(k)/p_k) g_{k-1},   y_k = g_k - (sup(k)/p_k) y_{k+1}
// (D_k = y_{k+1} - y_k), one operation fewer per row than the unscaled form.  Stored per row:
// ra, rb (divided by p_k on block rows), lo = sub/p_k (0 on a block's first row), up = sup/p_k,
// ip = 1/p_k, v, x = w on block rows; on a separator row: ra, rb plain, v = its multiplier in the
// separator elimination, ip = inverse pivot, x = the coupling to the next separator.
// parts[0] = P, parts[1 + b] = start_b, parts[1 + P] = K - 1.  Every block matrix and the
// separator system are strictly diagonally dominant, so no pivoting is needed.
//
// The end rows: in differences the interior right-hand side is 3 (h_k/h_{k-1}) D_{k-1} +
// 3 (h_{k-1}/h_k) D_k, and R_0 = (2 h_1 + 3 h_0) h_1 D_0/(h_0 (h_0 + h_1)) + h_0^2 D_1/(h_1 (h_0 +
// h_1)), so row 1's r_1 - R_0 has the coefficients h_1^2/(h_0 (h_0 + h_1)) and h_0 (2 h_0 +
// 3 h_1)/(h_1 (h_0 + h_1)); mirrored (hc = h_{K-3}, hd = h_{K-2}) row K-2's r_{K-2} - R_L has
// hd (3 hc + 2 hd)/(hc (hc + hd)) and hc^2/(hd (hc + hd)).  Rows 0 and K-1 hold the end slopes
//     s_0 = ra_0 D_0 + rb_0 D_1 - lo_0 s_1,   s_{K-1} = ra_{K-1} D_{K-3} + rb_{K-1} D_{K-2} -
//     lo_{K-1} s_{K-2}
// (the end rows divided by h_1 and hc).  K >= 4, so rows 1 and K-2 are distinct, and neither is
// a separator.
__global__ void __launch_bounds__(kFactorThreads) k_factor(const double *__restrict__ t, int K,
                                                             FactorArrays f)
{
    if (blockIdx.x != 0) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    double *h = f.h, *ip = f.ip, *fl = f.lo, *fu = f.up, *fv = f.v, *fx = f.x, *ra = f.ra,
           *rb = f.rb;
    const int S = K - 1, n = K - 2;
    // knot widths and cleared arrays (every thread a stride of k)
    for (int k = tid; k < S; k += nt) {
        h[k] = t[k + 1] - t[k];
        f.inv_h[k] = 1.0 / h[k];
    }
    for (int k = tid; k < K; k += nt) ip[k] = fl[k] = fu[k] = fv[k] = fx[k] = ra[k] = rb[k] = 0.0;
    constexpr int NS = kBuildParts - 1;
    for (int i = tid; i < NS * NS; i += nt) f.sinv[i] = 0.0;
    __syncthreads();
    auto dg = [&](int k) {
        if (k == 1) return h[0] + h[1];
        if (k == K - 2) return h[K - 3] + h[K - 2];
        return 2.0 * (h[k - 1] + h[k]);
    };
    auto sub = [&](int k) { return k >= 2 ? h[k] : 0.0; };
    auto sup = [&](int k) { return k <= K - 3 ? h[k - 1] : 0.0; };
    for (int k = 2 + tid; k <= K - 3; k += nt) {
        ra[k] = 3.0 * h[k] * f.inv_h[k - 1];
        rb[k] = 3.0 * h[k - 1] * f.inv_h[k];
    }
    const double h0 = h[0], h1 = h[1], hc = h[K - 3], hd = h[K - 2];
    if (tid == 0) {
        ra[1] = h1 * h1 / (h0 * (h0 + h1));
        rb[1] = h0 * (2.0 * h0 + 3.0 * h1) / (h1 * (h0 + h1));
        ra[K - 2] = hd * (3.0 * hc + 2.0 * hd) / (hc * (hc + hd));
        rb[K - 2] = hc * hc / (hd * (hc + hd));
    }
    // the partition (every thread derives the same)
    int P = (n + 1) / 2;
    if (P > kBuildParts) P = kBuildParts;
    if (P < 1) P = 1;
    const int nb = n - (P - 1), base = nb / P, extra = nb % P;
    int start[kBuildParts + 1];
    int k = 1;
    for (int b = 0; b < P; ++b) {
        start[b] = k;
        k += base + (b < extra ? 1 : 0) + 1;  // block rows, then its right separator
    }
    start[P] = K - 1;
    if (tid == 0) {
        f.parts[0] = P;
        for (int b = 0; b <= P; ++b) f.parts[1 + b] = start[b];
    }
    __syncthreads();
    // each block's elimination, responses and scaled rows: independent, one thread per block
    for (int b = tid; b < P; b += nt) {
        const int a = start[b], e = (b + 1 < P ? start[b + 1] - 1 : K - 1) - 1;
        double p = dg(a);
        ip[a] = 1.0 / p;
        for (int r = a + 1; r <= e; ++r) {  // fl holds the Thomas multipliers for now
            const double m = sub(r) / p;
            p = dg(r) - m * sup(r - 1);
            fl[r] = m;
            ip[r] = 1.0 / p;
        }
        if (b > 0) {  // v_b = A_b^-1 sub(a) e_first
            fv[a] = sub(a);
            for (int r = a + 1; r <= e; ++r) fv[r] = -fl[r] * fv[r - 1];
            fv[e] *= ip[e];
            for (int r = e - 1; r >= a; --r) fv[r] = (fv[r] - sup(r) * fv[r + 1]) * ip[r];
        }
        if (b + 1 < P) {  // w_b = A_b^-1 sup(e) e_last
            fx[e] = sup(e) * ip[e];
            for (int r = e - 1; r >= a; --r) fx[r] = -sup(r) * fx[r + 1] * ip[r];
        }
        for (int r = a; r <= e; ++r) {  // the pivot-scaled rows
            fl[r] = r > a ? sub(r) * ip[r] : 0.0;
            fu[r] = sup(r) * ip[r];
            ra[r] *= ip[r];
            rb[r] *= ip[r];
        }
    }
    __syncthreads();
    // the separator system's elimination (sequential, P - 1 <= 7 rows) and the end slopes
    if (tid == 0) {
        double piv = 0.0, cup_prev = 0.0;
        for (int i = 1; i < P; ++i) {
            const int sg = start[i] - 1, L = sg - 1, F = sg + 1;
            const double D = dg(sg) - sub(sg) * fx[L] - sup(sg) * fv[F];
            const double clo = -sub(sg) * fv[L], cup = -sup(sg) * fx[F];
            double mu = 0.0;
            if (i == 1) {
                piv = D;
            } else {
                mu = clo / piv;
                piv = D - mu * cup_prev;
            }
            fv[sg] = mu;
            ip[sg] = 1.0 / piv;
            fx[sg] = cup;
            cup_prev = cup;
        }
        ra[0] = (2.0 * h1 + 3.0 * h0) / (h0 * (h0 + h1));
        rb[0] = h0 * h0 / (h1 * h1 * (h0 + h1));
        fl[0] = (h0 + h1) / h1;
        ra[K - 1] = hd * hd / (hc * hc * (hc + hd));
        rb[K - 1] = (2.0 * hc + 3.0 * hd) / (hd * (hc + hd));
        fl[K - 1] = (hc + hd) / hc;
    }
    __syncthreads();
    // the separator system's inverse, column m from the unit right-hand side e_m (one thread per
    // column; entries past P - 1 stay zero): every lane of a spline then forms its right
    // separator's slope as one short dot product instead of a chain of 3 (P - 1) dependent
    // operations
    for (int m = 1 + tid; m < P; m += nt) {
        double gp[kBuildParts], X[kBuildParts + 1];
        for (int i = 1; i < P; ++i) {
            const double gi = i == m ? 1.0 : 0.0;
            gp[i] = i == 1 ? gi : gi - fv[start[i] - 1] * gp[i - 1];
        }
        X[P] = 0.0;
        for (int i = P - 1; i >= 1; --i)
            X[i] = (gp[i] - fx[start[i] - 1] * X[i + 1]) * ip[start[i] - 1];
        for (int i = 1; i < P; ++i) f.sinv[(i - 1) * NS + (m - 1)] = X[i];
    }
}

cudaError_t launch_factor(const double *t, int K, const FactorArrays &f, cudaStream_t st)
{
    k_factor<<<1, kFactorThreads, 0, st>>>(t, K, f);
    return cudaGetLastError();
}

__device__ __forceinline__ double load_y(const BuildJob &jb, int j, int k)
{
    if (j == 0) return jb.phi_phi[k];
    if (j == 1) return jb.phi_r[k];
    const int i = (j - 2) >> 1;
    const size_t idx = (size_t)k * jb.tr.N + i;
    return ((j - 2) & 1) ? jb.amp_im[idx] : jb.amp_re[idx];
}

// Bit 31 of the result is set iff x is infinite or NaN (exponent field all ones): the exponent
// field plus one carries into the sign position only from 0x7ff.  Integer pipe only, so the
// finiteness screen of the build takes nothing from the narrow FP64 pipe.
__device__ __forceinline__ unsigned nonfinite_bit(double x)
{
    return ((unsigned)__double2hiint(x) & 0x7ff00000u) + 0x00100000u;
}

// kBuildParts lanes per spline column (a spline's lanes are consecutive in a warp): lane b
// solves block b of the partitioned system (the pivot-scaled forward and back substitution with
// the shared factors, its values parked), the lanes exchange their blocks' end values by
// shuffles, every lane forms its right separator's slope from the separator system's inverse,
// and lane b corrects its rows, x = y - x_left v - x_right w.  The knot-only arrays are staged in
// shared memory; column values are fetched kChunk rows ahead.
//   kShared (K <= kBuildSharedKnots): values and slopes are parked in shared memory, [K][8
//     splines], and the block writes the Hermite data of its 8 consecutive columns together at
//     the end (a segment's 8 columns are 256 contiguous bytes).
//   otherwise: values are parked in the trajectory's slope scratch [K][J], and each lane writes
//     the Hermite data (y_k, y_{k+1}, s_k, s_{k+1}) of the segments beside its rows.
constexpr int kChunk = 16;  // rows of column values fetched at once per lane (loads in flight)
constexpr int kBuildStaged = 6;  // knot arrays in shared memory: ra, rb, lo, up, v, w
constexpr int kBuildSharedKnots = 180;  // largest K parked in shared memory (< 32 KB per block)
constexpr int kSepN = kBuildParts - 1;  // separators of a spline at most

template <bool kShared>
__global__ void __launch_bounds__(kBuildThreads)
k_build(const BuildJob *__restrict__ jobs, int n_jobs, unsigned *err)
{
    extern __shared__ double sk[];  // [kBuildStaged][K], then (kShared) values, slopes [K][8]
    __shared__ double s_sinv[kSepN * kSepN];
    __shared__ int s_parts[kBuildParts + 2];
    int lo = 0, hi = n_jobs - 1;
    const int blk = blockIdx.x;
    while (lo < hi) {  // job of this block: largest q with jobs[q].block_begin <= blk
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block_begin <= blk) lo = mid; else hi = mid - 1;
    }
    const BuildJob &jb = jobs[lo];
    const TrajDev &tr = jb.tr;
    const int K = tr.K, J = tr.J;
    double *ra = sk, *rb = sk + K, *fl = sk + 2 * K, *fu = sk + 3 * K, *fv = sk + 4 * K,
           *fx = sk + 5 * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        ra[k] = tr.fac_ra[k];
        rb[k] = tr.fac_rb[k];
        fl[k] = tr.fac_lo[k];
        fu[k] = tr.fac_up[k];
        fv[k] = tr.fac_v[k];
        fx[k] = tr.fac_x[k];
    }
    for (int i = threadIdx.x; i < kSepN * kSepN; i += blockDim.x) s_sinv[i] = tr.fac_sinv[i];
    if (threadIdx.x < kBuildParts + 2) s_parts[threadIdx.x] = tr.parts[threadIdx.x];
    __syncthreads();
    const int P = s_parts[0];
    const int b = threadIdx.x & (kBuildParts - 1);
    const int sl = threadIdx.x / kBuildParts;  // column slot in this block
    const int j0 = (blk - jb.block_begin) * kBuildSplines;
    const int j = j0 + sl;
    const bool live = j < J;
    const int jj = live ? j : 0;  // a column past J computes on column 0 and stores nothing
    const bool mine = b < P;      // this lane has a block
    double *yS = sk + kBuildStaged * K, *sS = yS + K * kBuildSplines;  // kShared only
    // parked values of this column: row k at park[prow(k)]
    double *park = kShared ? sS + sl : tr.slopes + jj;
    auto prow = [&](int k) -> size_t {
        return kShared ? (size_t)(k * kBuildSplines) : (size_t)k * J;
    };
    const bool pw = kShared || live;  // a column past J has no global row to park in
    unsigned bad = 0u;  // bit 31: some column value was not finite
    const int a = mine ? s_parts[1 + b] : 1;
    const int e = mine ? (b + 1 < P ? s_parts[2 + b] - 2 : K - 2) : 0;
    const int steps = e - a + 1;  // <= 0 for a lane without a block
    const bool sep = mine && b > 0;  // this lane's block has a left separator, row a - 1
    const double h_sep = sep ? tr.h[a - 1] : 0.0, h_sep1 = sep ? tr.h[a - 2] : 0.0;

    // forward substitution over the block, g_k = ra_k D_{k-1} + rb_k D_k - lo_k g_{k-1}, parked
    double yb = 0.0, yc = 0.0, ylm2 = 0.0;
    if (mine) {
        yb = load_y(jb, jj, a - 1);
        yc = load_y(jb, jj, a);
        bad |= nonfinite_bit(yb) | nonfinite_bit(yc);
        if (b > 0) ylm2 = load_y(jb, jj, a - 2);  // for the left separator's row
        if (kShared) {
            yS[(a - 1) * kBuildSplines + sl] = yb;
            yS[a * kBuildSplines + sl] = yc;
        }
    }
    const double y_sep_l = yb, y_first_col = yc;  // y_{a-1}, y_a
    // differences first: the phase arrays are large (1e5 rad) with small steps, and
    // y_{k+1} - y_k is exact where an expanded form would cancel; each difference is formed once
    // (row k's right difference is row k + 1's left one)
    const double d_left = yc - yb;  // D_{a-1}
    double dprev = d_left, dprev2 = 0.0, d_first = 0.0, g = 0.0;
    for (int i0 = 0; i0 < steps; i0 += kChunk) {
        double ya[kChunk];  // y_{k + 1} for the chunk's rows
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            ya[q] = (i0 + q < steps) ? load_y(jb, jj, a + i0 + q + 1) : 0.0;
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = i0 + q;
            if (i >= steps) break;
            const int k = a + i;
            bad |= nonfinite_bit(ya[q]);
            const double dr = ya[q] - yc;
            const double r = fma(ra[k], dprev, rb[k] * dr);
            g = i == 0 ? r : fma(-fl[k], g, r);
            if (i == 0) d_first = dr;
            if (pw) park[prow(k)] = g;
            if (kShared) yS[(k + 1) * kBuildSplines + sl] = ya[q];
            dprev2 = dprev;
            dprev = dr;
            yc = ya[q];
        }
    }
    // back substitution, y_k = g_k - up_k y_{k+1} (y_e = g_e is parked already)
    double y_next = g;
    const double y_last = y_next;
    for (int i0 = 1; i0 < steps; i0 += kChunk) {
        double pv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            pv[q] = (i0 + q < steps) ? park[prow(e - i0 - q)] : 0.0;
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            if (i0 + q >= steps) break;
            const int k = e - i0 - q;
            y_next = fma(-fu[k], y_next, pv[q]);
            if (pw) park[prow(k)] = y_next;
        }
    }
    const double y_first = y_next;  // y_a (y_e when the block has one row)

    // separator system: lane b (>= 1) forms the right-hand side of its left separator row
    const double y_last_left = __shfl_up_sync(0xffffffffu, y_last, 1, kBuildParts);
    double gs = 0.0;
    if (sep) {
        const int sg = a - 1;
        const double fs = fma(ra[sg], y_sep_l - ylm2, rb[sg] * (y_first_col - y_sep_l));
        gs = fs - h_sep * y_last_left - h_sep1 * y_first;
        bad |= nonfinite_bit(ylm2);
    }
    // lane b's right separator (number b + 1) from the inverse: X_{b+1} = sum_m Sinv[b][m-1] g_m
    // (lanes without a separator hold g = 0, and Sinv is zero past P - 1)
    const bool has_right = b + 1 < P;
    const double *srow = s_sinv + (has_right ? b : 0) * kSepN;
    double xr = 0.0;
#pragma unroll
    for (int m = 1; m < kBuildParts; ++m)
        xr = fma(srow[m - 1], __shfl_sync(0xffffffffu, gs, m, kBuildParts), xr);
    if (!has_right) xr = 0.0;
    const double xl_up = __shfl_up_sync(0xffffffffu, xr, 1, kBuildParts);
    const double xl = b == 0 ? 0.0 : xl_up;

    // correction, x_k = y_k - x_left v_k - x_right w_k; the Hermite data (y_k, y_{k+1}, s_k,
    // s_{k+1}) of every segment follow (the consumers form the power coefficients,
    // hermite_to_power)
    double *__restrict__ coef = tr.coef;
    auto put = [&](int seg, double yl, double yr, double sl_, double sr) {
        double2 *cc = reinterpret_cast<double2 *>(coef + ((size_t)seg * J + j) * 4);
        cc[0] = make_double2(yl, yr);
        cc[1] = make_double2(sl_, sr);
    };
    // the slope and value left of the block: row a - 1 (the left separator, or row 0)
    double s_prev = xl, y_prev = y_sep_l;
    for (int i0 = 0; i0 < steps; i0 += kChunk) {
        double pv[kChunk], yv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const bool act = i0 + q < steps;
            pv[q] = act ? park[prow(a + i0 + q)] : 0.0;
            yv[q] = (act && !kShared) ? load_y(jb, jj, a + i0 + q) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = i0 + q;
            if (i >= steps) break;
            const int k = a + i;
            const double x = fma(-xr, fx[k], fma(-xl, fv[k], pv[q]));
            if (i == 0 && b == 0) {  // s_0 = ra_0 D_0 + rb_0 D_1 - lo_0 s_1
                s_prev = fma(ra[0], d_left, fma(rb[0], d_first, -fl[0] * x));
                if (kShared) park[0] = s_prev;
            }
            if (kShared) {
                park[prow(k)] = x;
            } else if (live) {
                put(k - 1, y_prev, yv[q], s_prev, x);
            }
            s_prev = x;
            y_prev = yv[q];
        }
    }
    if (mine) {
        // s_{K-1} = ra_{K-1} D_{K-3} + rb_{K-1} D_{K-2} - lo_{K-1} s_{K-2} (the last block)
        const double s_last = fma(ra[K - 1], dprev2, fma(rb[K - 1], dprev, -fl[K - 1] * s_prev));
        if (kShared) {
            if (b > 0) park[prow(a - 1)] = xl;  // the left separator's slope
            if (!has_right) park[prow(K - 1)] = s_last;
        } else if (live) {
            if (has_right) {  // segment e between row e and the right separator
                put(e, y_prev, load_y(jb, jj, e + 1), s_prev, xr);
            } else {
                put(K - 2, y_prev, load_y(jb, jj, K - 1), s_prev, s_last);
            }
        }
    }
    if (kShared) {  // the block's 8 columns, segment by segment: 16-byte stores, 256 B per segment
        __syncthreads();
        constexpr int kPerSeg = 2 * kBuildSplines;
        for (int idx = threadIdx.x; idx < (K - 1) * kPerSeg; idx += blockDim.x) {
            const int seg = idx / kPerSeg, rr = idx - seg * kPerSeg, c = rr >> 1, half = rr & 1;
            if (j0 + c >= J) continue;
            const double *src = half ? sS : yS;
            *reinterpret_cast<double2 *>(coef + ((size_t)seg * J + j0 + c) * 4 + 2 * half) =
                make_double2(src[seg * kBuildSplines + c], src[(seg + 1) * kBuildSplines + c]);
        }
    }
    if ((bad & 0x80000000u) && live) atomicOr(err, ERRBIT_NONFINITE);
}

cudaError_t launch_build(const BuildJob *jobs_dev, int n_jobs, int total_blocks, int max_knots,
                         unsigned *err, cudaStream_t st)
{
    const bool shared = max_knots <= kBuildSharedKnots;
    const int per_knot = kBuildStaged + (shared ? 2 * kBuildSplines : 0);
    const int smem_bytes = per_knot * max_knots * (int)sizeof(double);
    auto kern = shared ? k_build<true> : k_build<false>;
    if (smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_bytes);
        if (e != cudaSuccess) return e;
    }
    if (total_blocks <= 0) return cudaSuccess;
    kern<<<total_blocks, kBuildThreads, smem_bytes, st>>>(jobs_dev, n_jobs, err);
    return cudaGetLastError();
}

}  // namespace fewsum
