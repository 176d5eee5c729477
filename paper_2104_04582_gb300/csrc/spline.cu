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
// the knots, so it is factorised once per trajectory (k_factor) in twisted form: top-down
// elimination of rows 1..m and bottom-up elimination of rows K-2..m, m = (K-1)/2, both stable
// by diagonal dominance.  Every spline reuses that factorisation with two threads (k_build): the
// top one sweeps rows 1..m, the bottom one rows K-2..m, they combine at row m
//     s_m = (y_m + z_m - rhs_m) / (p_m + q_m - d_m),
// and substitute away from m in opposite directions, each writing the slopes on its side;
// s_0 and s_{K-1} follow from the end rows.  The sweeps are serial chains of FP64 operations,
// so they carry nothing else; a second kernel (k_coef), one thread per (segment, spline), then
// forms the coefficients in the normalised local variable u = (t - t_k)/h_k in [0, 1]:
//     p(u) = y_k + h_k s_k u + (3 D - h_k (2 s_k + s_{k+1})) u^2 + (h_k (s_k + s_{k+1}) - 2 D) u^3,
// D = y_{k+1} - y_k.  The two phase arrays are fitted in radians as given (their reduction
// modulo 2 pi happens per segment and per sample in the summation kernel).
#include "fewsum_internal.h"

namespace fewsum {

// Shared twisted factorisation of the reduced not-a-knot matrix of one knot grid (single
// thread; O(K)).  fac_w[k] = w_k (top rows 2..m), fac_v[k] = v_k (bottom rows m..K-3),
// fac_ip[k] = 1/p_k (k < m), 1/q_k (k > m), 1/(p_m + q_m - d_m) (k = m).
__global__ void k_factor(const double *__restrict__ t, int K, double *h, double *inv_h,
                         double *fac_w, double *fac_ip, double *fac_v)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int S = K - 1, m = (K - 1) / 2;
    for (int k = 0; k < S; ++k) {
        h[k] = t[k + 1] - t[k];
        inv_h[k] = 1.0 / h[k];
    }
    for (int k = 0; k < K; ++k) fac_w[k] = fac_ip[k] = fac_v[k] = 0.0;
    // reduced rows 1..K-2: lo_k = h_k (k >= 2), up_k = h_{k-1} (k <= K-3), diagonal dg(k)
    auto dg = [&](int k) {
        if (k == 1) return h[0] + h[1];
        if (k == K - 2) return h[K - 3] + h[K - 2];
        return 2.0 * (h[k - 1] + h[k]);
    };
    double p = dg(1);
    fac_ip[1] = 1.0 / p;
    for (int k = 2; k <= m; ++k) {
        const double w = h[k] / p;
        p = dg(k) - w * h[k - 2];
        fac_w[k] = w;
        fac_ip[k] = 1.0 / p;
    }
    double q = dg(K - 2);
    if (K - 2 > m) fac_ip[K - 2] = 1.0 / q;
    for (int k = K - 3; k >= m; --k) {
        const double v = h[k - 1] / q;
        q = dg(k) - v * h[k + 1];
        fac_v[k] = v;
        if (k > m) fac_ip[k] = 1.0 / q;
    }
    fac_ip[m] = 1.0 / (p + q - dg(m));
}

cudaError_t launch_factor(const double *t, int K, double *h, double *inv_h, double *fac_w,
                          double *fac_ip, double *fac_v, cudaStream_t st)
{
    k_factor<<<1, 32, 0, st>>>(t, K, h, inv_h, fac_w, fac_ip, fac_v);
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

// Two threads per spline column: lane l (< 16) of a warp runs the top sweep and lane l + 16 the
// bottom sweep of the same column, in one instruction stream (direction and coefficients are
// per-lane data), so the pair meets at row m without divergence and exchanges its reduced
// right-hand side with one shuffle.  The knot-only arrays are staged in shared memory and the
// column values (and, in the substitution, the parked values) are fetched kChunk rows ahead
// into registers, so kChunk loads are in flight: the grid has only a few warps per SM, so
// memory latency is hidden by depth, not by occupancy.
constexpr int kChunk = 8;

__global__ void __launch_bounds__(kBuildThreads)
k_build(const BuildJob *__restrict__ jobs, int n_jobs, unsigned *err)
{
    extern __shared__ double sk[];  // [6][K]: h, ra, rb, top multipliers, inverse pivots, bottom multipliers
    // job of this block: largest q with jobs[q].block_begin <= blockIdx.x
    int lo = 0, hi = n_jobs - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block_begin <= b) lo = mid; else hi = mid - 1;
    }
    const BuildJob &jb = jobs[lo];
    const TrajDev &tr = jb.tr;
    const int K = tr.K, J = tr.J;
    // ra_k = 3 h_k / h_{k-1}, rb_k = 3 h_{k-1} / h_k: the interior right-hand side
    // 3 (h_k d_{k-1} + h_{k-1} d_k) becomes ra_k (y_k - y_{k-1}) + rb_k (y_{k+1} - y_k)
    double *h = sk, *ra = sk + K, *rb = sk + 2 * K, *fw = sk + 3 * K, *fip = sk + 4 * K, *fv = sk + 5 * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        h[k] = k < K - 1 ? tr.h[k] : 0.0;
        const bool in = k >= 1 && k <= K - 2;
        ra[k] = in ? 3.0 * tr.h[k] * tr.inv_h[k - 1] : 0.0;
        rb[k] = in ? 3.0 * tr.h[k - 1] * tr.inv_h[k] : 0.0;
        fw[k] = tr.fac_w[k];
        fip[k] = tr.fac_ip[k];
        fv[k] = tr.fac_v[k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const bool top = lane < 16;
    const int j = (b - jb.block_begin) * kBuildSplines + (threadIdx.x >> 5) * 16 + (lane & 15);
    const bool live = j < J;
    const int jj = live ? j : 0;  // a column past J computes on column 0 and stores nothing
    double *__restrict__ slopes = tr.slopes;
    unsigned bad = 0u;  // bit 31: some column value was not finite
    const int m = (K - 1) / 2;
    const int dir = top ? 1 : -1, k0 = top ? 1 : K - 2;
    const int steps = top ? m : K - 1 - m, steps_max = K - 1 - m;

    // elimination: acc = rhs_k - mult_k acc along rows k0, k0 + dir, ..., m; the window holds
    // y_{k - dir} (yb) and y_k (yc)
    double yb = load_y(jb, jj, k0 - dir), yc = load_y(jb, jj, k0);
    bad |= nonfinite_bit(yb) | nonfinite_bit(yc);
    double acc = 0.0, rend = 0.0, rm = 0.0;
    for (int i0 = 0; i0 < steps_max; i0 += kChunk) {
        double ya[kChunk];  // y_{k + dir} for the chunk's rows
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            ya[q] = (i0 + q < steps) ? load_y(jb, jj, k0 + dir * (i0 + q + 1)) : 0.0;
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = i0 + q;
            if (i >= steps) break;
            const int k = k0 + dir * i;
            bad |= nonfinite_bit(ya[q]);
            const double ylo = top ? yb : ya[q], yhi = top ? ya[q] : yb;  // y_{k-1}, y_{k+1}
            const double el = yc - ylo, er = yhi - yc;
            double r = fma(ra[k], el, rb[k] * er);
            if (k == 1 || k == K - 2) {
                const double dl = el / h[k - 1], dr = er / h[k];
                if (k == 1) {
                    const double R0 = ((2.0 * h[1] + 3.0 * h[0]) * h[1] * dl + h[0] * h[0] * dr) / (h[0] + h[1]);
                    r -= R0;
                    if (top) rend = R0;
                }
                if (k == K - 2) {
                    const double a = h[K - 2], c = h[K - 3];
                    const double RL = (a * a * dl + (2.0 * c + 3.0 * a) * c * dr) / (c + a);
                    r -= RL;
                    if (!top) rend = RL;
                }
            }
            if (k == m) rm = r;
            acc = r - (i == 0 ? 0.0 : (top ? fw[k] : fv[k])) * acc;
            if (k != m && live) slopes[(size_t)k * J + j] = acc;  // parked for the substitution
            yb = yc;
            yc = ya[q];
        }
    }
    // row m: both threads hold rhs_m and their own reduced value
    const double other = __shfl_xor_sync(0xffffffffu, acc, 16);
    double s_prev = (acc + other - rm) * fip[m];
    if (top && live) slopes[(size_t)m * J + j] = s_prev;

    // substitution away from m: rows m - 1, ..., 0 (top) or m + 1, ..., K - 1 (bottom); each
    // slope replaces the value parked in its place
    const int ds = -dir;
    for (int i0 = 0; i0 < steps_max; i0 += kChunk) {
        double pv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = i0 + q, k = m + ds * (1 + i);
            const bool act = i < steps;
            pv[q] = (act && k >= 1 && k <= K - 2) ? slopes[(size_t)k * J + jj] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int i = i0 + q;
            if (i >= steps) break;
            const int k = m + ds * (1 + i);
            double par, c, ipv;
            if (k == 0) {  // end row 0: h_1 s_0 + (h_0 + h_1) s_1 = R_0
                par = rend; c = h[0] + h[1]; ipv = 1.0 / h[1];
            } else if (k == K - 1) {  // end row K-1: (h_{K-2} + h_{K-3}) s_{K-2} + h_{K-3} s_{K-1} = R_L
                par = rend; c = h[K - 2] + h[K - 3]; ipv = 1.0 / h[K - 3];
            } else {  // s_k = (y_k - up_k s_{k+1}) / p_k  or  (z_k - lo_k s_{k-1}) / q_k
                par = pv[q]; c = top ? h[k - 1] : h[k]; ipv = fip[k];
            }
            const double s = (par - c * s_prev) * ipv;
            if (live) slopes[(size_t)k * J + j] = s;
            s_prev = s;
        }
    }
    if ((bad & 0x80000000u) && live) atomicOr(err, ERRBIT_NONFINITE);
}

// Cubic coefficients of every (segment, spline) once the knot slopes are known, one thread each
// (consecutive threads: consecutive splines of one segment, so the 32-byte rows are written
// contiguously): in the local variable u = (t - t_k)/h_k,
//     p(u) = y_k + h s_k u + (3 D - 2 h s_k - h s_{k+1}) u^2 + (h s_k + h s_{k+1} - 2 D) u^3,
// D = y_{k+1} - y_k, h = h_k.
__global__ void __launch_bounds__(kCoefThreads)
k_coef(const BuildJob *__restrict__ jobs, int n_jobs)
{
    int lo = 0, hi = n_jobs - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].coef_block_begin <= b) lo = mid; else hi = mid - 1;
    }
    const BuildJob &jb = jobs[lo];
    const TrajDev &tr = jb.tr;
    const int J = tr.J;
    const long long g = (long long)(b - jb.coef_block_begin) * kCoefThreads + threadIdx.x;
    if (g >= (long long)tr.S * J) return;
    const int seg = (int)(g / J), j = (int)(g - (long long)seg * J);
    const double yl = load_y(jb, j, seg), yr = load_y(jb, j, seg + 1);
    const double sl = tr.slopes[(size_t)seg * J + j], sr = tr.slopes[(size_t)(seg + 1) * J + j];
    const double hk = tr.h[seg];
    const double D = yr - yl, a = hk * sl, c = hk * sr;
    double2 *cc = reinterpret_cast<double2 *>(tr.coef + ((size_t)seg * J + j) * 4);
    cc[0] = make_double2(yl, a);
    cc[1] = make_double2(fma(-2.0, a, fma(3.0, D, -c)), fma(-2.0, D, a + c));
}

cudaError_t launch_build(const BuildJob *jobs_dev, int n_jobs, int total_blocks,
                         int total_coef_blocks, int max_knots, unsigned *err, cudaStream_t st)
{
    const int smem_bytes = 6 * max_knots * (int)sizeof(double);
    if (smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_bytes);
        if (e != cudaSuccess) return e;
    }
    if (total_blocks <= 0) return cudaSuccess;
    k_build<<<total_blocks, kBuildThreads, smem_bytes, st>>>(jobs_dev, n_jobs, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_coef<<<total_coef_blocks, kCoefThreads, 0, st>>>(jobs_dev, n_jobs);
    return cudaGetLastError();
}

}  // namespace fewsum
