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
// The matrix depends only on the knots, so it is factorised once per trajectory (k_factor,
// Thomas elimination without pivoting) and every spline reuses that factorisation: one thread
// per spline does the forward sweep and back substitution on its own right-hand side.
// Coefficients are stored in the normalised local variable u = (t - t_k)/h_k in [0, 1]:
//     p(u) = y_k + h_k s_k u + (3 D - h_k (2 s_k + s_{k+1})) u^2 + (h_k (s_k + s_{k+1}) - 2 D) u^3,
// D = y_{k+1} - y_k.  The two phase arrays are fitted in radians as given (their reduction
// modulo 2 pi happens per segment and per sample in the summation kernel).
#include "fewsum_internal.h"

namespace fewsum {

// Shared factorisation of the not-a-knot matrix of one knot grid (single thread; O(K)).
__global__ void k_factor(const double *__restrict__ t, int K, double *h, double *inv_h,
                         double *fac_w, double *fac_ip, double *fac_up)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int S = K - 1;
    for (int k = 0; k < S; ++k) {
        h[k] = t[k + 1] - t[k];
        inv_h[k] = 1.0 / h[k];
    }
    // row k: lo_k * s_{k-1} + dg_k * s_k + up_k * s_{k+1}
    double piv = 0.0;
    for (int k = 0; k < K; ++k) {
        double lo, dg, up;
        if (k == 0) {
            lo = 0.0; dg = h[1]; up = h[0] + h[1];
        } else if (k == K - 1) {
            lo = h[K - 2] + h[K - 3]; dg = h[K - 3]; up = 0.0;
        } else {
            lo = h[k]; dg = 2.0 * (h[k - 1] + h[k]); up = h[k - 1];
        }
        double w = (k == 0) ? 0.0 : lo / piv;
        double prev_up = (k == 0) ? 0.0 : fac_up[k - 1];
        piv = dg - w * prev_up;
        fac_w[k] = w;
        fac_ip[k] = 1.0 / piv;
        fac_up[k] = up;
    }
}

cudaError_t launch_factor(const double *t, int K, double *h, double *inv_h, double *fac_w,
                          double *fac_ip, double *fac_up, cudaStream_t st)
{
    k_factor<<<1, 32, 0, st>>>(t, K, h, inv_h, fac_w, fac_ip, fac_up);
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

// One thread per spline column.  Jobs are laid out in a flattened grid of column blocks.
// The sweeps are sequential in k, so each step would wait on its own global load; instead the
// knot-only arrays (h, 1/h, factorisation) are staged in shared memory and the column values
// are fetched kChunk knots ahead into registers, so kChunk loads are in flight at once.
constexpr int kChunk = 8;

__global__ void __launch_bounds__(kBuildThreads)
k_build(const BuildJob *__restrict__ jobs, int n_jobs, unsigned *err)
{
    extern __shared__ double sk[];  // [5][K]: h, 1/h, w, 1/pivot, up
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
    double *h = sk, *ih = sk + K, *fw = sk + 2 * K, *fip = sk + 3 * K, *fup = sk + 4 * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        h[k] = k < K - 1 ? tr.h[k] : 0.0;
        ih[k] = k < K - 1 ? tr.inv_h[k] : 0.0;
        fw[k] = tr.fac_w[k];
        fip[k] = tr.fac_ip[k];
        fup[k] = tr.fac_up[k];
    }
    __syncthreads();
    const int j = (b - jb.block_begin) * kBuildThreads + threadIdx.x;
    if (j >= J) return;
    double *__restrict__ coef = tr.coef;
    bool finite = true;

    // forward sweep: r'_k = r_k - w_k r'_{k-1}; r'_k is parked in coef[k][j][1] (k < K-1)
    double y0 = load_y(jb, j, 0), y1 = load_y(jb, j, 1), y2 = load_y(jb, j, 2);
    finite &= isfinite(y0) && isfinite(y1) && isfinite(y2);
    const double d0 = (y1 - y0) * ih[0], d1 = (y2 - y1) * ih[1];
    double rp = ((2.0 * h[1] + 3.0 * h[0]) * h[1] * d0 + h[0] * h[0] * d1) / (h[0] + h[1]);
    coef[(size_t)j * 4 + 1] = rp;
    double dprev = d0;  // d_{k-1}
    double ycur = y1;   // y_k
    double dkm3 = d0;   // d_{K-3}, kept for the last row
    for (int k0 = 1; k0 <= K - 2; k0 += kChunk) {
        double yn[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q)
            yn[q] = (k0 + q <= K - 2) ? load_y(jb, j, k0 + q + 1) : 0.0;
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int k = k0 + q;
            if (k > K - 2) break;
            finite &= isfinite(yn[q]);
            const double dk = (yn[q] - ycur) * ih[k];
            const double r = 3.0 * (h[k] * dprev + h[k - 1] * dk);
            rp = r - fw[k] * rp;
            coef[((size_t)k * J + j) * 4 + 1] = rp;
            if (k == K - 3) dkm3 = dk;
            dprev = dk;
            ycur = yn[q];
        }
    }
    {
        const double a = h[K - 2], c = h[K - 3];
        const double r = (a * a * dkm3 + (2.0 * c + 3.0 * a) * c * dprev) / (c + a);
        rp = r - fw[K - 1] * rp;
    }
    // back substitution and coefficients in u, with r'_k and y_k fetched a chunk ahead
    double s_next = rp * fip[K - 1];  // s_{K-1}
    double y_next = ycur;             // y_{K-1}
    for (int k0 = K - 2; k0 >= 0; k0 -= kChunk) {
        double rv[kChunk], yv[kChunk];
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int k = k0 - q;
            rv[q] = k >= 0 ? coef[((size_t)k * J + j) * 4 + 1] : 0.0;
            yv[q] = k >= 0 ? load_y(jb, j, k) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < kChunk; ++q) {
            const int k = k0 - q;
            if (k < 0) break;
            double *c = coef + ((size_t)k * J + j) * 4;
            const double s = (rv[q] - fup[k] * s_next) * fip[k];
            const double yk = yv[q];
            const double D = y_next - yk;
            const double hk = h[k];
            const double2 c01 = make_double2(yk, hk * s);
            const double2 c23 = make_double2(3.0 * D - hk * (2.0 * s + s_next),
                                             hk * (s + s_next) - 2.0 * D);
            reinterpret_cast<double2 *>(c)[0] = c01;
            reinterpret_cast<double2 *>(c)[1] = c23;
            s_next = s;
            y_next = yk;
        }
    }
    if (!finite) atomicOr(err, ERRBIT_NONFINITE);
}

cudaError_t launch_build(const BuildJob *jobs_dev, int n_jobs, int total_blocks, int max_knots,
                         unsigned *err, cudaStream_t st)
{
    const int smem_bytes = 5 * max_knots * (int)sizeof(double);
    if (smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem_bytes);
        if (e != cudaSuccess) return e;
    }
    if (total_blocks <= 0) return cudaSuccess;
    k_build<<<total_blocks, kBuildThreads, smem_bytes, st>>>(jobs_dev, n_jobs, err);
    return cudaGetLastError();
}

}  // namespace fewsum
