// select.cu -- Mode Selector on the device (arXiv:2104.04582 Sec. 3.D).
//
// At every knot of the trajectory, the power of each mode is |A(t_k)|^2, doubled for m > 0 (the
// mode also stands for its m < 0 partner of equal power).  The powers are sorted in descending
// order (ties: lower mode index first) and summed cumulatively; the knot keeps the shortest
// leading run whose cumulative power reaches (1 - eps) of the knot's total.  The selection is the
// union of the kept sets over all knots.
//
// One CTA per knot: bitonic sort of (power, index) pairs in shared memory, an FP64 inclusive
// scan of the sorted powers, and a search for the first rank whose prefix reaches the target.
// Kept modes are marked with plain byte stores of 1 into a mask zeroed beforehand (every
// writer stores the same value, so the union needs no atomics).
#include "fewsum_internal.h"

namespace fewsum {

constexpr int kSelectThreads = 1024;
constexpr int kSelectMaxModes = 4096;

// Non-negative doubles order exactly like their IEEE bit patterns read as unsigned integers, so
// the sort compares 64-bit integer keys (descending power = ascending inverted bits), with the
// mode index as the tie-break; integer compares avoid GB300's narrow FP64 pipe.
__device__ __forceinline__ unsigned long long power_key(double p)
{
    return ~static_cast<unsigned long long>(__double_as_longlong(p));
}

__device__ __forceinline__ bool sorts_before(unsigned long long ka, int ia, unsigned long long kb,
                                             int ib)
{
    return ka < kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(kSelectThreads)
k_mode_select(const double *__restrict__ amp_re, const double *__restrict__ amp_im, int N,
              const int *__restrict__ m, double eps, int P, unsigned char *__restrict__ mask)
{
    extern __shared__ double sel_smem[];
    double *pw = sel_smem;                                  // [P] sort keys, then prefix sums
    unsigned long long *key = reinterpret_cast<unsigned long long *>(sel_smem);
    int *ix = reinterpret_cast<int *>(sel_smem + P);        // [P] mode indices
    __shared__ double warp_tot[kSelectThreads / 32];
    __shared__ int s_cut;
    const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < P; i += nt) {
        if (i < N) {
            const double re = amp_re[(size_t)k * N + i], im = amp_im[(size_t)k * N + i];
            double p = re * re + im * im;
            if (m[i] > 0) p *= 2.0;
            key[i] = power_key(p);
            ix[i] = i;
        } else {
            key[i] = ~0ull;  // padding sorts after every real mode
            ix[i] = 0x7fffffff;
        }
    }
    if (tid == 0) s_cut = -1;
    __syncthreads();
    // bitonic sort into ascending "sorts_before" order
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P; i += nt) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long ki = key[i], kj = key[j];
                    const int ii = ix[i], ij = ix[j];
                    const bool swap = up ? sorts_before(kj, ij, ki, ii) : sorts_before(ki, ii, kj, ij);
                    if (swap) {
                        key[i] = kj; key[j] = ki;
                        ix[i] = ij; ix[j] = ii;
                    }
                }
            }
            __syncthreads();
        }
    }
    // inclusive scan of the first N sorted powers: per-thread chunks, then warp and block scans
    const int chunk = (N + nt - 1) / nt;
    const int b0 = tid * chunk, b1 = min(N, b0 + chunk);
    double run = 0.0;
    for (int i = b0; i < b1; ++i) {
        run += __longlong_as_double(static_cast<long long>(~key[i]));
        pw[i] = run;
    }
    double incl = run;
    const int lane = tid & 31, wid = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        double w = lane < nt / 32 ? warp_tot[lane] : 0.0;
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        if (lane < nt / 32) warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const double offset = (incl - run) + (wid > 0 ? warp_tot[wid - 1] : 0.0);
    for (int i = b0; i < b1; ++i) pw[i] += offset;
    __syncthreads();
    const double total = pw[N - 1];
    if (!(total > 0.0)) return;  // uniform: nothing kept at a knot without power
    const double target = (1.0 - eps) * total;
    for (int i = tid; i < N; i += nt)
        if (pw[i] >= target && (i == 0 || pw[i - 1] < target)) s_cut = i;
    __syncthreads();
    const int cut = s_cut < 0 ? N - 1 : s_cut;
    for (int i = tid; i <= cut; i += nt) mask[ix[i]] = 1;
}

cudaError_t launch_mode_select(const double *amp_re, const double *amp_im, int K, int N,
                               const int *m_dev, double eps, unsigned char *mask, cudaStream_t st)
{
    int P = 2;
    while (P < N) P <<= 1;
    const int smem = P * (int)(sizeof(double) + sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(k_mode_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(mask, 0, (size_t)N, st);
    if (e != cudaSuccess) return e;
    k_mode_select<<<K, kSelectThreads, smem, st>>>(amp_re, amp_im, N, m_dev, eps, P, mask);
    return cudaGetLastError();
}

int mode_select_max_modes() { return kSelectMaxModes; }

}  // namespace fewsum
