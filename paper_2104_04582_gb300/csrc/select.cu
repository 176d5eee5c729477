// select.cu -- Mode Selector on the device (arXiv:2104.04582 Sec. 3.D).
//
// At every knot of the trajectory, the power of each mode is |A(t_k)|^2, doubled for m > 0 (the
// mode also stands for its m < 0 partner of equal power).  The powers are sorted in descending
// order (ties: lower mode index first) and summed cumulatively; the knot keeps the shortest
// leading run whose cumulative power reaches (1 - eps) of the knot's total.  The selection is the
// union of the kept sets over all knots.
//
// One CTA per knot, P = max(128, next power of two >= N) sort slots, P/4 threads holding four
// consecutive slots each in registers.  Bitonic sort of (power, index) pairs: the exchanges at
// distances 1 and 2 stay inside a thread, distances 4..64 are warp shuffles (a warp holds 128
// consecutive slots), and only distances >= 128 pass through shared memory.  The sorted powers
// are then scanned in FP64 straight from the registers (thread, warp, block), the first rank whose
// prefix reaches the target is found with an atomic minimum, and the kept modes are marked with
// plain byte stores of 1 into a mask zeroed beforehand (every writer stores the same value, so
// the union needs no atomics).
#include "fewsum_internal.h"

namespace fewsum {

constexpr int kSelectMaxThreads = 1024;
constexpr int kSelectPerThread = 4;  // consecutive sort slots per thread
constexpr int kSelectWarpSlots = 32 * kSelectPerThread;

// Non-negative doubles order exactly like their IEEE bit patterns read as unsigned integers, so
// the sort compares 64-bit integer keys (descending power = ascending inverted bits), with the
// mode index as the tie-break; integer compares avoid GB300's narrow FP64 pipe.
__device__ __forceinline__ unsigned long long power_key(double p)
{
    return ~static_cast<unsigned long long>(__double_as_longlong(p));
}

__device__ __forceinline__ double key_power(unsigned long long key)
{
    return __longlong_as_double(static_cast<long long>(~key));
}

__device__ __forceinline__ bool sorts_before(unsigned long long ka, int ia, unsigned long long kb,
                                             int ib)
{
    return ka < kb || (ka == kb && ia < ib);
}

// Compare-exchange of two slots held by one thread: a precedes b in the final order when up.
__device__ __forceinline__ void cx_pair(unsigned long long &ka, int &ia, unsigned long long &kb,
                                        int &ib, bool up)
{
    const bool swap = up ? sorts_before(kb, ib, ka, ia) : sorts_before(ka, ia, kb, ib);
    if (swap) {
        const unsigned long long tk = ka; ka = kb; kb = tk;
        const int ti = ia; ia = ib; ib = ti;
    }
}

// One side of a compare-exchange whose partner slot is held by another thread: keep the element
// that comes first (keep_first) or second of the two.  Both sides take the same comparison, so
// exactly one of them ends up with each element.
__device__ __forceinline__ void cx_keep(unsigned long long &k, int &i, unsigned long long ko, int io,
                                        bool keep_first)
{
    if (sorts_before(ko, io, k, i) == keep_first) { k = ko; i = io; }
}

__global__ void __launch_bounds__(kSelectMaxThreads)
k_mode_select(const double *__restrict__ amp_re, const double *__restrict__ amp_im, int N,
              const __grid_constant__ ModeDoubling dbl, double eps, int P,
              unsigned char *__restrict__ mask)
{
    extern __shared__ __align__(16) unsigned long long sel_key[];  // [P] keys, then [P] indices
    int *sel_ix = reinterpret_cast<int *>(sel_key + P);
    __shared__ double warp_tot[kSelectMaxThreads / 32];
    __shared__ double s_total;
    __shared__ int s_cut;
    const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int p0 = kSelectPerThread * tid;  // first slot of this thread

    unsigned long long key[kSelectPerThread];
    int ix[kSelectPerThread];
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r) {
        const int i = p0 + r;
        if (i < N) {
            const double re = amp_re[(size_t)k * N + i], im = amp_im[(size_t)k * N + i];
            double p = re * re + im * im;
            if ((dbl.w[i >> 5] >> (i & 31)) & 1u) p *= 2.0;  // m > 0
            key[r] = power_key(p);
            ix[r] = i;
        } else {
            key[r] = ~0ull;  // padding: power +0, sorts after every real mode
            ix[r] = 0x7fffffff;
        }
    }
    if (tid == 0) s_cut = 0x7fffffff;

    // bitonic sort into ascending "sorts_before" order; slot p runs up when (p & size) == 0
    for (int size = 2; size <= P; size <<= 1) {
        int stride = size >> 1;
        if (stride >= kSelectWarpSlots) {
            ulonglong2 *kv = reinterpret_cast<ulonglong2 *>(sel_key + p0);
            kv[0] = make_ulonglong2(key[0], key[1]);
            kv[1] = make_ulonglong2(key[2], key[3]);
            *reinterpret_cast<int4 *>(sel_ix + p0) = make_int4(ix[0], ix[1], ix[2], ix[3]);
            __syncthreads();
            for (; stride >= kSelectWarpSlots; stride >>= 1) {
                for (int q = tid; q < P / 2; q += nt) {
                    const int lo = ((q & ~(stride - 1)) << 1) | (q & (stride - 1)), hi = lo + stride;
                    unsigned long long ka = sel_key[lo], kb = sel_key[hi];
                    int ia = sel_ix[lo], ib = sel_ix[hi];
                    const bool up = (lo & size) == 0;
                    const bool swap = up ? sorts_before(kb, ib, ka, ia) : sorts_before(ka, ia, kb, ib);
                    if (swap) {
                        sel_key[lo] = kb; sel_key[hi] = ka;
                        sel_ix[lo] = ib; sel_ix[hi] = ia;
                    }
                }
                __syncthreads();
            }
            const ulonglong2 a = kv[0], b = kv[1];
            key[0] = a.x; key[1] = a.y; key[2] = b.x; key[3] = b.y;
            const int4 v = *reinterpret_cast<const int4 *>(sel_ix + p0);
            ix[0] = v.x; ix[1] = v.y; ix[2] = v.z; ix[3] = v.w;
        }
        for (; stride >= kSelectPerThread; stride >>= 1) {
            const int lane_mask = stride / kSelectPerThread;
            const bool is_lo = (p0 & stride) == 0, up = (p0 & size) == 0;
#pragma unroll
            for (int r = 0; r < kSelectPerThread; ++r) {
                const unsigned long long ko = __shfl_xor_sync(0xffffffffu, key[r], lane_mask);
                const int io = __shfl_xor_sync(0xffffffffu, ix[r], lane_mask);
                cx_keep(key[r], ix[r], ko, io, up == is_lo);
            }
        }
        if (stride == 2) {
            const bool up = (p0 & size) == 0;  // size >= 4: the same for all four slots
            cx_pair(key[0], ix[0], key[2], ix[2], up);
            cx_pair(key[1], ix[1], key[3], ix[3], up);
            stride = 1;
        }
        // stride 1: slots (0,1) and (2,3); for size 2 the direction alternates inside the thread
        cx_pair(key[0], ix[0], key[1], ix[1], ((p0 + 0) & size) == 0);
        cx_pair(key[2], ix[2], key[3], ix[3], ((p0 + 2) & size) == 0);
    }

    // inclusive prefix sums of the sorted powers (padding adds +0): thread, warp, block
    double pre[kSelectPerThread];
    double run = 0.0;
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r) {
        run += key_power(key[r]);
        pre[r] = run;
    }
    double incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        double w = lane < nt / 32 ? warp_tot[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        double we = __shfl_up_sync(0xffffffffu, w, 1);
        if (lane == 0) we = 0.0;
        if (lane < nt / 32) warp_tot[lane] = we;  // exclusive over warps
    }
    __syncthreads();
    const double offset = excl + warp_tot[wid];
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r) {
        pre[r] += offset;
        if (p0 + r == N - 1) s_total = pre[r];  // the knot's total is the last real prefix
    }
    __syncthreads();
    const double total = s_total;
    if (!(total > 0.0)) return;  // uniform: nothing kept at a knot without power
    const double target = (1.0 - eps) * total;  // <= total, so some rank below N reaches it
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r) {
        if (p0 + r < N && pre[r] >= target) {
            atomicMin(&s_cut, p0 + r);
            break;
        }
    }
    __syncthreads();
    const int cut = s_cut;
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r)
        if (p0 + r <= cut) mask[ix[r]] = 1;
}

cudaError_t launch_mode_select(const double *amp_re, const double *amp_im, int K, int N,
                               const ModeDoubling &dbl, double eps, unsigned char *mask,
                               cudaStream_t st)
{
    int P = kSelectWarpSlots;
    while (P < N) P <<= 1;
    const int threads = P / kSelectPerThread;
    const int smem = P * (int)(sizeof(unsigned long long) + sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(k_mode_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(mask, 0, (size_t)N, st);
    if (e != cudaSuccess) return e;
    k_mode_select<<<K, threads, smem, st>>>(amp_re, amp_im, N, dbl, eps, P, mask);
    return cudaGetLastError();
}

int mode_select_max_modes() { return kSelectMaxModes; }

}  // namespace fewsum
