// select.cu -- Mode Selector on the device (arXiv:2104.04582 Sec. 3.D).
//
// At every knot of the trajectory, the power of each mode is |A(t_k)|^2, doubled for m > 0 (the
// mode also stands for its m < 0 partner of equal power).  The powers are sorted in descending
// order (ties: lower mode index first) and summed cumulatively; the knot keeps the shortest
// leading run whose cumulative power reaches (1 - eps) of the knot's total.  The selection is the
// union of the kept sets over all knots.
//
// The selection is index output, so it is decided exactly as the plain definition computes it:
// the power is fl(fl(re^2) + fl(im^2)) (no fused multiply-add), and the cumulative sums are the
// left-to-right FP64 sums over the sorted powers, c_j = fl(c_{j-1} + p_j), with the total equal
// to the last of them.  Any other summation order can round differently and move the cut.
//
// One CTA per knot, P = max(128, next power of two >= N) sort slots, P/4 threads holding four
// consecutive slots each in registers.  Each warp sorts its 128 slots of (power, index) pairs by
// a bitonic network (exchanges at distances 1 and 2 inside a thread, 4..64 by warp shuffles),
// then the sorted runs are merged pairwise in shared memory by merge path (a binary search per
// thread for where its four outputs split between the two runs), log2(P / 128) levels.  The
// sorted powers then go to shared memory.  The cumulative sums are exact integer prefix sums
// inside each binade of the running sum (see the comment at the scan), so the whole block
// computes them in a few rounds of a block-wide scan instead of one thread running N dependent
// FP64 additions.  The first rank whose sum reaches the target is found by all threads with an
// atomic minimum, and the kept modes are marked with plain byte stores of 1 into a mask zeroed
// beforehand (every writer stores the same value, so the union needs no atomics).
#include "fewsum_internal.h"

namespace fewsum {

constexpr int kSelectMaxThreads = 1024;
constexpr int kSelectPerThread = 4;  // consecutive sort slots per thread
constexpr int kSelectWarpSlots = 32 * kSelectPerThread;
constexpr int kSelectMaxRounds = 64;  // scan rounds before the sequential chain takes over

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
    __shared__ double s_total;
    __shared__ unsigned long long s_cbits;  // bits of the running sum where a round starts
    __shared__ unsigned long long s_wsum[kSelectMaxThreads / 32];
    __shared__ int s_a, s_exit, s_fallback, s_cut;
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
            double p = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
            if ((dbl.w[i >> 5] >> (i & 31)) & 1u) p *= 2.0;  // m > 0
            key[r] = power_key(p);
            ix[r] = i;
        } else {
            key[r] = ~0ull;  // padding: power +0, sorts after every real mode
            ix[r] = 0x7fffffff;
        }
    }
    if (tid == 0) s_cut = 0x7fffffff;

    // 1. each warp sorts its 128 slots (4 per lane) into ascending "sorts_before" order by a
    //    bitonic network in registers and shuffles; below the last stage slot p runs up when
    //    (p & size) == 0, the last stage runs up in every warp
    for (int size = 2; size <= kSelectWarpSlots; size <<= 1) {
        const bool last = size == kSelectWarpSlots;
        int stride = size >> 1;
        for (; stride >= kSelectPerThread; stride >>= 1) {
            const int lane_mask = stride / kSelectPerThread;
            const bool is_lo = (p0 & stride) == 0, up = last || (p0 & size) == 0;
#pragma unroll
            for (int r = 0; r < kSelectPerThread; ++r) {
                const unsigned long long ko = __shfl_xor_sync(0xffffffffu, key[r], lane_mask);
                const int io = __shfl_xor_sync(0xffffffffu, ix[r], lane_mask);
                cx_keep(key[r], ix[r], ko, io, up == is_lo);
            }
        }
        if (stride == 2) {
            const bool up = last || (p0 & size) == 0;  // size >= 4: the same for all four slots
            cx_pair(key[0], ix[0], key[2], ix[2], up);
            cx_pair(key[1], ix[1], key[3], ix[3], up);
            stride = 1;
        }
        // stride 1: slots (0,1) and (2,3); for size 2 the direction alternates inside the thread
        cx_pair(key[0], ix[0], key[1], ix[1], last || ((p0 + 0) & size) == 0);
        cx_pair(key[2], ix[2], key[3], ix[3], last || ((p0 + 2) & size) == 0);
    }
    // 2. the sorted runs merged pairwise in shared memory, log2(P / 128) levels (merge path): a
    //    thread finds by binary search how many of its 4 output ranks come from the first run,
    //    merges them in registers and stores them once the whole level has been read.  Every
    //    (key, index) pair of a real mode is distinct, so the order is the unique sorted one.
    for (int L = kSelectWarpSlots; L < P; L <<= 1) {
        ulonglong2 *kv = reinterpret_cast<ulonglong2 *>(sel_key + p0);
        kv[0] = make_ulonglong2(key[0], key[1]);
        kv[1] = make_ulonglong2(key[2], key[3]);
        *reinterpret_cast<int4 *>(sel_ix + p0) = make_int4(ix[0], ix[1], ix[2], ix[3]);
        __syncthreads();
        const int base = p0 & ~(2 * L - 1), d = p0 - base;  // this thread's first output rank
        const unsigned long long *ak = sel_key + base, *bk = ak + L;
        const int *ai = sel_ix + base, *bi = ai + L;
        int lo = d > L ? d - L : 0, hi = d < L ? d : L;
        while (lo < hi) {  // first i whose A[i] does not precede B[d - 1 - i]
            const int mid = (lo + hi) >> 1;
            if (sorts_before(ak[mid], ai[mid], bk[d - 1 - mid], bi[d - 1 - mid]))
                lo = mid + 1;
            else
                hi = mid;
        }
        int i = lo, j = d - lo;
#pragma unroll
        for (int r = 0; r < kSelectPerThread; ++r) {
            const bool take_a = j >= L || (i < L && sorts_before(ak[i], ai[i], bk[j], bi[j]));
            key[r] = take_a ? ak[i] : bk[j];
            ix[r] = take_a ? ai[i] : bi[j];
            i += take_a ? 1 : 0;
            j += take_a ? 0 : 1;
        }
        __syncthreads();  // every thread has read this level before any stores the next
    }

    // sorted powers to shared memory (slot j = rank j; padding holds +0)
    double *s_pw = reinterpret_cast<double *>(sel_key);
    double *s_cs = s_pw;  // c_j overwrites p_j: a round writes only ranks below where the next starts
    __syncthreads();  // the last shared-memory exchange stage may still be read
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r) s_pw[p0 + r] = key_power(key[r]);
    __syncthreads();

    // the cumulative sums c_j = fl(c_{j-1} + p_j), c_{-1} = 0, into s_cs[j] for every j < N.
    // While c stays in one binade [2^E, 2^(E+1)) (ulp U = 2^(E-52), E >= -1022), c/U is an
    // integer below 2^53 and fl(c + p) adds to it the integer nearest p/U (p <= c, so p/U < 2^53
    // and is read off p's bits); those additions are prefix sums, computed block-wide at once.
    // A step whose integer sum reaches 2^53 (the sum leaves the binade) or whose p/U lies exactly
    // halfway between integers (a tie, resolved by the parity of the sum) is taken by the FP64
    // adder itself, and the block starts again from there: a few rounds (binade changes are at
    // most log2 N + 1 apart) give the same bits as the left-to-right chain.
    const unsigned long long kTop = 1ull << 53;
    unsigned long long pm[kSelectPerThread];
    int pe[kSelectPerThread];
    double pv[kSelectPerThread];
    unsigned bad = 0u;
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r) {
        pv[r] = key_power(key[r]);
        const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(pv[r]));
        const int ef = (int)((bits >> 52) & 0x7ffu);
        pm[r] = (bits & (kTop / 2 - 1)) | (ef ? kTop / 2 : 0ull);
        pe[r] = ef ? ef - 1023 : -1022;
        if (p0 + r < N && ef == 0x7ff) bad = 1u;  // inf or nan: the chain below handles them
    }
    if (tid == 0) {
        s_cbits = static_cast<unsigned long long>(__double_as_longlong(s_pw[0]));
        s_cs[0] = s_pw[0];
        s_a = 1;
        s_fallback = 0;
    }
    __syncthreads();
    if (bad) s_fallback = 1;
    for (int round = 0;; ++round) {
        __syncthreads();
        const int a = s_a;
        if (a >= N || s_fallback) break;
        if (round >= kSelectMaxRounds) {  // many ties: finish with the sequential chain
            if (tid == 0) s_fallback = 1;
            continue;
        }
        const unsigned long long cb = s_cbits;
        const int cef = (int)((cb >> 52) & 0x7ffu);
        const int E = cef ? cef - 1023 : -1022;
        const unsigned long long Mc = (cb & (kTop / 2 - 1)) | (cef ? kTop / 2 : 0ull);
        unsigned long long q[kSelectPerThread], run = 0ull;
        bool tie[kSelectPerThread];
#pragma unroll
        for (int r = 0; r < kSelectPerThread; ++r) {
            const int j = p0 + r;
            q[r] = 0ull;
            tie[r] = false;
            if (j >= a && j < N) {
                const int d = E - pe[r];  // >= 0: p_j <= c
                if (d == 0) {
                    q[r] = pm[r];
                } else if (d < 64) {
                    const unsigned long long rem = pm[r] & ((1ull << d) - 1ull), half = 1ull << (d - 1);
                    q[r] = (pm[r] >> d) + (rem > half ? 1ull : 0ull);
                    tie[r] = rem == half;
                }  // d >= 64: p/U < 1/2, nothing added
            }
            run += q[r];
        }
        // block-wide exclusive prefix of the threads' sums
        unsigned long long incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_wsum[wid] = incl;
        if (tid == 0) s_exit = 0x7fffffff;
        __syncthreads();
        // every warp sums the totals of the warps before it itself (integer sums: exact in any
        // order), so no second barrier is needed
        unsigned long long wp = lane < wid ? s_wsum[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wp += __shfl_xor_sync(0xffffffffu, wp, o);
        unsigned long long M[kSelectPerThread];
        unsigned long long m = Mc + wp + (incl - run);
        int jfirst = 0x7fffffff;  // this thread's first step that leaves the binade or ties
#pragma unroll
        for (int r = 0; r < kSelectPerThread; ++r) {
            m += q[r];
            M[r] = m;
            const int j = p0 + r;
            if (j >= a && j < N && (m >= kTop || tie[r]) && j < jfirst) jfirst = j;
        }
        jfirst = __reduce_min_sync(0xffffffffu, jfirst);
        if (lane == 0 && jfirst != 0x7fffffff) atomicMin(&s_exit, jfirst);
        __syncthreads();
        const int jx = s_exit;
        // c_j = M_j U for the steps inside the binade: exponent field E + 1022 plus M's bits
        const unsigned long long ebase = static_cast<unsigned long long>(E + 1022) << 52;
#pragma unroll
        for (int r = 0; r < kSelectPerThread; ++r) {
            const int j = p0 + r;
            if (j >= a && j < N && j < jx) s_cs[j] = __longlong_as_double((long long)(ebase + M[r]));
            if (j == jx) {  // the FP64 adder takes the step that leaves the binade or ties
                const double cprev = j == a ? __longlong_as_double((long long)cb)
                                            : __longlong_as_double((long long)(ebase + M[r] - q[r]));
                const double cnew = __dadd_rn(cprev, pv[r]);
                s_cs[j] = cnew;
                s_cbits = static_cast<unsigned long long>(__double_as_longlong(cnew));
                s_a = j + 1;
            }
        }
        if (jx == 0x7fffffff && tid == 0) s_a = N;
    }
    __syncthreads();
    // the sequential chain from where the rounds stopped (non-finite powers, many ties)
    if (s_fallback && tid == 0) {
        int j = s_a;
        double c = s_cs[j - 1];
        for (; j < N; ++j) {
            c = __dadd_rn(c, s_pw[j]);
            s_cs[j] = c;
        }
    }
    if (tid == 0) s_total = s_cs[N - 1];
    __syncthreads();
    const double total = s_total;
    if (!(total > 0.0)) return;  // uniform: nothing kept at a knot without power
    const double target = (1.0 - eps) * total;
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r) {
        const int j = p0 + r;
        if (j >= N) break;
        const double cj = s_cs[j];
        if (cj >= target) {
            atomicMin(&s_cut, j);
            break;
        }
    }
    __syncthreads();
    const int cut = s_cut;  // no rank reaching the target keeps every mode
#pragma unroll
    for (int r = 0; r < kSelectPerThread; ++r)
        if (p0 + r < N && p0 + r <= cut) mask[ix[r]] = 1;
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
