// rb.cu -- mode amplitudes from reduced-basis coefficients (arXiv:2104.04582 Sec. 3.E).
//
// Each knot k carries Nb complex coefficients alpha_k; its N mode amplitudes are
//     A_k,i = s_k sum_j alpha_k,j B_j,i,
// with s_k = nu_k / ||alpha_k B|| when target norms nu_k are given (the renormalisation of the
// network's output to the trajectory's norm spline), else s_k = 1.  The norm comes from the
// basis Gram matrix, ||alpha B||^2 = sum_jl alpha_j conj(alpha_l) G_jl with G = B B^H, so the
// scale is known before the product and no second pass over the output is needed.
//
// FP64 path: a tiled complex GEMM on the FP64 pipe.
// Mixed path: the complex product as one real GEMM on the tcgen05 tensor cores,
//     [Re A_i, Im A_i] = sum_q a_q Bhat_q,(2i, 2i+1),  a = [Re(s alpha) | Im(s alpha)] (2 Nb),
//     Bhat_q,2i = (Re B_qi | -Im B_qi),  Bhat_q,2i+1 = (Im B_qi | Re B_qi),
// in bf16 with FP32 accumulation in tensor memory.  To keep FP32 accuracy every operand is split
// into three bf16 parts x = hi + mid + lo (8 significant bits each) and the six products of
// order <= 2^-16 (hi.hi, hi.mid, mid.hi, hi.lo, mid.mid, lo.hi) are laid side by side along K,
// so one GEMM of depth 6 x 2 Nb sums them all.
//
// Operands are packed once into the canonical K-major layout without swizzle that the tensor
// core's shared-memory descriptors read: 8 x 8 bf16 "core matrices" of 16-byte rows, core
// matrices adjacent in K 128 bytes apart, 8-row groups 1024 bytes apart.  A k-block of 64
// columns of a 128-row (A) or 256-row (B) tile is one contiguous 16 / 32 KB block in global
// memory, so each pipeline stage is filled by two bulk asynchronous copies.
#include <cuda_bf16.h>

#include "async.cuh"
#include "fewsum_internal.h"

namespace fewsum {

constexpr int kRbTileM = 128;   // knots per tile: tensor-memory lanes
constexpr int kRbTileN = 256;   // real output columns per tile: 128 modes, re/im interleaved
constexpr int kRbTileK = 64;    // bf16 columns per k-block: 128 bytes per row
constexpr int kRbStages = 4;    // shared-memory pipeline depth
constexpr int kRbParts = 6;     // split products laid along K
constexpr uint32_t kRbABytes = kRbTileM * kRbTileK * 2;  // 16 KB
constexpr uint32_t kRbBBytes = kRbTileN * kRbTileK * 2;  // 32 KB
constexpr uint32_t kRbStageBytes = kRbABytes + kRbBBytes;

// Which bf16 part of the A (coefficient) and B (basis) operand each K segment holds, so that
// segment g multiplies A part kPartA[g] by B part kPartB[g] (0 = hi, 1 = mid, 2 = lo).
__constant__ int kPartA[kRbParts] = {0, 0, 1, 0, 1, 2};
__constant__ int kPartB[kRbParts] = {0, 1, 0, 2, 1, 0};

__host__ __device__ constexpr uint32_t core_offset(int r, int c)
{
    return (uint32_t)(r >> 3) * 1024u + (uint32_t)(c >> 3) * 128u + (uint32_t)(r & 7) * 16u +
           (uint32_t)(c & 7) * 2u;
}

__device__ __forceinline__ __nv_bfloat16 split_part(float x, int part)
{
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    if (part == 0) return hi;
    const float r1 = x - __bfloat162float(hi);  // exact: x and hi share the leading bits
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    if (part == 1) return mid;
    return __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// ---- basis set-up -------------------------------------------------------------------------

// Gram matrix G_jl = sum_i B_ji conj(B_li), stored transposed (gt[l][j] = G_jl) so that the
// lanes of a warp, one per j, read consecutive entries; FP64 and an FP32 copy.
__global__ void k_rb_gram(const double *__restrict__ bre, const double *__restrict__ bim, int Nb,
                          int N, double2 *__restrict__ gt64, float2 *__restrict__ gt32)
{
    const int j = blockIdx.x % Nb, l = blockIdx.x / Nb;
    double sr = 0.0, si = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double ar = bre[(size_t)j * N + i], ai = bim[(size_t)j * N + i];
        const double cr = bre[(size_t)l * N + i], ci = bim[(size_t)l * N + i];
        sr += ar * cr + ai * ci;  // B_ji conj(B_li)
        si += ai * cr - ar * ci;
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) { red[0][w] = sr; red[1][w] = si; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int k = 0; k < nw; ++k) { tr += red[0][k]; ti += red[1][k]; }
        gt64[(size_t)l * Nb + j] = make_double2(tr, ti);
        gt32[(size_t)l * Nb + j] = make_float2((float)tr, (float)ti);
    }
}

// Basis operand of the real GEMM, split and packed: row n' of tile n'/256 is real output column
// n' (mode n'/2, real part for even n', imaginary for odd); column c = g * 2Nb + q holds part
// kPartB[g] of Bhat_q,n'.  Rows past 2N and columns past 6 x 2Nb are zero.
__global__ void k_rb_pack_b(const double *__restrict__ bre, const double *__restrict__ bim, int Nb,
                            int N, int n_kb, int n_tiles, unsigned char *__restrict__ bpack)
{
    const long long chunks = (long long)n_tiles * kRbTileN * n_kb * (kRbTileK / 8);
    const int Kr = 2 * Nb;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < chunks;
         t += (long long)gridDim.x * blockDim.x) {
        const int q8 = (int)(t % (n_kb * (kRbTileK / 8)));
        const int row = (int)(t / (n_kb * (kRbTileK / 8)));
        const int c0 = q8 * 8;
        uint32_t w[4];
        for (int e = 0; e < 8; e += 2) {
            __nv_bfloat16 v[2];
            for (int h = 0; h < 2; ++h) {
                const int c = c0 + e + h, g = c / Kr, q = c % Kr;
                float x = 0.0f;
                int part = 0;
                if (g < kRbParts && row < 2 * N) {
                    const int i = row >> 1, j = q % Nb;
                    const bool imag_out = row & 1, from_im = q >= Nb;
                    const double br = bre[(size_t)j * N + i], bi = bim[(size_t)j * N + i];
                    x = (float)(imag_out ? (from_im ? br : bi) : (from_im ? -bi : br));
                    part = kPartB[g];
                }
                v[h] = split_part(x, part);
            }
            w[e / 2] = pack2(v[0], v[1]);
        }
        const int tile = row / kRbTileN, kb = c0 / kRbTileK;
        unsigned char *blk = bpack + ((size_t)tile * n_kb + kb) * kRbBBytes;
        *reinterpret_cast<uint4 *>(blk + core_offset(row % kRbTileN, c0 % kRbTileK)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ---- per call -----------------------------------------------------------------------------

// s_k = nu_k / sqrt(sum_j alpha_j sum_l G_jl conj(alpha_l)), one warp per knot, in the
// arithmetic type T of the path.  A non-finite or negative target norm latches
// ERRBIT_NONFINITE; a zero quadratic form (alpha_k B = 0) gives s_k = 0.
template <typename T, typename C>
__global__ void k_rb_scale(const double *__restrict__ are, const double *__restrict__ aim, int M,
                           int Nb, const C *__restrict__ gt, const double *__restrict__ nu,
                           double *__restrict__ scale, unsigned *__restrict__ err)
{
    extern __shared__ unsigned char rb_scale_smem[];
    const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *al = reinterpret_cast<T *>(rb_scale_smem) + (size_t)w * 2 * Nb;  // [re | im] of alpha_k
    for (int k = blockIdx.x * warps + w; k < M; k += gridDim.x * warps) {
        for (int j = lane; j < Nb; j += 32) {
            al[j] = (T)are[(size_t)k * Nb + j];
            al[Nb + j] = (T)aim[(size_t)k * Nb + j];
        }
        __syncwarp();
        T q = 0;
        for (int j = lane; j < Nb; j += 32) {
            T tr = 0, ti = 0;  // sum_l G_jl conj(alpha_l)
            for (int l = 0; l < Nb; ++l) {
                const C g = gt[(size_t)l * Nb + j];
                const T xr = al[l], xi = al[Nb + l];
                tr += (T)g.x * xr + (T)g.y * xi;
                ti += (T)g.y * xr - (T)g.x * xi;
            }
            q += al[j] * tr - al[Nb + j] * ti;  // Re(alpha_j t_j)
        }
        for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
        if (lane == 0) {
            const double v = nu[k];
            if (!(v >= 0.0) || !isfinite(v)) atomicOr(err, ERRBIT_NONFINITE);
            scale[k] = q > (T)0 ? v / sqrt((double)q) : 0.0;
        }
        __syncwarp();
    }
}

// Coefficient operand: row k of tile k/128, column c = g * 2Nb + q holds part kPartA[g] of
// s_k alpha_k,q (real parts for q < Nb, imaginary parts after).  Rows past M are zero.
__global__ void k_rb_pack_a(const double *__restrict__ are, const double *__restrict__ aim, int M,
                            int Nb, int n_kb, int m_tiles, const double *__restrict__ scale,
                            unsigned char *__restrict__ apack)
{
    const long long chunks = (long long)m_tiles * kRbTileM * n_kb * (kRbTileK / 8);
    const int Kr = 2 * Nb;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < chunks;
         t += (long long)gridDim.x * blockDim.x) {
        const int q8 = (int)(t % (n_kb * (kRbTileK / 8)));
        const int row = (int)(t / (n_kb * (kRbTileK / 8)));
        const int c0 = q8 * 8;
        const double s = (scale && row < M) ? scale[row] : 1.0;
        uint32_t w[4];
        for (int e = 0; e < 8; e += 2) {
            __nv_bfloat16 v[2];
            for (int h = 0; h < 2; ++h) {
                const int c = c0 + e + h, g = c / Kr, q = c % Kr;
                float x = 0.0f;
                int part = 0;
                if (g < kRbParts && row < M) {
                    const double a = q < Nb ? are[(size_t)row * Nb + q] : aim[(size_t)row * Nb + q - Nb];
                    x = (float)(s * a);
                    part = kPartA[g];
                }
                v[h] = split_part(x, part);
            }
            w[e / 2] = pack2(v[0], v[1]);
        }
        const int tile = row / kRbTileM, kb = c0 / kRbTileK;
        unsigned char *blk = apack + ((size_t)tile * n_kb + kb) * kRbABytes;
        *reinterpret_cast<uint4 *>(blk + core_offset(row % kRbTileM, c0 % kRbTileK)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ---- tensor-core GEMM ---------------------------------------------------------------------

// Shared-memory matrix descriptor (tcgen05): start address, leading (K-direction) and stride
// (8-row group) byte offsets, each in 16-byte units; bits 46-48 hold the fixed value 0b001;
// base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), bf16 A and B (bits 7-9
// and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kRbIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kRbTileN >> 3) << 17) |
                              ((uint32_t)(kRbTileM >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every tcgen05.mma this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct RbMmaArgs {
    const unsigned char *apack;  // [m_tiles][n_kb] blocks of kRbABytes
    const unsigned char *bpack;  // [n_tiles][n_kb] blocks of kRbBBytes
    double *out_re, *out_im;     // [M][N]
    int M, N, n_kb;
    unsigned *err;
};

// One CTA per (basis tile, knot tile): thread 0 streams the k-blocks through a kRbStages ring
// of shared-memory stages and issues the MMAs; then the four warps read the 128 x 256 FP32
// accumulator from tensor memory (warp w owns lanes 32w..32w+31, i.e. knots) and store FP64.
__global__ void __launch_bounds__(128, 1) k_rb_mma(RbMmaArgs a)
{
    extern __shared__ unsigned char rb_mma_smem[];
    __shared__ __align__(8) uint64_t full[kRbStages], empty[kRbStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = blockIdx.x, mt = blockIdx.y;
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(rb_mma_smem) + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base, *sB = base + kRbStages * kRbABytes;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"((uint32_t)kRbTileN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kRbStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (tid == 0) {
        const unsigned char *ga = a.apack + (size_t)mt * a.n_kb * kRbABytes;
        const unsigned char *gb = a.bpack + (size_t)nt * a.n_kb * kRbBBytes;
        const int pre = a.n_kb < kRbStages ? a.n_kb : kRbStages;
        for (int s = 0; s < pre; ++s) {
            mbar_arrive_expect_tx(&full[s], kRbStageBytes);
            bulk_g2s(sA + s * kRbABytes, ga + (size_t)s * kRbABytes, kRbABytes, &full[s]);
            bulk_g2s(sB + s * kRbBBytes, gb + (size_t)s * kRbBBytes, kRbBBytes, &full[s]);
        }
        int issued = pre, consumed = 0;
        bool ok = true;
        for (int kb = 0; kb < a.n_kb; ++kb) {
            const int s = kb % kRbStages;
            if (!mbar_wait_bounded(&full[s], (uint32_t)((kb / kRbStages) & 1))) { ok = false; break; }
            consumed = kb + 1;
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * kRbABytes), b0 = smem_u32(sB + s * kRbBBytes);
#pragma unroll
            for (int k = 0; k < kRbTileK / 16; ++k)  // K = 16 per MMA: two core matrices
                tc_mma(tmem, smem_desc(a0 + k * 256, 128, 1024), smem_desc(b0 + k * 256, 128, 1024),
                       kRbIdesc, (uint32_t)((kb | k) != 0));
            tc_commit(&empty[s]);
            // refill the stage of the previous k-block once its MMAs have drained
            const int kp = kb - 1, nk = kp + kRbStages;
            if (kp >= 0 && nk < a.n_kb) {
                const int sp = kp % kRbStages;
                if (!mbar_wait_bounded(&empty[sp], (uint32_t)((kp / kRbStages) & 1))) { ok = false; break; }
                mbar_arrive_expect_tx(&full[sp], kRbStageBytes);
                bulk_g2s(sA + sp * kRbABytes, ga + (size_t)nk * kRbABytes, kRbABytes, &full[sp]);
                bulk_g2s(sB + sp * kRbBBytes, gb + (size_t)nk * kRbBBytes, kRbBBytes, &full[sp]);
                issued = nk + 1;
            }
        }
        if (!ok) {
            // let copies already in flight land before the CTA can exit
            for (int kb = consumed; kb < issued; ++kb)
                mbar_wait_bounded(&full[kb % kRbStages], (uint32_t)((kb / kRbStages) & 1));
            s_abort = 1;
        }
        tc_commit(&done);
    }
    __syncthreads();
    if (!mbar_wait_bounded(&done, 0)) s_abort = 1;
    tc_fence_after();
    __syncthreads();
    if (!s_abort) {
        const int row = mt * kRbTileM + warp * 32 + lane;
        for (int c = 0; c < kRbTileN / 32; ++c) {
            uint32_t v[32];
            tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
            if (row < a.M) {
                const int i0 = nt * (kRbTileN / 2) + c * 16;
                double *ore = a.out_re + (size_t)row * a.N, *oim = a.out_im + (size_t)row * a.N;
#pragma unroll
                for (int t = 0; t < 16; ++t)
                    if (i0 + t < a.N) {
                        ore[i0 + t] = (double)__uint_as_float(v[2 * t]);
                        oim[i0 + t] = (double)__uint_as_float(v[2 * t + 1]);
                    }
            }
        }
    } else if (tid == 0) {
        atomicOr(a.err, ERRBIT_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)kRbTileN)
                     : "memory");
}

// ---- FP64 GEMM ----------------------------------------------------------------------------

constexpr int kRb64Rows = 32, kRb64Modes = 64, kRb64J = 16;

// 32 knots x 64 modes per block of 256 threads; thread (ty, tx) owns knots ty, ty + 16 and
// modes tx + 16 q, q < 4; coefficient and basis tiles staged in shared memory.
__global__ void __launch_bounds__(256) k_rb_fp64(const double *__restrict__ are,
                                                 const double *__restrict__ aim,
                                                 const double *__restrict__ bre,
                                                 const double *__restrict__ bim, int M, int Nb, int N,
                                                 const double *__restrict__ scale,
                                                 double *__restrict__ ore, double *__restrict__ oim)
{
    __shared__ double2 sa[kRb64Rows][kRb64J];
    __shared__ double2 sb[kRb64J][kRb64Modes];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int k0 = blockIdx.y * kRb64Rows, i0 = blockIdx.x * kRb64Modes;
    double accr[2][4] = {}, acci[2][4] = {};
    for (int j0 = 0; j0 < Nb; j0 += kRb64J) {
        for (int e = threadIdx.x; e < kRb64Rows * kRb64J; e += 256) {
            const int r = e / kRb64J, j = e % kRb64J, k = k0 + r, jj = j0 + j;
            sa[r][j] = (k < M && jj < Nb) ? make_double2(are[(size_t)k * Nb + jj], aim[(size_t)k * Nb + jj])
                                          : make_double2(0.0, 0.0);
        }
        for (int e = threadIdx.x; e < kRb64J * kRb64Modes; e += 256) {
            const int j = e / kRb64Modes, c = e % kRb64Modes, jj = j0 + j, i = i0 + c;
            sb[j][c] = (jj < Nb && i < N) ? make_double2(bre[(size_t)jj * N + i], bim[(size_t)jj * N + i])
                                          : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < kRb64J; ++j) {
            const double2 x0 = sa[ty][j], x1 = sa[ty + 16][j];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double2 b = sb[j][tx + 16 * q];
                accr[0][q] = fma(x0.x, b.x, fma(-x0.y, b.y, accr[0][q]));
                acci[0][q] = fma(x0.x, b.y, fma(x0.y, b.x, acci[0][q]));
                accr[1][q] = fma(x1.x, b.x, fma(-x1.y, b.y, accr[1][q]));
                acci[1][q] = fma(x1.x, b.y, fma(x1.y, b.x, acci[1][q]));
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = k0 + ty + 16 * h;
        if (k >= M) continue;
        const double s = scale ? scale[k] : 1.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tx + 16 * q;
            if (i < N) {
                ore[(size_t)k * N + i] = s * accr[h][q];
                oim[(size_t)k * N + i] = s * acci[h][q];
            }
        }
    }
}

// ---- launchers ----------------------------------------------------------------------------

RbLayout rb_layout(int Nb, int N, int M)
{
    RbLayout L;
    L.n_kb = (kRbParts * 2 * Nb + kRbTileK - 1) / kRbTileK;
    L.n_tiles = (2 * N + kRbTileN - 1) / kRbTileN;
    L.m_tiles = (M + kRbTileM - 1) / kRbTileM;
    L.bpack_bytes = (size_t)L.n_tiles * L.n_kb * kRbBBytes;
    L.apack_bytes = (size_t)L.m_tiles * L.n_kb * kRbABytes;
    return L;
}

cudaError_t launch_rb_basis(const double *bre, const double *bim, int Nb, int N, double2 *gt64,
                            float2 *gt32, unsigned char *bpack, int sm_count, cudaStream_t st)
{
    const RbLayout L = rb_layout(Nb, N, 0);
    k_rb_gram<<<Nb * Nb, 128, 0, st>>>(bre, bim, Nb, N, gt64, gt32);
    k_rb_pack_b<<<sm_count * 8, 256, 0, st>>>(bre, bim, Nb, N, L.n_kb, L.n_tiles, bpack);
    return cudaGetLastError();
}

cudaError_t launch_rb(const double *are, const double *aim, int M, int Nb, int N, const double *nu,
                      bool fp64, const double *bre, const double *bim, const double2 *gt64,
                      const float2 *gt32, const unsigned char *bpack, double *scale,
                      unsigned char *apack, double *ore, double *oim, unsigned *err, int sm_count,
                      cudaStream_t st)
{
    if (M == 0) return cudaSuccess;
    const RbLayout L = rb_layout(Nb, N, M);
    if (nu) {
        const int warps = 8;
        const int blocks = (M + warps - 1) / warps;
        const int grid = blocks < sm_count * 8 ? blocks : sm_count * 8;
        if (fp64)
            k_rb_scale<double, double2><<<grid, warps * 32, warps * 2 * Nb * sizeof(double), st>>>(
                are, aim, M, Nb, gt64, nu, scale, err);
        else
            k_rb_scale<float, float2><<<grid, warps * 32, warps * 2 * Nb * sizeof(float), st>>>(
                are, aim, M, Nb, gt32, nu, scale, err);
    }
    const double *sc = nu ? scale : nullptr;
    if (fp64) {
        dim3 grid((N + kRb64Modes - 1) / kRb64Modes, (M + kRb64Rows - 1) / kRb64Rows);
        k_rb_fp64<<<grid, 256, 0, st>>>(are, aim, bre, bim, M, Nb, N, sc, ore, oim);
        return cudaGetLastError();
    }
    k_rb_pack_a<<<sm_count * 8, 256, 0, st>>>(are, aim, M, Nb, L.n_kb, L.m_tiles, sc, apack);
    const int smem = kRbStages * (int)kRbStageBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_rb_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    RbMmaArgs args{apack, bpack, ore, oim, M, N, L.n_kb, err};
    k_rb_mma<<<dim3(L.n_tiles, L.m_tiles), 128, smem, st>>>(args);
    return cudaGetLastError();
}

}  // namespace fewsum
