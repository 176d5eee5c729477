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
//     [Re A_i, Im A_i] = s sum_q a_q Bhat_q,(2i, 2i+1),  a = [Re alpha | Im alpha] (2 Nb),
//     Bhat_q,2i = (Re B_qi | -Im B_qi),  Bhat_q,2i+1 = (Im B_qi | Re B_qi),
// in fp16 with FP32 accumulation in tensor memory.  To keep near-FP32 accuracy every operand is
// split into two fp16 parts x = hi + lo (11 significant bits each) and the three products of
// order <= 2^-11 (hi.hi, hi.lo, lo.hi) are laid side by side along K, so one GEMM of depth
// 3 x 2 Nb sums them all.  fp16's narrow exponent range is handled by exact power-of-two
// scaling: each knot's coefficient row and each mode's basis column are scaled so that their
// largest magnitude lies in [2^14, 2^15) before the split, and the epilogue multiplies the
// accumulator back by both inverse powers and by the knot's renormalisation s (so the scale's
// kernels run beside the coefficient pack, on a second stream, and are joined before the
// product).  An entry far below its row or column maximum keeps
// an absolute error near 2^-24 of that maximum.
//
// The product is computed transposed, A^T = Bhat^T a^T: the MMA's M side (tensor-memory lanes)
// is 128 real output columns of 64 modes (rows 0-63 the real parts, 64-127 the imaginary parts)
// and its N side (tensor-memory columns) 256 knots.  A lane of the accumulator then holds one
// output column for consecutive knots, so for each knot a warp stores 32 consecutive modes (256
// contiguous bytes) straight from registers.  Operands are packed once into the canonical K-major
// layout without swizzle that the tensor core's shared-memory descriptors read: 8 x 8 fp16 "core
// matrices" of 16-byte rows, core matrices adjacent in K 128 bytes apart, 8-row groups 1024
// bytes apart.  A k-block of 64 columns of a 128-row basis tile or a 256-row coefficient tile is
// one contiguous 16 / 32 KB block in global memory, so each pipeline stage is filled by two bulk
// asynchronous copies.
#include <cuda_fp16.h>

#include "async.cuh"
#include "convert.cuh"
#include "fewsum_internal.h"

namespace fewsum {

constexpr int kRbTileM = 128;   // MMA M, tensor-memory lanes: real output columns of 64 modes
constexpr int kRbModes = kRbTileM / 2;  // modes per basis tile
constexpr int kRbTileN = 256;   // MMA N, tensor-memory columns: knots per coefficient tile
constexpr int kRbTileK = 64;    // fp16 columns per k-block: 128 bytes per row
constexpr int kRbStages = 4;    // shared-memory pipeline depth
constexpr int kRbParts = 3;     // split products laid along K
constexpr uint32_t kRbABytes = kRbTileM * kRbTileK * 2;  // 16 KB: basis (A operand)
constexpr uint32_t kRbBBytes = kRbTileN * kRbTileK * 2;  // 32 KB: coefficients (B operand)
constexpr uint32_t kRbStageBytes = kRbABytes + kRbBBytes;

// Which fp16 part of the A (coefficient) and B (basis) operand each K segment g < kRbParts
// holds (0 = hi, 1 = lo): the segments multiply hi x hi, hi x lo and lo x hi.  Arithmetic, not a
// table, so lanes at different segments need no divergent constant-memory reads.
__host__ __device__ constexpr int part_a(int g) { return g == 2 ? 1 : 0; }
__host__ __device__ constexpr int part_b(int g) { return g == 1 ? 1 : 0; }
constexpr int kRbMaxExp = 100;  // bound on the power-of-two scaling exponents

__host__ __device__ constexpr uint32_t core_offset(int r, int c)
{
    return (uint32_t)(r >> 3) * 1024u + (uint32_t)(c >> 3) * 128u + (uint32_t)(r & 7) * 16u +
           (uint32_t)(c & 7) * 2u;
}

__device__ __forceinline__ __half split_part(float x, int part)
{
    const __half hi = __float2half_rn(x);
    if (part == 0) return hi;
    return __float2half_rn(x - __half2float(hi));  // the difference is exact in FP32
}

__device__ __forceinline__ uint32_t pack2(__half a, __half b)
{
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// 2^e as a float, |e| <= kRbMaxExp.
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }

// Exponent e with m 2^e in [2^14, 2^15) for m > 0 (0 for m = 0), clamped to +-kRbMaxExp.
__device__ __forceinline__ int scale_exp(float m)
{
    if (!(m > 0.0f)) return 0;
    const int e = 14 - (int)((__float_as_uint(m) >> 23) & 0xffu) + 127;
    return e > kRbMaxExp ? kRbMaxExp : (e < -kRbMaxExp ? -kRbMaxExp : e);
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

// Scaling exponent of each mode's basis column: bexp[i] puts max_j max(|Re B_ji|, |Im B_ji|)
// into [2^14, 2^15); padded modes get 0.
__global__ void k_rb_bexp(const double *__restrict__ bre, const double *__restrict__ bim, int Nb,
                          int N, int n_modes_padded, int *__restrict__ bexp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_modes_padded) return;
    double m = 0.0;
    if (i < N)
        for (int j = 0; j < Nb; ++j)
            m = fmax(m, fmax(fabs(bre[(size_t)j * N + i]), fabs(bim[(size_t)j * N + i])));
    bexp[i] = scale_exp((float)m);
}

// Basis operand (the MMA's A side), scaled, split and packed: row r of basis tile b is the real
// (r < 64) or imaginary (r >= 64) output column of mode 64 b + (r mod 64); column c = g 2Nb + q
// holds part part_b(g) of 2^bexp[mode] Bhat for that column.  Modes past N and columns past
// 3 x 2Nb are zero.
__global__ void k_rb_pack_b(const double *__restrict__ bre, const double *__restrict__ bim, int Nb,
                            int N, int n_kb, int n_tiles, const int *__restrict__ bexp,
                            unsigned char *__restrict__ bpack)
{
    const long long chunks = (long long)n_tiles * kRbTileM * n_kb * (kRbTileK / 8);
    const int Kr = 2 * Nb;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < chunks;
         t += (long long)gridDim.x * blockDim.x) {
        const int q8 = (int)(t % (n_kb * (kRbTileK / 8)));
        const int row = (int)(t / (n_kb * (kRbTileK / 8)));
        const int c0 = q8 * 8;
        const int rr = row % kRbTileM, i = (row / kRbTileM) * kRbModes + (rr % kRbModes);
        const bool imag_out = rr >= kRbModes;
        uint32_t w[4];
        for (int e = 0; e < 8; e += 2) {
            __half v[2];
            for (int h = 0; h < 2; ++h) {
                const int c = c0 + e + h, g = c / Kr, q = c % Kr;
                float x = 0.0f;
                int part = 0;
                if (g < kRbParts && i < N) {
                    const int j = q % Nb;
                    const bool from_im = q >= Nb;
                    const double br = bre[(size_t)j * N + i], bi = bim[(size_t)j * N + i];
                    const double v = imag_out ? (from_im ? br : bi) : (from_im ? -bi : br);
                    x = (float)ldexp(v, bexp[i]);
                    part = part_b(g);
                }
                v[h] = split_part(x, part);
            }
            w[e / 2] = pack2(v[0], v[1]);
        }
        const int tile = row / kRbTileM, kb = c0 / kRbTileK;
        unsigned char *blk = bpack + ((size_t)tile * n_kb + kb) * kRbABytes;
        *reinterpret_cast<uint4 *>(blk + core_offset(rr, c0 % kRbTileK)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ---- per call -----------------------------------------------------------------------------

// Quadratic form q_k = ||alpha_k B||^2 = sum_j Re(alpha_j t_j), t_j = sum_l G_jl conj(alpha_l), in
// the arithmetic type T of the path, as a small register-blocked product: a block takes 32 knots
// and 64 values of j, l advancing in chunks of 64 staged in (dynamic) shared memory; a thread owns
// 4 knots x 2 values of j (j and j + 32), so 6 shared-memory reads feed 16 complex multiply-adds.
// Partial sums over j are reduced per warp and added to q (FP64, zeroed beforehand); k_rb_norm
// then forms s_k.  Used by the FP64 path and, in FP32, for bases of more than 128 vectors.
constexpr int kQRows = 32, kQJ = 64, kQL = 64, kQThreads = 256, kQPer = 4;

template <typename C>
constexpr int rb_quad_smem() { return (kQL * kQJ + kQRows * kQL) * (int)sizeof(C); }

template <typename T, typename C>
__global__ void __launch_bounds__(kQThreads)
k_rb_quad(const double *__restrict__ are, const double *__restrict__ aim, int M, int Nb,
          const C *__restrict__ gt, double *__restrict__ q)
{
    extern __shared__ __align__(16) unsigned char rb_quad_smem_raw[];
    C(*sg)[kQJ] = reinterpret_cast<C(*)[kQJ]>(rb_quad_smem_raw);                       // G_jl [l][j]
    C(*sa)[kQL] = reinterpret_cast<C(*)[kQL]>(rb_quad_smem_raw + kQL * kQJ * sizeof(C));  // alpha
    const int tid = threadIdx.x, jl = tid & 31, rg = tid >> 5;  // rg: knots 4 rg .. 4 rg + 3
    const int j0 = blockIdx.x * kQJ + jl, k0 = blockIdx.y * kQRows;
    T tr[kQPer][2], ti[kQPer][2];
#pragma unroll
    for (int i = 0; i < kQPer; ++i) tr[i][0] = tr[i][1] = ti[i][0] = ti[i][1] = 0;
    for (int l0 = 0; l0 < Nb; l0 += kQL) {
        const int lc = Nb - l0 < kQL ? Nb - l0 : kQL;
        __syncthreads();
        for (int e = tid; e < lc * kQJ; e += kQThreads) {
            const int l = l0 + e / kQJ, jx = blockIdx.x * kQJ + e % kQJ;
            sg[e / kQJ][e % kQJ] = jx < Nb ? gt[(size_t)l * Nb + jx] : C{};
        }
        for (int e = tid; e < kQRows * lc; e += kQThreads) {
            const int r = e / lc, l = l0 + e % lc, k = k0 + r;
            C v{};
            if (k < M) {
                v.x = (T)are[(size_t)k * Nb + l];
                v.y = (T)aim[(size_t)k * Nb + l];
            }
            sa[r][e % lc] = v;
        }
        __syncthreads();
#pragma unroll 2
        for (int l = 0; l < lc; ++l) {
            const C g0 = sg[l][jl], g1 = sg[l][jl + 32];
#pragma unroll
            for (int i = 0; i < kQPer; ++i) {
                const C x = sa[rg * kQPer + i][l];
                tr[i][0] += g0.x * x.x + g0.y * x.y;  // G_jl conj(alpha_l)
                ti[i][0] += g0.y * x.x - g0.x * x.y;
                tr[i][1] += g1.x * x.x + g1.y * x.y;
                ti[i][1] += g1.y * x.x - g1.x * x.y;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kQPer; ++i) {
        const int k = k0 + rg * kQPer + i;
        T c = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + 32 * h;
            if (k < M && j < Nb)
                c += (T)are[(size_t)k * Nb + j] * tr[i][h] - (T)aim[(size_t)k * Nb + j] * ti[i][h];
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (jl == 0 && k < M) atomicAdd(q + k, (double)c);
    }
}

// Mixed path, Nb <= 128: the renormalisation scale in one kernel, one wave.  A block takes
// kTRows knots; their FP32 coefficients and the whole FP32 Gram matrix (j padded to 128) sit in
// shared memory.  The sum over l is split among kTParts thread groups (l = part mod kTParts);
// within a group thread (rg, jg) owns knots 4 rg .. 4 rg + 3 and j = jg + 16 t, t < 8, so 12
// shared-memory reads (half of them broadcasts) feed 128 multiply-adds per l.  The 16 threads of
// a knot group share a half-warp and reduce their partial q_k by shuffles; the groups' partials
// are added in group order and s_k = nu_k / sqrt(q_k) written directly (0 for q_k = 0; a
// non-finite or negative nu_k latches ERRBIT_NONFINITE).
constexpr int kTRows = 48, kTJ = 128, kTGroup = (kTRows / 4) * 16, kTParts = 3;
constexpr int kTThreads = kTGroup * kTParts;
constexpr int kTMaxBasis = kTJ;

__global__ void __launch_bounds__(kTThreads)
k_rb_scale_tile(const double *__restrict__ are, const double *__restrict__ aim, int M, int Nb,
                const float2 *__restrict__ gt, const double *__restrict__ nu,
                double *__restrict__ scale, unsigned *__restrict__ err)
{
    extern __shared__ __align__(16) float2 rb_tile_smem[];
    float2 *as = rb_tile_smem;                 // [kTRows][Nb] alpha
    float2 *gs = rb_tile_smem + kTRows * Nb;   // [Nb][kTJ] G_jl stored [l][j], zero for j >= Nb
    __shared__ float q_part[kTParts][kTRows];
    const int tid = threadIdx.x, part = tid / kTGroup, local = tid - part * kTGroup;
    const int jg = local & 15, rg = local >> 4;
    const int k0 = blockIdx.x * kTRows;
    // staging: 8 independent loads in flight per thread per round trip
    constexpr int kU = 8;
    for (int e0 = tid; e0 < kTRows * Nb; e0 += kTThreads * kU) {
        double vr[kU], vi[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = e0 + u * kTThreads, k = k0 + e / (Nb > 0 ? Nb : 1);
            const bool ok = e < kTRows * Nb && k < M;
            vr[u] = ok ? are[(size_t)k0 * Nb + e] : 0.0;  // rows k0.. are contiguous: index k0*Nb + e
            vi[u] = ok ? aim[(size_t)k0 * Nb + e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = e0 + u * kTThreads;
            if (e < kTRows * Nb) as[e] = make_float2(f64_to_f32(vr[u]), f64_to_f32(vi[u]));
        }
    }
    for (int e0 = tid; e0 < Nb * kTJ; e0 += kTThreads * kU) {
        float2 v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = e0 + u * kTThreads, l = e / kTJ, j = e % kTJ;
            v[u] = (e < Nb * kTJ && j < Nb) ? gt[(size_t)l * Nb + j] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int e = e0 + u * kTThreads;
            if (e < Nb * kTJ) gs[e] = v[u];
        }
    }
    __syncthreads();
    float tr[4][8], ti[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < 8; ++t) tr[r][t] = ti[r][t] = 0.f;
    for (int l = part; l < Nb; l += kTParts) {
        float2 x[4], g[8];
#pragma unroll
        for (int r = 0; r < 4; ++r) x[r] = as[(rg * 4 + r) * Nb + l];
#pragma unroll
        for (int t = 0; t < 8; ++t) g[t] = gs[l * kTJ + jg + 16 * t];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                tr[r][t] += g[t].x * x[r].x + g[t].y * x[r].y;  // G_jl conj(alpha_l)
                ti[r][t] += g[t].y * x[r].x - g[t].x * x[r].y;
            }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int row = rg * 4 + r;
        float q = 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = jg + 16 * t;
            if (j < Nb) {
                const float2 a = as[row * Nb + j];
                q += a.x * tr[r][t] - a.y * ti[r][t];  // Re(alpha_j t_j)
            }
        }
        for (int o = 8; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (jg == 0) q_part[part][row] = q;
    }
    __syncthreads();
    if (tid < kTRows && k0 + tid < M) {
        const int k = k0 + tid;
        float q = q_part[0][tid];
#pragma unroll
        for (int p = 1; p < kTParts; ++p) q += q_part[p][tid];
        const double v = nu[k];
        if (!(v >= 0.0) || !isfinite(v)) atomicOr(err, ERRBIT_NONFINITE);
        scale[k] = q > 0.f ? v / sqrt((double)q) : 0.0;
    }
}

// s_k = nu_k / sqrt(q_k) (0 when q_k = 0, i.e. alpha_k B = 0).  A non-finite or negative target
// norm latches ERRBIT_NONFINITE.
__global__ void k_rb_norm(const double *__restrict__ q, const double *__restrict__ nu, int M,
                          double *__restrict__ scale, unsigned *__restrict__ err)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const double v = nu[k], qk = q[k];
    if (!(v >= 0.0) || !isfinite(v)) atomicOr(err, ERRBIT_NONFINITE);
    scale[k] = qk > 0.0 ? v / sqrt(qk) : 0.0;
}

// Coefficient operand (the MMA's B side), one warp per row: row k of tile k/256, column
// c = g * 2Nb + q holds part part_a(g) of 2^aexp[k] x_q, x_q = alpha_k,q (real parts for q < Nb,
// imaginary parts after; the renormalisation s_k is applied by the product's epilogue, so this
// pack does not wait for it).  The row's x_q are converted once (on the integer pipe) into shared
// memory, its largest magnitude sets aexp[k], then the lanes write its 16-byte chunks.  Rows past
// M are zero.
constexpr int kRbPackWarps = 8;

__global__ void __launch_bounds__(kRbPackWarps * 32)
k_rb_pack_a(const double *__restrict__ are, const double *__restrict__ aim, int M, int Nb, int n_kb,
            int m_tiles, unsigned char *__restrict__ apack, int *__restrict__ aexp)
{
    __shared__ float xs[kRbPackWarps][2 * FEW_MAX_BASIS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, Kr = 2 * Nb;
    float *x = xs[w];
    const int rows = m_tiles * kRbTileN, chunks = n_kb * (kRbTileK / 8);
    for (int row = blockIdx.x * kRbPackWarps + w; row < rows; row += gridDim.x * kRbPackWarps) {
        const bool live = row < M;
        float mx = 0.0f;
        for (int q = lane; q < Kr; q += 32) {
            x[q] = live ? f64_to_f32(q < Nb ? are[(size_t)row * Nb + q] : aim[(size_t)row * Nb + q - Nb])
                        : 0.0f;
            mx = fmaxf(mx, fabsf(x[q]));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int e = scale_exp(mx);
        const float f = pow2f(e);
        if (lane == 0) aexp[row] = e;
        __syncwarp();
        unsigned char *tile = apack + (size_t)(row / kRbTileN) * n_kb * kRbBBytes;
        for (int q8 = lane; q8 < chunks; q8 += 32) {
            const int c0 = q8 * 8;
            int g = c0 / Kr, q = c0 - g * Kr;  // segment and column of c0, then stepped
            uint32_t wv[4];
#pragma unroll
            for (int e2 = 0; e2 < 8; e2 += 2) {
                __half v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    v[h] = g < kRbParts ? split_part(x[q] * f, part_a(g)) : __float2half_rn(0.0f);
                    if (++q == Kr) { q = 0; ++g; }
                }
                wv[e2 / 2] = pack2(v[0], v[1]);
            }
            *reinterpret_cast<uint4 *>(tile + (size_t)(c0 / kRbTileK) * kRbBBytes +
                                       core_offset(row % kRbTileN, c0 % kRbTileK)) =
                make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        __syncwarp();
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

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), fp16 A and B (bits 7-9
// and 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kRbIdesc = (1u << 4) | ((uint32_t)(kRbTileN >> 3) << 17) | ((uint32_t)(kRbTileM >> 4) << 24);

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
    const unsigned char *apack;  // coefficients: [m_tiles][n_kb] blocks of kRbBBytes (B operand)
    const unsigned char *bpack;  // basis: [n_tiles][n_kb] blocks of kRbABytes (A operand)
    double *out_re, *out_im;     // [M][N]
    const int *aexp, *bexp;      // scaling exponents of the coefficient rows and basis columns
    const double *scale;         // [M] renormalisation s_k, applied in the epilogue (or null)
    int M, N, n_kb, m_tiles, n_tiles;
    int k16_last;                // K = 16 steps of the last k-block holding real columns
    unsigned *err;
};

constexpr int kRbEpiWarps = 16;  // four per tensor-memory lane quarter, every fourth 32-column chunk
constexpr int kRbEpiPerQuarter = kRbEpiWarps / 4;
constexpr int kRbMmaThreads = 64 + 32 * kRbEpiWarps;  // producer warp, MMA warp, epilogue warps
constexpr uint32_t kRbTmemCols = 2 * kRbTileN;         // two accumulator buffers

__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity)
{
    return __all_sync(0xffffffffu, mbar_wait_bounded(bar, parity));
}

// Persistent: CTA b takes tiles b, b + grid, ... (tile t = knot tile t / n_tiles, basis tile
// t % n_tiles).  Warp 0 (one lane) streams each tile's k-blocks through a kRbStages ring of
// shared-memory stages with bulk copies; warp 1 (one lane) issues the MMAs of a tile into one of
// two tensor-memory accumulators of 256 columns and commits; warps 2.. drain the other
// accumulator meanwhile: warp w reads lanes 32 (w % 4) .. + 31 (32 output columns: real parts
// for w % 4 < 2, imaginary parts otherwise) and one in kRbEpiPerQuarter chunks of 32 knots, and
// for each knot stores the 32 columns' FP64 values, 256 contiguous bytes, from registers.  Every wait is bounded; a timeout latches ERRBIT_TIMEOUT and the CTA waits
// for its copies and MMAs in flight before it frees tensor memory.
__global__ void __launch_bounds__(kRbMmaThreads, 1) k_rb_mma(RbMmaArgs a)
{
    extern __shared__ unsigned char rb_mma_smem[];
    __shared__ __align__(8) uint64_t full[kRbStages], empty[kRbStages], tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ uint32_t s_issued, s_consumed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int total = a.m_tiles * a.n_tiles;
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(rb_mma_smem) + 127) & ~(uintptr_t)127);
    unsigned char *sA = base, *sB = base + kRbStages * kRbABytes;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(kRbTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kRbStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kRbEpiWarps);
        }
        mbar_init(&drain, 1);
        fence_mbar_init();
        s_abort = 0;
        s_issued = s_consumed = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // producer
            const uint64_t keep = l2_evict_last_policy();  // operands are re-read by other CTAs
            uint32_t g = 0;
            for (int t = blockIdx.x; t < total && !s_abort; t += gridDim.x) {
                const unsigned char *ga = a.bpack + (size_t)(t % a.n_tiles) * a.n_kb * kRbABytes;  // basis
                const unsigned char *gb = a.apack + (size_t)(t / a.n_tiles) * a.n_kb * kRbBBytes;  // coefficients
                for (int kb = 0; kb < a.n_kb; ++kb, ++g) {
                    const int s = g % kRbStages;
                    if (!mbar_wait_bounded(&empty[s], ((g / kRbStages) & 1) ^ 1)) { s_abort = 1; break; }
                    mbar_arrive_expect_tx(&full[s], kRbStageBytes);
                    bulk_g2s_hint(sA + s * kRbABytes, ga + (size_t)kb * kRbABytes, kRbABytes, &full[s], keep);
                    bulk_g2s_hint(sB + s * kRbBBytes, gb + (size_t)kb * kRbBBytes, kRbBBytes, &full[s], keep);
                }
            }
            s_issued = g;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            uint32_t g = 0;
            int u = 0;
            for (int t = blockIdx.x; t < total && !s_abort; t += gridDim.x, ++u) {
                const int b = u & 1;
                if (!mbar_wait_bounded(&tempty[b], ((u >> 1) & 1) ^ 1)) { s_abort = 1; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kRbTileN);
                bool ok = true;
                for (int kb = 0; kb < a.n_kb; ++kb, ++g) {
                    const int s = g % kRbStages;
                    if (!mbar_wait_bounded(&full[s], (g / kRbStages) & 1)) { s_abort = 1; ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * kRbABytes), b0 = smem_u32(sB + s * kRbBBytes);
                    // the last k-block's columns past 3 x 2 Nb are zero: their MMAs are skipped
                    const int nk = kb + 1 < a.n_kb ? kRbTileK / 16 : a.k16_last;
#pragma unroll
                    for (int k = 0; k < kRbTileK / 16; ++k)  // K = 16 per MMA: two core matrices
                        if (k < nk)
                            tc_mma(d, smem_desc(a0 + k * 256, 128, 1024),
                                   smem_desc(b0 + k * 256, 128, 1024), kRbIdesc,
                                   (uint32_t)((kb | k) != 0));
                    tc_commit(&empty[s]);
                }
                if (!ok) break;
                tc_commit(&tfull[b]);
            }
            s_consumed = g;
            tc_commit(&drain);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {  // epilogue
        const int e = warp - 2, qd = warp & 3;  // a warp reads tensor-memory lanes 32 (warp % 4) ..
        const int c_first = e / 4;              // and chunks c_first + kRbEpiPerQuarter i
        int u = 0;
        for (int t = blockIdx.x; t < total && !__any_sync(0xffffffffu, s_abort != 0); t += gridDim.x, ++u) {
            const int b = u & 1;
            if (!warp_wait(&tfull[b], (u >> 1) & 1)) { s_abort = 1; break; }
            tc_fence_after();
            const int mode = (t % a.n_tiles) * kRbModes + (qd & 1) * 32 + lane;  // this lane's column
            double *dst = qd < 2 ? a.out_re : a.out_im;
            const float fb = pow2f(-a.bexp[mode]);  // undo the column scaling (exact)
            const int k0 = (t / a.n_tiles) * kRbTileN;
            for (int c = c_first; c < kRbTileN / 32; c += kRbEpiPerQuarter) {
                uint32_t v[32];
                tc_ld32(tmem + (uint32_t)(b * kRbTileN) + ((uint32_t)(32 * qd) << 16) + (uint32_t)(32 * c), v);
                const int kc = k0 + 32 * c;
                // knot kc + lane's row scaling (exact) times its renormalisation s_k
                float fa_lane = pow2f(-a.aexp[kc + lane]);
                if (a.scale && kc + lane < a.M) fa_lane *= (float)a.scale[kc + lane];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float fa = __shfl_sync(0xffffffffu, fa_lane, j);
                    if (kc + j < a.M && mode < a.N)  // streamed once: evict-first
                        __stcs(dst + (size_t)(kc + j) * a.N + mode, f32_to_f64(__uint_as_float(v[j]) * fb * fa));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }

    __syncthreads();
    if (!warp_wait(&drain, 0)) s_abort = 1;  // no MMA of this CTA still running
    if (tid == 0 && s_abort) {
        atomicOr(a.err, ERRBIT_TIMEOUT);
        for (uint32_t g = s_consumed; g < s_issued; ++g)  // let copies in flight land
            mbar_wait_bounded(&full[g % kRbStages], (g / kRbStages) & 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kRbTmemCols)
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
    L.n_tiles = (N + kRbModes - 1) / kRbModes;
    L.m_tiles = (M + kRbTileN - 1) / kRbTileN;
    L.modes_padded = L.n_tiles * kRbModes;
    L.rows_padded = L.m_tiles * kRbTileN;
    L.bpack_bytes = (size_t)L.n_tiles * L.n_kb * kRbABytes;
    L.apack_bytes = (size_t)L.m_tiles * L.n_kb * kRbBBytes;
    return L;
}

cudaError_t launch_rb_basis(const double *bre, const double *bim, int Nb, int N, double2 *gt64,
                            float2 *gt32, int *bexp, unsigned char *bpack, int sm_count, cudaStream_t st)
{
    const RbLayout L = rb_layout(Nb, N, 0);
    k_rb_gram<<<Nb * Nb, 128, 0, st>>>(bre, bim, Nb, N, gt64, gt32);
    k_rb_bexp<<<(L.modes_padded + 127) / 128, 128, 0, st>>>(bre, bim, Nb, N, L.modes_padded, bexp);
    k_rb_pack_b<<<sm_count * 8, 256, 0, st>>>(bre, bim, Nb, N, L.n_kb, L.n_tiles, bexp, bpack);
    return cudaGetLastError();
}

cudaError_t launch_rb(const double *are, const double *aim, int M, int Nb, int N, const double *nu,
                      bool fp64, const double *bre, const double *bim, const double2 *gt64,
                      const float2 *gt32, const int *bexp, const unsigned char *bpack, double *scale,
                      int *aexp, unsigned char *apack, double *ore, double *oim, unsigned *err,
                      int sm_count, cudaStream_t st, cudaStream_t side, cudaEvent_t fork_ev,
                      cudaEvent_t join_ev)
{
    if (M == 0) return cudaSuccess;
    const RbLayout L = rb_layout(Nb, N, M);
    cudaError_t e;
    const double *sc = nullptr;
    // mixed path: the scale is applied in the product's epilogue, so its kernels run on the side
    // stream beside the coefficient pack and are joined before the product
    const bool fork = nu && !fp64 && side;
    cudaStream_t ss = fork ? side : st;
    if (fork) {
        if ((e = cudaEventRecord(fork_ev, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, fork_ev, 0)) != cudaSuccess) return e;
    }
    // a failure after the fork waits for the side stream, so nothing of it outlives the call's
    // scratch, which the caller releases on `st`
    auto fail = [&](cudaError_t err) {
        if (fork) cudaStreamSynchronize(side);
        return err;
    };
    if (nu && !fp64 && Nb <= kTMaxBasis) {
        const int smem = (kTRows * Nb + Nb * kTJ) * (int)sizeof(float2);
        e = cudaFuncSetAttribute(k_rb_scale_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return fail(e);
        k_rb_scale_tile<<<(M + kTRows - 1) / kTRows, kTThreads, smem, ss>>>(are, aim, M, Nb, gt32, nu,
                                                                             scale, err);
        sc = scale;
    } else if (nu) {
        double *q = scale + M;  // the caller's scratch holds scale [M] then q [M]
        e = cudaMemsetAsync(q, 0, sizeof(double) * (size_t)M, ss);
        if (e != cudaSuccess) return fail(e);
        const dim3 grid((Nb + kQJ - 1) / kQJ, (M + kQRows - 1) / kQRows);
        if (fp64) {
            e = cudaFuncSetAttribute(k_rb_quad<double, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     rb_quad_smem<double2>());
            if (e != cudaSuccess) return fail(e);
            k_rb_quad<double, double2><<<grid, kQThreads, rb_quad_smem<double2>(), ss>>>(are, aim, M, Nb, gt64, q);
        } else {
            e = cudaFuncSetAttribute(k_rb_quad<float, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     rb_quad_smem<float2>());
            if (e != cudaSuccess) return fail(e);
            k_rb_quad<float, float2><<<grid, kQThreads, rb_quad_smem<float2>(), ss>>>(are, aim, M, Nb, gt32, q);
        }
        k_rb_norm<<<(M + 255) / 256, 256, 0, ss>>>(q, nu, M, scale, err);
        sc = scale;
    }
    if (fork && (e = cudaEventRecord(join_ev, side)) != cudaSuccess) return fail(e);
    if (fp64) {
        dim3 grid((N + kRb64Modes - 1) / kRb64Modes, (M + kRb64Rows - 1) / kRb64Rows);
        k_rb_fp64<<<grid, 256, 0, st>>>(are, aim, bre, bim, M, Nb, N, sc, ore, oim);
        return cudaGetLastError();
    }
    const int rows = L.m_tiles * kRbTileN;
    const int pgrid = (rows + kRbPackWarps - 1) / kRbPackWarps;
    k_rb_pack_a<<<pgrid < sm_count * 8 ? pgrid : sm_count * 8, kRbPackWarps * 32, 0, st>>>(
        are, aim, M, Nb, L.n_kb, L.m_tiles, apack, aexp);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    if (fork && (e = cudaStreamWaitEvent(st, join_ev, 0)) != cudaSuccess) return fail(e);
    const int smem = kRbStages * (int)kRbStageBytes + 128;
    e = cudaFuncSetAttribute(k_rb_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int tiles = L.m_tiles * L.n_tiles;
    const int k_last = kRbParts * 2 * Nb - (L.n_kb - 1) * kRbTileK;  // real columns, last block
    RbMmaArgs args{apack, bpack, ore, oim, aexp, bexp, sc, M, N, L.n_kb, L.m_tiles, L.n_tiles,
                   (k_last + 15) / 16, err};
    k_rb_mma<<<tiles < sm_count ? tiles : sm_count, kRbMmaThreads, smem, st>>>(args);
    return cudaGetLastError();
}

}  // namespace fewsum
