// probe.cu -- measured throughput of the arithmetic pipes the summation kernels use.
//
// The roofline of the summation is set by plain ALU pipes, not by HBM or tensor cores: FP32 FMA
// (mixed path), FP64 FMA (plain path) and the SFU.  Each probe runs many independent dependency
// chains per thread over a grid of several CTAs per SM, long enough (tens of ms) to reach the
// clocks of a sustained load, and reports operations per second timed with CUDA events.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T *out, int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == (T)12345.678) out[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_sfu(float *out, int iters)
{
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = __sinf(a[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// Every FMA reads three distinct registers (no constant-bank operand).
__global__ void __launch_bounds__(256) k_fma_regs(float *out, const float *in, int iters)
{
    float a[kChains], b[kChains], c[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        a[j] = in[(threadIdx.x + j) & 255];
        b[j] = in[(threadIdx.x + 3 * j + 1) & 255];
        c[j] = in[(threadIdx.x + 5 * j + 2) & 255];
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b[j], c[(j + 1) % kChains]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// Packed FP32x2 FMA with three distinct register pairs.
__global__ void __launch_bounds__(256) k_fma2_regs(float *out, const float *in, int iters)
{
    float2 a[kChains], b[kChains], c[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        a[j] = make_float2(in[(threadIdx.x + j) & 255], in[(threadIdx.x + j + 7) & 255]);
        b[j] = make_float2(in[(threadIdx.x + 3 * j + 1) & 255], in[(threadIdx.x + 2 * j) & 255]);
        c[j] = make_float2(in[(threadIdx.x + 5 * j + 2) & 255], in[(threadIdx.x + j + 9) & 255]);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], b[j], c[(j + 1) % kChains]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j].x + a[j].y;
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// The Horner form of the summation: distinct accumulator and multiplier registers, one addend
// register shared by consecutive FMAs (the slot coefficient is common to a thread's samples).
__global__ void __launch_bounds__(256) k_fma_shared_c(float *out, const float *in, int iters)
{
    float a[kChains], b[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        a[j] = in[(threadIdx.x + j) & 255];
        b[j] = in[(threadIdx.x + 3 * j + 1) & 255];
    }
    float c0 = in[(threadIdx.x + 2) & 255], c1 = in[(threadIdx.x + 5) & 255];
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b[j], c0);
        const float t = c0;  // rotate the shared addend so it is not loop-invariant
        c0 = c1;
        c1 = t;
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

// The summation's per-slot block for 4 samples: each slot's 8 coefficients read from a shared-
// memory table (as the summation kernel reads its per-segment table), two cubics in u (the
// coefficients common to the samples) and the complex step a <- a z + K: 40 FMAs per slot.
// The instruction order is the compiler's: stage-major orders, z as the first multiplicand and
// 8 samples per thread all measured within 10 % of this form.
__global__ void __launch_bounds__(256) k_horner4(float *out, const float *in, int iters)
{
    __shared__ float4 tab[64][2];
    for (int e = threadIdx.x; e < 128; e += blockDim.x)
        tab[e >> 1][e & 1] = make_float4(in[(e * 4) & 255], in[(e * 4 + 1) & 255], in[(e * 4 + 2) & 255],
                                         in[(e * 4 + 3) & 255]);
    __syncthreads();
    float u[4], zr[4], zi[4], ar[4], ai[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        u[r] = in[(threadIdx.x + r) & 255];
        zr[r] = in[(threadIdx.x + 3 * r + 1) & 255];
        zi[r] = in[(threadIdx.x + 5 * r + 2) & 255];
        ar[r] = ai[r] = 0.f;
    }
    for (int i = 0; i < iters; ++i) {
        const float4 lo = tab[i & 63][0], hi = tab[i & 63][1];
        const float c[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float kr = fmaf(fmaf(fmaf(c[3], u[r], c[2]), u[r], c[1]), u[r], c[0]);
            const float ki = fmaf(fmaf(fmaf(c[7], u[r], c[6]), u[r], c[5]), u[r], c[4]);
            const float nr = fmaf(ar[r], zr[r], fmaf(-ai[r], zi[r], kr));
            const float ni = fmaf(ar[r], zi[r], fmaf(ai[r], zr[r], ki));
            ar[r] = nr;
            ai[r] = ni;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) s += ar[r] + ai[r];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" {

// which: 0 = FP32 FMA, 1 = FP64 FMA, 2 = SFU sine (__sinf), 3 = FP32 FMA with three register
// operands, 4 = packed FP32x2 FMA with three register pairs (counts 2 operations each), 5 = FP32
// FMA with distinct accumulator and multiplier registers and a shared addend register, 6 = the
// summation's per-slot block for 4 samples (40 FMAs per iteration).  Returns 0 on success and writes the
// measured rate (operations per second; an FMA counts as one operation) and the elapsed ms.
int fewprobe_measure(int device, int which, int iters, double *ops_per_s, float *ms_out)
{
    if (which < 0 || which > 6) return 1;
    if (cudaSetDevice(device) != cudaSuccess) return 1;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
    const int threads = 256, blocks = sms * 8;
    float *out = nullptr, *in = nullptr;
    if (cudaMalloc(&out, sizeof(float) * 2 * blocks) != cudaSuccess) return 1;
    if (cudaMalloc(&in, sizeof(float) * 256) != cudaSuccess) return 1;
    cudaMemset(in, 0, sizeof(float) * 256);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int it) {
        if (which == 0) k_fma<float><<<blocks, threads, 0, st>>>(out, it, 0.9999f, 1e-4f);
        else if (which == 1)
            k_fma<double><<<blocks, threads, 0, st>>>(reinterpret_cast<double *>(out), it, 0.9999, 1e-4);
        else if (which == 2) k_sfu<<<blocks, threads, 0, st>>>(out, it);
        else if (which == 3) k_fma_regs<<<blocks, threads, 0, st>>>(out, in, it);
        else if (which == 4) k_fma2_regs<<<blocks, threads, 0, st>>>(out, in, it);
        else if (which == 5) k_fma_shared_c<<<blocks, threads, 0, st>>>(out, in, it);
        else k_horner4<<<blocks, threads, 0, st>>>(out, in, it);
    };
    launch(iters / 8 + 1);  // warm-up
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    int rc = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = 1;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(out);
    cudaFree(in);
    if (cudaGetLastError() != cudaSuccess) rc = 1;
    if (rc) return rc;
    *ms_out = ms;
    const double per_iter = which == 6 ? 40.0 : (double)kChains * (which == 4 ? 2 : 1);
    *ops_per_s = (double)blocks * threads * (double)iters * per_iter /
                 (ms * 1e-3);
    return 0;
}

}  // extern "C"
