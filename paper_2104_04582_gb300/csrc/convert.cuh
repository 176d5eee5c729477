// convert.cuh -- number conversions that stay off GB300's narrow FP64 pipe.
#pragma once

namespace fewsum {

// FP64 -> FP32 with round-to-nearest-even, on the integer pipe.  GB300 runs FP64 -> FP32
// conversions on its narrow FP64 pipe, which would bound the mixed-precision kernels; the bit
// arithmetic keeps them on the integer and FP32 pipes.  Magnitudes below 2^-126 flush to a signed
// zero; finite overflow, inf and nan give a signed infinity (inputs here are finite amplitudes
// and harmonics).  Written with early returns only: every branch is a select, so the callers'
// loads stay hoisted ahead of the arithmetic.
__device__ __forceinline__ float f64_to_f32(double d)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
    const unsigned int hi = static_cast<unsigned int>(b >> 32), lo = static_cast<unsigned int>(b);
    const unsigned int sign = hi & 0x80000000u;
    const int fe = static_cast<int>((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
    unsigned int f = sign | (static_cast<unsigned int>(fe) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned int rem = lo & 0x1fffffffu, half = 0x10000000u;
    if (rem > half || (rem == half && (f & 1u))) f += 1u;  // a carry rounds into the exponent
    return __uint_as_float(f);
}

// Branchless FP64 -> FP32 for streaming kernels: round to nearest with ties away from zero (a
// 64-bit add of half a float ulp, then truncation; it differs from the even-tie cast only on exact
// ties), exponent rebiased and shifted into place by one funnel shift.  Classified on the
// unrounded bits: magnitudes below 2^-126 give a signed zero (also the few just below that would
// round up to it), magnitudes from 2^128 up, inf and nan give a signed infinity.
__device__ __forceinline__ float f64_to_f32_fast(double d)
{
    const unsigned long long raw = static_cast<unsigned long long>(__double_as_longlong(d));
    const unsigned int rhi = static_cast<unsigned int>(raw >> 32), rmag = rhi & 0x7fffffffu;
    const unsigned int sign = rhi & 0x80000000u;
    const unsigned long long b = raw + 0x10000000ull;
    const unsigned int hi = static_cast<unsigned int>(b >> 32), lo = static_cast<unsigned int>(b);
    unsigned int f = __funnelshift_l(lo, hi - (896u << 20), 3) | sign;
    f = rmag < (897u << 20) ? sign : f;
    f = rmag >= (1151u << 20) ? (sign | 0x7f800000u) : f;
    return __uint_as_float(f);
}

// FP32 -> FP64 on the integer pipe: exact for normal floats (rebias the exponent 127 -> 1023,
// widen the significand); zero and subnormal inputs give a signed zero, inf and nan stay so.
__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned int u = __float_as_uint(x), sign = u & 0x80000000u;
    const unsigned int e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned int hi = sign | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
    if (e == 0u) hi = sign, lo = 0u;
    if (e == 255u) hi = sign | 0x7ff00000u | (m >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

}  // namespace fewsum
