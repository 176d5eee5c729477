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

}  // namespace fewsum
