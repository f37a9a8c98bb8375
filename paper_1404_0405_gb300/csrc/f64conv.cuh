// FP64 -> FP32 rounding (to nearest, ties to even) with integer operations only.
//
// The spherical geometry is kept in FP64 on the device and rounded to FP32 where
// the FP32 form's stencils use it.  On this GPU the FP64 pipe runs at a small
// fraction of the FP32 rate, and a conversion instruction occupies it; this
// rounding is written from the binary64/binary32 encodings (IEEE 754) instead and
// runs on the integer pipe: keep the sign, rebias the exponent (1023 -> 127), keep
// the 23 leading fraction bits and round on the 29 dropped ones (above half: up;
// exactly half: up when the kept fraction is odd), letting a carry run into the
// exponent.  It covers results that are normal FP32 numbers and zero; anything
// else (|x| below 2^-126 or at least 2^128, infinities, NaN) goes to the FP64
// conversion instruction.
#pragma once

// the values outside the fast path, through the conversion instruction (a call, so
// that the instruction is not issued, predicated off, on the fast path)
__device__ __noinline__ float f64_to_f32_rn_slow(double x) { return __double2float_rn(x); }

__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned hi = static_cast<unsigned>(__double2hiint(x));
    const unsigned lo = static_cast<unsigned>(__double2loint(x));
    const unsigned e = (hi >> 20) & 0x7ffu;
    // normal FP32 results: biased FP64 exponent 897..1150
    if (e - 897u > 253u) return ((hi << 1) | lo) == 0u ? __uint_as_float(hi) : f64_to_f32_rn_slow(x);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);   // 23 kept fraction bits
    // +1 when the 29 dropped bits are above half, or exactly half with m odd; a carry
    // runs into the exponent (at the top of the range it gives infinity, which is
    // also the correctly rounded result)
    const unsigned inc = ((lo & 0x1fffffffu) + 0x0fffffffu + (m & 1u)) >> 29;
    return __uint_as_float((hi & 0x80000000u) | (((e - 896u) << 23) + m + inc));
}
