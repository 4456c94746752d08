// da_fixed.cuh -- conversions between fp32 and the fixed-point grid 2^-S of
// the exact field recompute, in integer arithmetic.
//
// The recompute's definition is  v = round(w 2^S)  (to nearest, ties to even)
// for every coefficient and  g = fl32(sum) 2^-S  for every field.  Written with
// the 64-bit conversions of the instruction set (__float2ll_rn, __ll2float_rn)
// those run on the fp64 pipe, which is a small fraction of the fp32 rate on
// this GPU; the versions below use the integer and fp32 pipes only and return
// the same bits for every argument the recompute produces.
#pragma once
#include <cstdint>

namespace da {

// round(w 2^S) for finite w with |w 2^S| < 2^63; equal to
// __float2ll_rn(ldexpf(w, S)) (values whose scaled magnitude is below 1/2,
// including those that ldexpf would round to subnormals, give 0 both ways).
__device__ __forceinline__ long long fixed_of_f32(float w, int S)
{
    const uint32_t b = __float_as_uint(w);
    const uint32_t E = (b >> 23) & 0xFFu;
    const uint32_t m = E ? ((b & 0x7FFFFFu) | 0x800000u) : (b & 0x7FFFFFu);
    const int sh = (E ? (int)E : 1) - 150 + S;   // |w| 2^S = m 2^sh
    unsigned long long mag;
    if (sh >= 0) {
        mag = (unsigned long long)m << sh;
    } else if (sh <= -25) {
        mag = 0;                                 // m 2^sh < 1/2
    } else {
        const int rs = -sh;
        const uint32_t q = m >> rs;
        const uint32_t rem = m & ((1u << rs) - 1u);
        const uint32_t half = 1u << (rs - 1);
        mag = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
    }
    return (b >> 31) ? -(long long)mag : (long long)mag;
}

// round(w 2^S) for w = 0 or a normal number with (exponent field - 150 + S) >= 0,
// i.e. when w 2^S is an integer (the significand shifted left): equal to
// fixed_of_f32(w, S) there, without its rounding path.
__device__ __forceinline__ long long fixed_of_f32_shift(float w, int S)
{
    const uint32_t b = __float_as_uint(w);
    const uint32_t E = (b >> 23) & 0xFFu;
    const uint32_t m = E ? ((b & 0x7FFFFFu) | 0x800000u) : 0u;
    const int sh = E ? (int)E - 150 + S : 0;
    const unsigned long long mag = (unsigned long long)m << sh;
    return (b >> 31) ? -(long long)mag : (long long)mag;
}

// fl32(v) 2^-S: v rounded to fp32 (to nearest, ties to even), then scaled;
// equal to ldexpf(__ll2float_rn(v), -S).  Results outside the normal range
// are left to ldexpf.
__device__ __forceinline__ float scaled_f32_of(long long v, int S)
{
    if (v == 0) return 0.f;
    const uint32_t sign = v < 0 ? 0x80000000u : 0u;
    const unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    int e = 63 - __clzll((long long)u);          // u in [2^e, 2^(e+1))
    uint32_t mant;
    if (e <= 23) {
        mant = (uint32_t)(u << (23 - e));
    } else {
        const int rs = e - 23;
        const unsigned long long q = u >> rs;
        const unsigned long long rem = u & ((1ull << rs) - 1ull);
        const unsigned long long half = 1ull << (rs - 1);
        mant = (uint32_t)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
        if (mant == (1u << 24)) {
            mant >>= 1;
            ++e;
        }
    }
    const int be = e - S + 127;
    if (be >= 1 && be <= 254) return __uint_as_float(sign | ((uint32_t)be << 23) | (mant & 0x7FFFFFu));
    return ldexpf(__uint_as_float(sign | ((uint32_t)(e + 127) << 23) | (mant & 0x7FFFFFu)), -S);
}

// The integer value of an fp32 that holds an integer of magnitude < 2^22
// (the tensor cores' digit sums): adding 1.5 2^23 puts it in the mantissa.
__device__ __forceinline__ int small_int_of(float f)
{
    return __float_as_int(__fadd_rn(f, 12582912.0f)) - 0x4B400000;
}

}  // namespace da
